// FP32 two-step register apply passes, lengths 192-256.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V2(192)
    FSA_REG_V2(256)
)
