// FP32 two-step register apply passes, lengths 384-512.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V2(384)
    FSA_REG_V2(512)
)
