// FP32 two-step register apply passes, lengths 8-48.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V2(8)
    FSA_REG_V2(12)
    FSA_REG_V2(16)
    FSA_REG_V2(24)
    FSA_REG_V2(32)
    FSA_REG_V2(48)
)
