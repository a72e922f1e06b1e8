// FP32 first-generation (Stockham radix-8) apply passes, lengths 192-1024.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V1(fsa::kArithF32G1, float2, 192)
    FSA_REG_V1(fsa::kArithF32G1, float2, 256)
    FSA_REG_V1(fsa::kArithF32G1, float2, 384)
    FSA_REG_V1(fsa::kArithF32G1, float2, 512)
    FSA_REG_V1(fsa::kArithF32G1, float2, 768)
    FSA_REG_V1(fsa::kArithF32G1, float2, 1024)
)
