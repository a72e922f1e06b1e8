// Native FP64 apply passes, lengths 8-128.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V1(fsa::kArithF64, double2, 8)
    FSA_REG_V1(fsa::kArithF64, double2, 12)
    FSA_REG_V1(fsa::kArithF64, double2, 16)
    FSA_REG_V1(fsa::kArithF64, double2, 24)
    FSA_REG_V1(fsa::kArithF64, double2, 32)
    FSA_REG_V1(fsa::kArithF64, double2, 48)
    FSA_REG_V1(fsa::kArithF64, double2, 64)
    FSA_REG_V1(fsa::kArithF64, double2, 96)
    FSA_REG_V1(fsa::kArithF64, double2, 128)
)
