// Native FP64 apply passes, every supported length.
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
    FSA_REG_V1(fsa::kArithF64, double2, 192)
    FSA_REG_V1(fsa::kArithF64, double2, 256)
    FSA_REG_V1(fsa::kArithF64, double2, 384)
    FSA_REG_V1(fsa::kArithF64, double2, 512)
    FSA_REG_V1(fsa::kArithF64, double2, 768)
    FSA_REG_V1(fsa::kArithF64, double2, 1024)
)
