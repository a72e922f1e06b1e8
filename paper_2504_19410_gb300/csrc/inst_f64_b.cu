// Native FP64 apply passes, lengths 192-1024.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V1(fsa::kArithF64, double2, 192)
    FSA_REG_V1(fsa::kArithF64, double2, 256)
    FSA_REG_V1(fsa::kArithF64, double2, 384)
    FSA_REG_V1(fsa::kArithF64, double2, 512)
    FSA_REG_V1(fsa::kArithF64, double2, 768)
    FSA_REG_V1(fsa::kArithF64, double2, 1024)
)
