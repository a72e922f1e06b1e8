// Double-word apply passes, lengths 8-24.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 8)
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 12)
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 16)
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 24)
)
