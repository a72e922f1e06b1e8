// Double-word apply passes, lengths 96-128.
// Compiled as its own translation unit so that the library's kernel
// instances build in parallel; registers its launchers at library load.
#include "passes_impl.cuh"

FSA_REGISTER(
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 96)
    FSA_REG_V1(fsa::kArithDW, fsa::cdw, 128)
)
