// FP64 instances of the apply passes (double2 complex, 8 lines per tile).
#include "passes_impl.cuh"

namespace fsa {
template struct Passes<double2>;
}
