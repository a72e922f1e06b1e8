// FP32 instances of the apply passes (float2 complex, 16 lines per tile).
#include "passes_impl.cuh"

namespace fsa {
template struct Passes<float2>;
}
