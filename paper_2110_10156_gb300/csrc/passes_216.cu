// FFT passes instantiated for transform length 216.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(216)
}  // namespace csngf
