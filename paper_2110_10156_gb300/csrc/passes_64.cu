// FFT passes instantiated for transform length 64.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(64)
}  // namespace csngf
