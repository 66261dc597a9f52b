// FFT passes instantiated for transform length 16.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(16)
}  // namespace csngf
