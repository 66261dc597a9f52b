// FFT passes instantiated for transform length 512.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(512)
}  // namespace csngf
