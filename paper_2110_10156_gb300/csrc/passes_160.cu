// FFT passes instantiated for transform length 160.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(160)
}  // namespace csngf
