// FFT passes instantiated for transform length 256.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(256)
}  // namespace csngf
