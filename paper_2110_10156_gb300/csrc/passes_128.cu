// FFT passes instantiated for transform length 128.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(128)
}  // namespace csngf
