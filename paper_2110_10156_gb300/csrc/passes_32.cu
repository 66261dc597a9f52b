// FFT passes instantiated for transform length 32.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(32)
}  // namespace csngf
