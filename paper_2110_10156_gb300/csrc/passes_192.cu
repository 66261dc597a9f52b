// FFT passes instantiated for transform length 192.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(192)
}  // namespace csngf
