// FFT passes instantiated for transform length 200.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(200)
}  // namespace csngf
