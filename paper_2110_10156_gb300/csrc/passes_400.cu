// FFT passes instantiated for transform length 400.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(400)
}  // namespace csngf
