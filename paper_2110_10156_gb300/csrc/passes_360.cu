// FFT passes instantiated for transform length 360.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(360)
}  // namespace csngf
