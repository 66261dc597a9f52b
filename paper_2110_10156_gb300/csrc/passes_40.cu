// FFT passes instantiated for transform length 40.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(40)
}  // namespace csngf
