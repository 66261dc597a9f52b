// FFT passes instantiated for transform length 80.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(80)
}  // namespace csngf
