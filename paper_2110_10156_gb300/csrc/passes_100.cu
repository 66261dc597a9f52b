// FFT passes instantiated for transform length 100.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(100)
}  // namespace csngf
