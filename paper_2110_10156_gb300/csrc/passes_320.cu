// FFT passes instantiated for transform length 320.
#include "passes.cuh"

namespace csngf {
CSNGF_INSTANTIATE_PASSES(320)
}  // namespace csngf
