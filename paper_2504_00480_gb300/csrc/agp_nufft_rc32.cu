// Spreading and interpolation kernels instantiated for a block of 32
// right-hand sides (see agp_nufft_kernels.cuh).
#include "agp_nufft_kernels.cuh"

namespace agp {
AGP_NUFFT_RC_DEFINE(float, 32)
}  // namespace agp
