// Spreading and interpolation kernels instantiated for a block of 1
// right-hand side (see agp_nufft_kernels.cuh).
#include "agp_nufft_kernels.cuh"

namespace agp {
AGP_NUFFT_RC_DEFINE(float, 1)
AGP_NUFFT_RC_DEFINE(double, 1)
}  // namespace agp
