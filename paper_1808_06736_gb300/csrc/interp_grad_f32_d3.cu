// Instantiation of the interpolation-with-gradient kernels: float, d = 3 (interp_grad.cuh).
#include "interp_grad.cuh"

namespace nufft {
NUFFT_DEFINE_GRAD(f32, float, 3)
}  // namespace nufft
