// Instantiation of the interpolation-with-gradient kernels: float, d = 2 (interp_grad.cuh).
#include "interp_grad.cuh"

namespace nufft {
NUFFT_DEFINE_GRAD(f32, float, 2)
}  // namespace nufft
