// Instantiation of the interpolation-with-gradient kernels: double, d = 3 (interp_grad.cuh).
#include "interp_grad.cuh"

namespace nufft {
NUFFT_DEFINE_GRAD(f64, double, 3)
}  // namespace nufft
