// Instantiation of the interpolation-with-gradient kernels: double, d = 1 (interp_grad.cuh).
#include "interp_grad.cuh"

namespace nufft {
NUFFT_DEFINE_GRAD(f64, double, 1)
}  // namespace nufft
