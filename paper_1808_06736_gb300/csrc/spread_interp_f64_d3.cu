// Instantiations of the spread / interp kernels for double data in 3D, all
// kernel widths w = 2..16 (one translation unit per precision and dimension
// so the build compiles them in parallel).
#include "spread_interp.cuh"

namespace nufft {
NUFFT_DEFINE_SI(f64, double, 3)
}  // namespace nufft
