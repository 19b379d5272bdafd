// Instantiations of the spread / interp kernels for float data in 3D, all
// kernel widths w = 2..16 (one translation unit per precision and dimension
// so the build compiles them in parallel).
#include "spread_interp.cuh"

namespace nufft {
NUFFT_DEFINE_SI(f32, float, 3)
}  // namespace nufft
