// Internal declarations shared by the translation units of libnufft_gb300.
// Nothing here is part of the C ABI (include/nufft_gb300.h is).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>

#include "../../include/nufft_gb300.h"

namespace nufft {

// Geometry of the fine grid, the bins and the shared-memory tiles; passed by
// value to every kernel.  Dimensions above d have n = B = T = nb = 1.
struct Geom {
  int d;         // 1, 2 or 3
  int w;         // kernel width in fine-grid cells
  int half;      // floor(w / 2): tile origin = bin origin - half
  int n[3];      // fine-grid size per dimension
  int B[3];      // bin extent per dimension
  int nb[3];     // bins per dimension = ceil(n / B)
  int T[3];      // tile extent per dimension = B + w
  int sb[3];     // bins per super-block per dimension (powers of two)
  int lsb[3];    // log2(sb)
  int ns[3];     // super-blocks per dimension = ceil(nb / sb)
  int nbins;     // bin ids in use: ns[0] ns[1] ns[2] sb[0] sb[1] sb[2] (ids of padding bins stay empty)
  int ntile;     // T[0] T[1] T[2]
  int maxsub;    // most points in one subproblem
  int sparse_max;  // subproblems with at most this many points take the per-warp path (0: none)
  int horner;      // 1: kernel values from the piecewise polynomial of Sec. 5.3 (horner_table)
  int kernel;      // 0: the ES kernel, Eq. (ES); 1: 2 e^-beta cosh(beta sqrt(1 - z^2)) (Remark in Sec. 7)
  // Bank-grouped tile layout of the 3D kernels for even w (0 when it does not apply): rows of qs0
  // cells (qs0 = 8 mod 16, at least T[0] + 1: the tile's x-origin is rounded down to an even grid
  // index), qt1 rows per plane (qt1 = w mod 4, at least T[1]), qtile = qs0 qt1 T[2] cells.  With
  // these strides the cell of stencil row rho = l1 + w l2 lies rho qs0 cells (mod 32) after the
  // row start, which the quad spread and paired interpolation orders rely on.
  int qs0, qt1, qtile;
};
// true when the bank-grouped tile layout applies (3D, even w)
__host__ __device__ __forceinline__ bool quad_layout(const Geom& g) { return g.qs0 > 0; }
// Dynamic shared memory of the bank-grouped complex64 kernels (each with 128 bytes of slack to
// align the tile for TMA).  Spread: re and im planes of qtile ints, maxsub staged strengths, the
// gapless point order (3 maxsub shorts).  Interp: the tile (qtile float2), the point order.
__host__ __device__ inline size_t spread_q_bytes(const Geom& g) {
  // the spread's gapless point order needs 3 maxsub shorts (the interpolation's aligned one 5)
  return 128 + 2 * (size_t)g.qtile * 4 + (((size_t)g.maxsub * 8 + (size_t)g.maxsub * 3 * 2 + 15) & ~(size_t)15);
}
__host__ __device__ inline size_t interp_q_bytes(const Geom& g) {
  return 128 + (size_t)g.qtile * 8 + (size_t)g.maxsub * 5 * 2;
}
// The complex128 spread with 32-bit fixed-point words (spread_dw.cuh) runs kernel widths up to
// kDwMaxW, one block of 512 threads per SM.  Its shared memory: six int planes of ntile cells
// (rounded up to 16 bytes), maxsub staged strengths, the gapless point order (3 maxsub shorts).
constexpr int kDwMaxW = 12;
__host__ __device__ inline size_t spread_dw_bytes(const Geom& g) {
  return ((6 * (size_t)g.ntile * 4 + 15) & ~(size_t)15) + (size_t)g.maxsub * 16 + (size_t)g.maxsub * 3 * 2;
}

// Bin ids run over super-blocks of sb[0] x sb[1] x sb[2] bins, dimension 1
// fastest inside a super-block and across super-blocks.  Subproblems are
// processed in id order, so neighbouring bins -- whose tiles overlap in their
// halos -- are handled close together in time and their fine-grid lines are
// still in L2.
__host__ __device__ __forceinline__ int bin_id(const Geom& g, int b0, int b1, int b2) {
  const int s0 = b0 >> g.lsb[0], s1 = b1 >> g.lsb[1], s2 = b2 >> g.lsb[2];
  const int l0 = b0 & (g.sb[0] - 1), l1 = b1 & (g.sb[1] - 1), l2 = b2 & (g.sb[2] - 1);
  const int sup = (s2 * g.ns[1] + s1) * g.ns[0] + s0;
  return (((sup << g.lsb[2]) + l2) << (g.lsb[1] + g.lsb[0])) + (l1 << g.lsb[0]) + l0;
}
__host__ __device__ __forceinline__ void bin_coords(const Geom& g, int id, int* b) {
  const int sbv = g.sb[0] * g.sb[1] * g.sb[2];
  int s = id / sbv, l = id - s * sbv;
  const int l0 = l % g.sb[0];
  l /= g.sb[0];
  const int l1 = l % g.sb[1], l2 = l / g.sb[1];
  const int s0 = s % g.ns[0];
  s /= g.ns[0];
  const int s1 = s % g.ns[1], s2 = s / g.ns[1];
  b[0] = s0 * g.sb[0] + l0;
  b[1] = s1 * g.sb[1] + l1;
  b[2] = s2 * g.sb[2] + l2;
}
// Fill T, nb, sb, ns, ntile, nbins from d, w, n and B.
void finish_geom(Geom& g);

// One binned point: coordinates relative to the origin of its bin, in units
// of fine-grid cells (v in [0, B)), and its index in the caller's arrays.
struct alignas(16) RecF {
  float v[3];
  int idx;
};
struct alignas(16) RecD {
  double v[3];
  int idx;
  int pad;
};

template <typename T>
struct Traits;
template <>
struct Traits<float> {
  using C = float2;
  using Rec = RecF;
};
template <>
struct Traits<double> {
  using C = double2;
  using Rec = RecD;
};

// Per-transform geometry of a batch of transforms that share d, w, the bin
// extents B (so tiles have one size) and precision, but not their mode counts.
struct BatchGeom {
  int n[3], nb[3], ns[3], sb[3], lsb[3];
  int N[3];
  int nbins;          // bin ids of this transform
  int boff;           // its first global bin id
  long long goff;     // its fine grid within the batch grid (complex elements)
  long long moff;     // its modes within the batch mode array (complex elements)
  int pkoff[3];       // its correction factors within the batch factor array
  long long growoff;  // its first fine-grid row (n_2 n_3 rows) among all transforms
  long long mrowoff;  // its first mode row (N_2 N_3 rows) among all transforms
  double fs[3];       // n / (2 pi) per dimension, and its float hi / lo split
  float fs_hi[3], fs_lo[3];
};
// Passed to the kernels; B = 0 means a single transform (no table).
struct BatchTable {
  const BatchGeom* bg;  // [B]
  const int* boff;      // [B + 1] first global bin id of each transform
  const int* poff;      // [B + 1] first point of each transform
  const long long* growoff;  // [B + 1]
  const long long* mrowoff;  // [B + 1]
  int B;
};

// index t with first[t] <= key < first[t + 1] (first ascending, first[0] = 0)
template <typename I>
__host__ __device__ __forceinline__ int batch_find(const I* first, int B, I key) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= key) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__host__ __device__ __forceinline__ void batch_apply(Geom& g, const BatchGeom& t) {
  for (int i = 0; i < 3; ++i) {
    g.n[i] = t.n[i];
    g.nb[i] = t.nb[i];
    g.ns[i] = t.ns[i];
    g.sb[i] = t.sb[i];
    g.lsb[i] = t.lsb[i];
  }
  g.nbins = t.nbins;
}

// Device arrays produced by setpts and read by spread / interp.
struct Sorted {
  const void* rec;     // RecF / RecD [M], in bin order
  const int* sub_bin;  // [nsub] bin of each subproblem
  const int* sub_pt0;  // [nsub] first record of each subproblem
  const int* sub_cnt;  // [nsub] number of records
  const int* nsub;     // device scalar: tiled subproblems, list entries [0, nsub)
  const int* nsparse;  // device scalar: per-warp subproblems, entries [nsub, nsub + nsparse)
  int* err = nullptr;  // device error word (NUFFT_ERR_*) a kernel sets when a bounded wait runs out
};

// --- setpts (binsort.cu) ------------------------------------------------------
struct FoldConst {  // n / (2 pi) per dimension split into a hi and lo part
  double s[3];
  float s_hi[3];
  float s_lo[3];
};
FoldConst make_fold_const(const Geom& g);

// Replicated bin counters / scatter cursors (nrep a power of two; nrep <= 1:
// none, bin_count and cursor are used directly).  count and cursor hold
// nrep * nbins ints, replica-major.
struct Replicas {
  int nrep;
  int* count;
  int* cursor;
};
// replicas for nbins bins: up to 32, at most about 4M counters in all
inline int replicas_for(long long nbins) {
  int r = 32;
  while (r > 1 && (long long)r * nbins > (4LL << 20)) r >>= 1;
  return r;
}

// Enqueue the whole setpts pipeline.  Work arrays are owned by the plan.
cudaError_t launch_setpts(bool dbl, const Geom& g, const FoldConst& fc, int64_t M, const void* x,
                          const void* y, const void* z, int chkbnds, int* bin_count, int* bin_start,
                          int* sub_first, int* cursor, void* rec, int* sub_bin, int* sub_pt0,
                          int* sub_cnt, int* nsub, int* nsparse, int* err, cudaStream_t st,
                          cudaEvent_t* ev /* 4 events or nullptr */,
                          const BatchTable& bt = BatchTable{nullptr, nullptr, nullptr, nullptr, nullptr, 0},
                          int nbins = 0 /* bin ids over all transforms; 0: g.nbins */,
                          const Replicas& rp = Replicas{1, nullptr, nullptr});

// --- spread / interp (spread_interp_*.cu) --------------------------------------
struct LaunchCfg {
  int threads;
  int blocks;   // persistent grid
  size_t smem;  // dynamic shared memory bytes
  // interpolation only: a tensor map (CUtensorMap, 128 bytes) over the plan's own fine grid as
  // float pairs, box of one bank-grouped tile; NULL: tiles are fetched with per-cell copies
  const void* tmap = nullptr;
};
// Encode *tmap (a CUtensorMap) for TMA loads of bank-grouped tiles from a complex64 fine grid
// of g.n cells (this GPU's own memory).  Returns false when the layout or the driver does not allow it.
bool encode_tile_map(const Geom& g, const void* grid, void* tmap);
// smem bytes a spread / interp kernel needs for this geometry
size_t spread_smem_bytes(bool dbl, const Geom& g, int threads);
size_t interp_smem_bytes(bool dbl, const Geom& g, int threads);
// configure (max dynamic smem attribute) and size the persistent grid
cudaError_t spread_config(bool dbl, const Geom& g, int threads, LaunchCfg* cfg);
cudaError_t interp_config(bool dbl, const Geom& g, int threads, LaunchCfg* cfg);

cudaError_t launch_spread(bool dbl, const Geom& g, double beta, const Sorted& s, const void* c,
                          void* grid, int* work, const LaunchCfg& cfg, cudaStream_t st,
                          const BatchTable& bt = BatchTable{nullptr, nullptr, nullptr, nullptr, nullptr, 0});
cudaError_t launch_interp(bool dbl, const Geom& g, double beta, const Sorted& s, const void* grid,
                          void* c, int* work, const LaunchCfg& cfg, cudaStream_t st,
                          const BatchTable& bt = BatchTable{nullptr, nullptr, nullptr, nullptr, nullptr, 0});

// per-precision, per-dimension entry points (one translation unit each)
#define NUFFT_DECL_SI(P, D)                                                                      \
  cudaError_t spread_##P##_d##D(const Geom&, double, const Sorted&, const void*, void*, int*,   \
                                const LaunchCfg&, cudaStream_t, bool configure_only,            \
                                const BatchTable&);                                             \
  cudaError_t interp_##P##_d##D(const Geom&, double, const Sorted&, const void*, void*, int*,   \
                                const LaunchCfg&, cudaStream_t, bool configure_only,            \
                                const BatchTable&);
NUFFT_DECL_SI(f32, 1)
NUFFT_DECL_SI(f32, 2)
NUFFT_DECL_SI(f32, 3)
NUFFT_DECL_SI(f64, 1)
NUFFT_DECL_SI(f64, 2)
NUFFT_DECL_SI(f64, 3)
#undef NUFFT_DECL_SI

// --- interpolation with the gradient in the point (interp_grad.cuh) ---------
struct GradOut {
  void* dc[3];      // derivative of c_j in x_1, x_2, x_3 (M complex values each)
  double scale[3];  // (2 / w) n_d / (2 pi)
};
#define NUFFT_DECL_GRAD(P, D)                                                                          \
  cudaError_t interp_grad_##P##_d##D(const Geom&, double, const Sorted&, const void*, void*, const GradOut&, \
                                     int*, const LaunchCfg&, cudaStream_t, bool);
NUFFT_DECL_GRAD(f32, 1)
NUFFT_DECL_GRAD(f32, 2)
NUFFT_DECL_GRAD(f32, 3)
NUFFT_DECL_GRAD(f64, 1)
NUFFT_DECL_GRAD(f64, 2)
NUFFT_DECL_GRAD(f64, 3)
#undef NUFFT_DECL_GRAD

// --- deconvolve / pre-correct (deconv.cu) -------------------------------------
struct ModeGeom {
  int d;
  int N[3];   // modes per dimension (1 above d)
  int n[3];   // fine grid per dimension
  int modeord;
};
cudaError_t launch_deconv(bool dbl, const ModeGeom& m, const void* grid, void* f, const void* p1,
                          const void* p2, const void* p3, cudaStream_t st);
cudaError_t launch_precorrect(bool dbl, const ModeGeom& m, const void* f, void* grid, const void* p1,
                              const void* p2, const void* p3, cudaStream_t st);
// all transforms of a batch in one launch: nrows rows in total, maxlen the
// longest row; pk holds every transform's correction factors
cudaError_t launch_deconv_batch(bool dbl, int d, int modeord, long long nrows, int maxlen, const BatchTable& bt,
                                const void* grid, void* f, const void* pk, cudaStream_t st);
cudaError_t launch_precorrect_batch(bool dbl, int d, int modeord, long long nrows, int maxlen, const BatchTable& bt,
                                    const void* f, void* grid, const void* pk, cudaStream_t st);

// --- plan internals used by the serving layer (plan.cu) ------------------------
// Execute with the plan's grid, points and cuFFT plan but another type / sign
// (type 1 on a type-2 plan is its adjoint when isign is flipped).
int plan_execute_as(nufft_plan p, int type, int isign, void* c, void* f);
int plan_execute_grad(nufft_plan p, void* c, void* dc, const void* f);
int plan_set_stream(nufft_plan p, cudaStream_t s);
int plan_reserve(nufft_plan p, int64_t mcap);  // point capacity without setting points
size_t plan_device_bytes(nufft_plan p);
int plan_estimate_bytes(int dim, const int64_t* nmodes, double eps, int prec, int64_t mcap, size_t* bytes,
                        double sigma = 2.0);
int plan_modes(nufft_plan p, int64_t* N, int* dim);
void plan_choose_bins(Geom& g, bool dbl, const nufft_opts& o);  // bin extents for a grid (plan.cu's rule)
void gl_positive_nodes(int p, double* q, double* wq);            // Gauss-Legendre rule of Eq. (quad)
double sigma_from_opts(const nufft_opts& o);
// w x (w + 4) monomial coefficients of Sec. 5.3's piecewise polynomial (see nufft_horner_coeffs);
// computed once per (w, beta) and kept for the life of the process
const double* horner_table(int w, double beta, int kernel);
// phi(z) on the host for kernel 0 (ES) or 1 (cosh variant); 0 outside [-1, 1]
double kernel_value(double z, double beta, int kernel);

}  // namespace nufft
