// Host side of libnufft_gb300: the C ABI of include/nufft_gb300.h.
//
// makeplan  parameters (Eq. (params), Sec. 3.1.1), correction factors
//           (Eq. (pk1)/(pk) via the Gauss-Legendre rule of Eq. (quad) with
//           phase winding), fine grid, cuFFT plan
// setpts    binning pipeline (binsort.cu)
// execute   type 1: zero grid, spread, FFT, deconvolve
//           type 2: pre-correct/pad, FFT, interpolate
#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

// The binned points setpts produces: one record per point in bin order, the subproblem list and
// its two counts.  Plans share one set after nufft_setpts_from; a plan that sets new points while
// its set is shared gets a set of its own first, so no plan ever overwrites points another reads.
struct PointSet {
  int device = 0;
  void* rec = nullptr;
  int* sub_bin = nullptr;
  int* sub_pt0 = nullptr;
  int* sub_cnt = nullptr;
  int* counts = nullptr;  // device: [0] tiled subproblems, [1] per-warp subproblems
  int64_t Mcap = 0, subcap = 0;
  ~PointSet() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(device);
    void* bufs[] = {rec, sub_bin, sub_pt0, sub_cnt, counts};
    for (void* b : bufs)
      if (b) cudaFree(b);
    cudaSetDevice(dev);
  }
};

struct nufft_plan_s {
  int type = 0, dim = 0, isign = 0, ntransf = 1, prec = 0;
  nufft_opts opts;
  int64_t N[3] = {1, 1, 1};
  int64_t Ntot = 1;
  int w = 0;
  double beta = 0;
  Geom g;
  int64_t ngrid = 1;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool dbl = false;
  size_t csize = 8;  // bytes per complex
  void* grid = nullptr;
  void* pk[3] = {nullptr, nullptr, nullptr};
  int* bin_count = nullptr;
  int* bin_start = nullptr;
  int* sub_first = nullptr;
  int* cursor = nullptr;  // scatter cursors, nrep * nbins (replica-major)
  int* rep_count = nullptr;  // replicated bin counters, nrep * nbins (nrep > 1)
  int nrep = 1;
  int* small = nullptr;  // [0] error word, [2] work counter of the spread / interp kernels
  int64_t M = -1;
  std::shared_ptr<PointSet> ps;  // binned points (possibly shared with other plans)
  cufftHandle fft = 0;
  bool fft_ok = false;
  alignas(64) unsigned char tmap[128];  // CUtensorMap over grid for the interpolation's tile loads
  LaunchCfg spread_cfg{0, 0, 0}, interp_cfg{0, 0, 0}, grad_cfg{0, 0, 0};
  cudaEvent_t ev[8];
  bool ev_ok = false;
  int last_steps = 0;  // which timing slots the last call filled: 1 setpts, 2 execute
};

namespace {

const double kPi = 3.141592653589793238462643383279502884;

#define CUDA_TRY(x)                          \
  do {                                       \
    if ((x) != cudaSuccess) return NUFFT_ERR_CUDA; \
  } while (0)

int64_t next235_impl(int64_t m) {
  if (m < 1) return -1;
  for (int64_t n = m; n < ((int64_t)1 << 62); ++n) {
    int64_t r = n;
    while (r % 2 == 0) r /= 2;
    while (r % 3 == 0) r /= 3;
    while (r % 5 == 0) r /= 5;
    if (r == 1) return n;
  }
  return -1;
}

// Kernel width, clamped to [2, 16] (*capped set when the clamp from above applied).
//   sigma = 2 (Eq. (params)): w = ceil(log10(1/eps)) + 1 (guarded against
//     log10 rounding at exact powers of ten).
//   sigma = 5/4: the slope of Eq. (ESerr) in log10(1/eps),
//     ln(10) / (pi gamma sqrt(1 - 1/sigma - (gamma^-2 - 1) / (4 sigma^2))) = 1.714 at
//     gamma = 0.976, plus 0.43: the smallest offset for which the transform's
//     error stays below eps for eps = 1e-3 .. 1e-9 (measured).
int width_for(double eps, double sigma, bool* capped) {
  double lw;
  if (sigma == 2.0) lw = std::ceil(std::log10(1.0 / eps) - 1e-9) + 1.0;
  else lw = std::ceil(1.714 * std::log10(1.0 / eps) + 0.43 - 1e-9);
  if (!(lw >= 2.0)) lw = 2.0;
  if (capped) *capped = lw > 16.0;
  if (lw > 16.0) lw = 16.0;
  return (int)lw;
}

// beta = gamma pi w (1 - 1/(2 sigma)) (Eq. (gam)); gamma = 0.976 gives the
// paper's beta = 2.30 w at sigma = 2 (Eq. (params)).
double beta_for(int w, double sigma) {
  if (sigma == 2.0) return 2.30 * w;
  return 0.976 * 3.14159265358979323846 * w * (1.0 - 1.0 / (2.0 * sigma));
}

int choose_params_impl(int dim, const int64_t* N, double eps, int prec, int* w, double* beta, int64_t* n,
                       double sigma = 2.0) {
  if (dim < 1 || dim > 3 || !N || !(eps > 0.0) || !std::isfinite(eps) ||
      (prec != NUFFT_C64 && prec != NUFFT_C128) || (sigma != 2.0 && sigma != 1.25))
    return NUFFT_ERR_BAD_ARG;
  for (int i = 0; i < dim; ++i)
    if (N[i] < 1) return NUFFT_ERR_BAD_ARG;
  bool capped = false;
  int ww = width_for(eps, sigma, &capped);
  if (w) *w = ww;
  if (beta) *beta = beta_for(ww, sigma);
  for (int i = 0; i < dim; ++i) {
    // n_i = next 2^a 3^b 5^c >= max(sigma N_i, 2 w)
    int64_t sn = sigma == 2.0 ? 2 * N[i] : (5 * N[i] + 3) / 4;
    int64_t m = std::max<int64_t>(sn, 2 * (int64_t)ww);
    int64_t v = next235_impl(m);
    if (v < 0) return NUFFT_ERR_BAD_ARG;
    if (n) n[i] = v;
  }
  double floor_eps = (prec == NUFFT_C64) ? 1e-6 : 1e-15;
  // The correction p_k amplifies the grid's rounding by up to rmax per
  // dimension, rmax ~ exp((1 - sqrt(1 - (2 sigma - 1)^-2)) beta) (Eq. (rmax)):
  // e^{0.057 beta} at sigma = 2 but e^{0.25 beta} at 5/4, so at 5/4 warn when
  // unit roundoff times rmax^dim exceeds eps (e.g. complex64 in 3D below eps = 1e-3).
  bool amplified = false;
  if (sigma != 2.0) {
    const double u = (prec == NUFFT_C64) ? 5.96e-8 : 1.11e-16;
    const double g = 1.0 / (2.0 * sigma - 1.0);
    amplified = u * std::exp(dim * (1.0 - std::sqrt(1.0 - g * g)) * beta_for(ww, sigma)) > eps;
  }
  return (eps < floor_eps || capped || amplified) ? NUFFT_WARN_EPS_TOO_SMALL : NUFFT_OK;
}

// upsampling factor from the options: 0 means 2
double sigma_of(const nufft_opts& o) { return o.upsampfac == 0.0 ? 2.0 : o.upsampfac; }

// Positive nodes / weights of the 2p-point Gauss-Legendre rule by Newton's
// method on the three-term Legendre recurrence.
void gauss_legendre_positive(int p, std::vector<double>& q, std::vector<double>& wq) {
  const int m = 2 * p;
  q.assign(p, 0.0);
  wq.assign(p, 0.0);
  for (int i = 0; i < p; ++i) {
    // i-th largest root; classical initial guess
    double x = std::cos(kPi * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= m; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute the derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= m; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = m * (x * p1 - p0) / (x * x - 1.0);
    q[i] = x;
    wq[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

}  // namespace

namespace nufft {
double kernel_value(double z, double beta, int kernel) {
  if (std::fabs(z) > 1.0) return 0.0;
  const double s = std::sqrt(std::max(1.0 - z * z, 0.0));
  if (kernel == 1) return 2.0 * std::exp(-beta) * std::cosh(beta * s);
  return std::exp(beta * (s - 1.0));
}
}  // namespace nufft

namespace {

// Eq. (pk1) with Eq. (quad): p_k = 2 / (w phi^(alpha k)),
// phi^(xi) = 2 sum_j w_j phi(q_j) cos(xi q_j) over the p positive nodes,
// p = ceil(1.5 w + 2).  cos(alpha k q_j) by phase winding over k (a complex
// multiply per step), re-anchored with a direct cos/sin every 256 steps.
int correction_impl(int64_t N, int64_t n, int w, double beta, double* out, int kernel = 0) {
  if (N < 1 || n < 1 || w < 2 || w > 16 || !out) return NUFFT_ERR_BAD_ARG;
  const int p = (int)std::ceil(1.5 * w + 2.0);
  std::vector<double> q, wq;
  gauss_legendre_positive(p, q, wq);
  std::vector<double> a(p);
  for (int j = 0; j < p; ++j) a[j] = 2.0 * wq[j] * nufft::kernel_value(q[j], beta, kernel);
  const double alpha = kPi * w / (double)n;
  const int64_t kmax = N - 1 - N / 2;   // largest k; |k| <= N/2
  const int64_t kabs = std::max<int64_t>(kmax, N / 2);
  std::vector<double> ft(kabs + 1, 0.0);
  std::vector<double> cr(p), ci(p), zr(p), zi(p);
  for (int j = 0; j < p; ++j) {
    cr[j] = 1.0;
    ci[j] = 0.0;
    zr[j] = std::cos(alpha * q[j]);
    zi[j] = std::sin(alpha * q[j]);
  }
  for (int64_t k = 0; k <= kabs; ++k) {
    if (k % 256 == 0 && k > 0)
      for (int j = 0; j < p; ++j) {
        cr[j] = std::cos(alpha * (double)k * q[j]);
        ci[j] = std::sin(alpha * (double)k * q[j]);
      }
    double s = 0.0;
    for (int j = 0; j < p; ++j) s += a[j] * cr[j];
    ft[k] = s;
    for (int j = 0; j < p; ++j) {
      double r = cr[j] * zr[j] - ci[j] * zi[j];
      double i = cr[j] * zi[j] + ci[j] * zr[j];
      cr[j] = r;
      ci[j] = i;
    }
  }
  for (int64_t m = 0; m < N; ++m) {
    int64_t k = m - N / 2;
    out[m] = 2.0 / (w * ft[k < 0 ? -k : k]);
  }
  return NUFFT_OK;
}

// Bin shapes in order of preference; the first whose spread kernel fits the
// shared-memory budget wins.
void choose_bins(Geom& g, bool dbl, const nufft_opts& o) {
  static const int c3[][3] = {{16, 8, 8}, {8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {4, 4, 4}};
  static const int c2[][3] = {{32, 32, 1}, {32, 16, 1}, {16, 16, 1}, {16, 8, 1}, {8, 8, 1}};
  static const int c1[][3] = {{1024, 1, 1}, {512, 1, 1}, {256, 1, 1}, {128, 1, 1}, {64, 1, 1}};
  const int(*c)[3] = g.d == 3 ? c3 : (g.d == 2 ? c2 : c1);
  // two blocks per SM; the complex128 spread with 32-bit words runs one 512-thread block per SM
  const size_t budget = (dbl && g.w <= kDwMaxW) ? 216 * 1024 : 110 * 1024;
  for (int k = 0; k < 5; ++k) {
    for (int i = 0; i < 3; ++i) {
      int b = (o.bin_size[i] > 0 && i < g.d) ? o.bin_size[i] : c[k][i];
      if (i >= g.d) b = 1;
      g.B[i] = std::max(1, std::min(b, g.n[i]));
    }
    finish_geom(g);
    size_t need = spread_smem_bytes(dbl, g, 256);
    if (need <= budget || (o.bin_size[0] > 0)) break;
  }
}

// subproblems of at most this many points take the per-warp path (0: none)
int sparse_max_of(const nufft_opts& o) {
  if (o.sparse_max < 0) return 0;
  return o.sparse_max == 0 ? 32 : std::min(o.sparse_max, 32);
}

// a new, empty point set on the plan's device
int new_point_set(nufft_plan p) {
  auto ps = std::make_shared<PointSet>();
  ps->device = p->device;
  if (cudaMalloc((void**)&ps->counts, 2 * sizeof(int)) != cudaSuccess) {
    ps->counts = nullptr;
    return NUFFT_ERR_ALLOC;
  }
  if (cudaMemsetAsync(ps->counts, 0, 2 * sizeof(int), p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  p->ps = ps;
  return NUFFT_OK;
}

// room for mcap points in the plan's own (unshared) point set
int reserve_points(nufft_plan p, int64_t mcap) {
  if (p->ps.use_count() > 1) {
    int st = new_point_set(p);
    if (st != NUFFT_OK) return st;
  }
  PointSet& ps = *p->ps;
  const Geom& g = p->g;
  if (mcap > ps.Mcap) {
    cudaFree(ps.rec);
    ps.rec = nullptr;
    ps.Mcap = 0;
    size_t rsz = p->dbl ? sizeof(RecD) : sizeof(RecF);
    if (cudaMalloc(&ps.rec, rsz * (size_t)std::max<int64_t>(mcap, 1)) != cudaSuccess) {
      ps.rec = nullptr;
      return NUFFT_ERR_ALLOC;
    }
    ps.Mcap = mcap;
  }
  int64_t need = std::min<int64_t>(g.nbins, mcap) + mcap / g.maxsub + 1;
  if (need > ps.subcap) {
    cudaFree(ps.sub_bin);
    cudaFree(ps.sub_pt0);
    cudaFree(ps.sub_cnt);
    ps.sub_bin = ps.sub_pt0 = ps.sub_cnt = nullptr;
    ps.subcap = 0;
    if (cudaMalloc((void**)&ps.sub_bin, sizeof(int) * (size_t)need) != cudaSuccess ||
        cudaMalloc((void**)&ps.sub_pt0, sizeof(int) * (size_t)need) != cudaSuccess ||
        cudaMalloc((void**)&ps.sub_cnt, sizeof(int) * (size_t)need) != cudaSuccess)
      return NUFFT_ERR_ALLOC;
    ps.subcap = need;
  }
  return NUFFT_OK;
}

Sorted sorted_of(nufft_plan p) {
  const PointSet& ps = *p->ps;
  return Sorted{ps.rec, ps.sub_bin, ps.sub_pt0, ps.sub_cnt, ps.counts, ps.counts + 1, p->small};
}

int fail(nufft_plan p, int code) {
  nufft_destroy(p);
  return code;
}

template <typename P>
cudaError_t dev_alloc(P** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  return cudaMalloc((void**)ptr, bytes);
}

}  // namespace

namespace nufft {

size_t spread_smem_bytes(bool dbl, const Geom& g, int) {
  if (!dbl && quad_layout(g)) return spread_q_bytes(g);
  if (dbl && g.w <= kDwMaxW) return spread_dw_bytes(g);
  size_t ci = dbl ? 8 : 4, cc = dbl ? 16 : 8;
  // the spread's point order is gapless: res, rank and order of maxsub entries each
  return 2 * (size_t)g.ntile * ci + (size_t)g.maxsub * cc + (size_t)g.maxsub * 3 * 2;
}
// the tile with its halo and the aligned point order of the per-point interpolation kernels
static size_t interp_plain_bytes(bool dbl, const Geom& g) {
  size_t cc = dbl ? 16 : 8;
  return (size_t)g.ntile * cc + (size_t)g.maxsub * 5 * 2;
}
size_t interp_smem_bytes(bool dbl, const Geom& g, int) {
  if (!dbl && quad_layout(g)) return interp_q_bytes(g);
  return interp_plain_bytes(dbl, g);
}

// Tensor map for TMA loads of one bank-grouped tile from a complex64 fine grid, seen as a 3D
// array of floats (2 n_1, n_2, n_3): box (2 qs0, qt1, T_3), no swizzle, zero fill outside the
// grid (the kernel uses the TMA only for tiles that need no periodic wrap).
bool encode_tile_map(const Geom& g, const void* grid, void* tmap) {
  if (!quad_layout(g) || g.d != 3 || (g.n[0] & 1) || !grid || ((uintptr_t)grid & 15)) return false;
  if (2 * g.qs0 > 256 || g.qt1 > 256 || g.T[2] > 256) return false;  // TMA box limits
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)f;
    looked = true;
  }
  if (!fn) return false;
  const cuuint64_t dims[3] = {2 * (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  const cuuint64_t strides[2] = {8 * (cuuint64_t)g.n[0], 8 * (cuuint64_t)g.n[0] * (cuuint64_t)g.n[1]};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * g.qs0), (cuuint32_t)g.qt1, (cuuint32_t)g.T[2]};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(tmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(grid),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static cudaError_t si_dispatch(bool spread, bool dbl, const Geom& g, double beta, const Sorted& s,
                               const void* a, void* b, int* work, const LaunchCfg& cfg,
                               cudaStream_t st, bool conf, const BatchTable& bt) {
  if (spread) {
    if (!dbl) {
      if (g.d == 1) return spread_f32_d1(g, beta, s, a, b, work, cfg, st, conf, bt);
      if (g.d == 2) return spread_f32_d2(g, beta, s, a, b, work, cfg, st, conf, bt);
      return spread_f32_d3(g, beta, s, a, b, work, cfg, st, conf, bt);
    }
    if (g.d == 1) return spread_f64_d1(g, beta, s, a, b, work, cfg, st, conf, bt);
    if (g.d == 2) return spread_f64_d2(g, beta, s, a, b, work, cfg, st, conf, bt);
    return spread_f64_d3(g, beta, s, a, b, work, cfg, st, conf, bt);
  }
  if (!dbl) {
    if (g.d == 1) return interp_f32_d1(g, beta, s, a, b, work, cfg, st, conf, bt);
    if (g.d == 2) return interp_f32_d2(g, beta, s, a, b, work, cfg, st, conf, bt);
    return interp_f32_d3(g, beta, s, a, b, work, cfg, st, conf, bt);
  }
  if (g.d == 1) return interp_f64_d1(g, beta, s, a, b, work, cfg, st, conf, bt);
  if (g.d == 2) return interp_f64_d2(g, beta, s, a, b, work, cfg, st, conf, bt);
  return interp_f64_d3(g, beta, s, a, b, work, cfg, st, conf, bt);
}

static cudaError_t configure(bool spread, bool dbl, const Geom& g, int threads, LaunchCfg* cfg) {
  cfg->threads = threads;
  cfg->smem = spread ? spread_smem_bytes(dbl, g, threads) : interp_smem_bytes(dbl, g, threads);
  cfg->blocks = 0;
  Sorted s{};
  BatchTable none{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  cudaError_t e = si_dispatch(spread, dbl, g, 0.0, s, nullptr, nullptr, nullptr, *cfg, nullptr, true, none);
  if (e != cudaSuccess) return e;
  int per_sm = cfg->blocks, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cfg->blocks = per_sm * sms;
  return cudaSuccess;
}

static cudaError_t grad_dispatch(bool dbl, const Geom& g, double beta, const Sorted& s, const void* grid, void* c,
                                 const GradOut& go, int* work, const LaunchCfg& cfg, cudaStream_t st, bool conf) {
  if (!dbl) {
    if (g.d == 1) return interp_grad_f32_d1(g, beta, s, grid, c, go, work, cfg, st, conf);
    if (g.d == 2) return interp_grad_f32_d2(g, beta, s, grid, c, go, work, cfg, st, conf);
    return interp_grad_f32_d3(g, beta, s, grid, c, go, work, cfg, st, conf);
  }
  if (g.d == 1) return interp_grad_f64_d1(g, beta, s, grid, c, go, work, cfg, st, conf);
  if (g.d == 2) return interp_grad_f64_d2(g, beta, s, grid, c, go, work, cfg, st, conf);
  return interp_grad_f64_d3(g, beta, s, grid, c, go, work, cfg, st, conf);
}

static cudaError_t grad_config(bool dbl, const Geom& g, int threads, LaunchCfg* cfg) {
  cfg->threads = threads;
  cfg->smem = interp_plain_bytes(dbl, g);  // the gradient kernels keep the per-point tile layout
  cfg->blocks = 0;
  Sorted s{};
  GradOut go{};
  cudaError_t e = grad_dispatch(dbl, g, 0.0, s, nullptr, nullptr, go, nullptr, *cfg, nullptr, true);
  if (e != cudaSuccess) return e;
  int per_sm = cfg->blocks, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cfg->blocks = per_sm * sms;
  return cudaSuccess;
}

cudaError_t spread_config(bool dbl, const Geom& g, int threads, LaunchCfg* cfg) {
  return configure(true, dbl, g, threads, cfg);
}
cudaError_t interp_config(bool dbl, const Geom& g, int threads, LaunchCfg* cfg) {
  return configure(false, dbl, g, threads, cfg);
}
cudaError_t launch_spread(bool dbl, const Geom& g, double beta, const Sorted& s, const void* c,
                          void* grid, int* work, const LaunchCfg& cfg, cudaStream_t st, const BatchTable& bt) {
  return si_dispatch(true, dbl, g, beta, s, c, grid, work, cfg, st, false, bt);
}
cudaError_t launch_interp(bool dbl, const Geom& g, double beta, const Sorted& s, const void* grid,
                          void* c, int* work, const LaunchCfg& cfg, cudaStream_t st, const BatchTable& bt) {
  return si_dispatch(false, dbl, g, beta, s, grid, c, work, cfg, st, false, bt);
}

}  // namespace nufft

extern "C" {

int nufft_default_opts(nufft_opts* o) {
  if (!o) return NUFFT_ERR_BAD_ARG;
  std::memset(o, 0, sizeof(*o));
  return NUFFT_OK;
}

int64_t nufft_next235(int64_t m) { return next235_impl(m); }

int nufft_choose_params(int dim, const int64_t* nmodes, double eps, int prec, int* w, double* beta,
                        int64_t* n) {
  return choose_params_impl(dim, nmodes, eps, prec, w, beta, n);
}

int nufft_choose_params_sigma(int dim, const int64_t* nmodes, double eps, int prec, double sigma, int* w,
                              double* beta, int64_t* n) {
  return choose_params_impl(dim, nmodes, eps, prec, w, beta, n, sigma);
}

int nufft_horner_coeffs(int w, double beta, double* out) {
  if (w < 2 || w > 16 || !(beta > 0.0) || !out) return NUFFT_ERR_BAD_ARG;
  const double* a = nufft::horner_table(w, beta, 0);
  std::memcpy(out, a, sizeof(double) * (size_t)w * (size_t)(w + 4));
  return NUFFT_OK;
}

int nufft_correction_factors(int64_t N, int64_t n, int w, double beta, double* out) {
  return correction_impl(N, n, w, beta, out);
}

const char* nufft_strerror(int code) {
  switch (code) {
    case NUFFT_OK: return "success";
    case NUFFT_WARN_EPS_TOO_SMALL: return "warning: eps below what this precision can deliver";
    case NUFFT_ERR_BAD_ARG: return "invalid argument";
    case NUFFT_ERR_OUT_OF_RANGE: return "a point lies outside [-3 pi, 3 pi] or is not finite";
    case NUFFT_ERR_ALLOC: return "device allocation failed";
    case NUFFT_ERR_CUDA: return "CUDA runtime error";
    case NUFFT_ERR_CUFFT: return "cuFFT error";
    case NUFFT_ERR_NOT_SET: return "execute called before setpts";
    case NUFFT_ERR_TOO_BIG: return "problem too large for the index types";
    case NUFFT_ERR_TIMEOUT: return "request not done within the server's time limit";
    case NUFFT_ERR_REJECTED: return "request needs more device memory than the server's budget";
    case NUFFT_ERR_SHUTDOWN: return "server destroyed before the request ran";
    default: return "unknown status";
  }
}

int nufft_makeplan(int type, int dim, const int64_t* nmodes, int isign, int ntransf, double eps,
                   int prec, void* stream, const nufft_opts* opts, nufft_plan* out) {
  if (!out) return NUFFT_ERR_BAD_ARG;
  *out = nullptr;
  if ((type != 1 && type != 2) || (isign != 1 && isign != -1) || ntransf < 1) return NUFFT_ERR_BAD_ARG;
  int w;
  double beta;
  int64_t n[3] = {1, 1, 1};
  int warn = choose_params_impl(dim, nmodes, eps, prec, &w, &beta, n, opts ? sigma_of(*opts) : 2.0);
  if (warn < 0) return warn;
  for (int i = 0; i < dim; ++i)
    if (nmodes[i] > (1 << 29) || n[i] > (1 << 30)) return NUFFT_ERR_TOO_BIG;

  nufft_plan p = new (std::nothrow) nufft_plan_s();
  if (!p) return NUFFT_ERR_ALLOC;
  p->type = type;
  p->dim = dim;
  p->isign = isign;
  p->ntransf = ntransf;
  p->prec = prec;
  p->dbl = (prec == NUFFT_C128);
  p->csize = p->dbl ? 16 : 8;
  if (opts) p->opts = *opts;
  else nufft_default_opts(&p->opts);
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(p, NUFFT_ERR_CUDA);
  p->w = w;
  p->beta = beta;
  p->Ntot = 1;
  p->ngrid = 1;
  for (int i = 0; i < 3; ++i) {
    p->N[i] = i < dim ? nmodes[i] : 1;
    p->Ntot *= p->N[i];
    p->ngrid *= n[i];
  }
  Geom& g = p->g;
  g.d = dim;
  g.w = w;
  g.half = w / 2;
  for (int i = 0; i < 3; ++i) g.n[i] = (int)n[i];
  g.maxsub = p->opts.max_subprob > 0 ? std::min(p->opts.max_subprob, 8192) : (p->dbl ? 512 : 1024);
  g.sparse_max = sparse_max_of(p->opts);
  g.horner = p->opts.kerevalmeth == 1 ? 1 : 0;
  g.kernel = p->opts.kernel == 1 ? 1 : 0;
  choose_bins(g, p->dbl, p->opts);
  int threads = p->opts.threads > 0 ? p->opts.threads : 256;
  if (threads % 32 != 0 || threads > 256 || p->opts.kerevalmeth < 0 || p->opts.kerevalmeth > 1 ||
      p->opts.kernel < 0 || p->opts.kernel > 1)
    return fail(p, NUFFT_ERR_BAD_ARG);

  // device buffers owned by the plan
  if (dev_alloc(&p->grid, p->ngrid * p->csize) != cudaSuccess) return fail(p, NUFFT_ERR_ALLOC);
  size_t rs = p->dbl ? 8 : 4;
  for (int i = 0; i < 3; ++i) {
    std::vector<double> pk((size_t)p->N[i], 1.0);
    if (i < dim && correction_impl(p->N[i], n[i], w, beta, pk.data(), p->opts.kernel) != NUFFT_OK)
      return fail(p, NUFFT_ERR_BAD_ARG);
    if (dev_alloc(&p->pk[i], (size_t)p->N[i] * rs) != cudaSuccess) return fail(p, NUFFT_ERR_ALLOC);
    if (p->dbl) {
      if (cudaMemcpy(p->pk[i], pk.data(), pk.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(p, NUFFT_ERR_CUDA);
    } else {
      std::vector<float> pf(pk.begin(), pk.end());
      if (cudaMemcpy(p->pk[i], pf.data(), pf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(p, NUFFT_ERR_CUDA);
    }
  }
  if (dev_alloc(&p->bin_count, sizeof(int) * (size_t)g.nbins) != cudaSuccess ||
      dev_alloc(&p->bin_start, sizeof(int) * (size_t)g.nbins) != cudaSuccess ||
      dev_alloc(&p->sub_first, sizeof(int) * (size_t)g.nbins) != cudaSuccess ||
      dev_alloc(&p->cursor, sizeof(int) * (size_t)g.nbins * (size_t)(p->nrep = replicas_for(g.nbins))) != cudaSuccess ||
      dev_alloc(&p->rep_count, sizeof(int) * (size_t)g.nbins * (size_t)p->nrep) != cudaSuccess ||
      dev_alloc(&p->small, sizeof(int) * 4) != cudaSuccess)
    return fail(p, NUFFT_ERR_ALLOC);
  if (cudaMemset(p->small, 0, sizeof(int) * 4) != cudaSuccess) return fail(p, NUFFT_ERR_CUDA);
  if (new_point_set(p) != NUFFT_OK) return fail(p, NUFFT_ERR_ALLOC);

  // both launch shapes: the serving layer runs a plan's adjoint (type 1 on a type-2 plan)
  if (spread_config(p->dbl, g, threads, &p->spread_cfg) != cudaSuccess ||
      interp_config(p->dbl, g, threads, &p->interp_cfg) != cudaSuccess)
    return fail(p, NUFFT_ERR_CUDA);
  if (!p->dbl && quad_layout(g) && encode_tile_map(g, p->grid, p->tmap)) {
    p->interp_cfg.tmap = p->tmap;  // tile loads (interpolation)
    p->spread_cfg.tmap = p->tmap;  // tile reductions (spreading); the same box over the same grid
  }

  // cuFFT: dimensions slowest first
  int nn[3];
  for (int i = 0; i < dim; ++i) nn[i] = (int)n[dim - 1 - i];
  if (cufftPlanMany(&p->fft, dim, nn, nullptr, 1, 0, nullptr, 1, 0, p->dbl ? CUFFT_Z2Z : CUFFT_C2C, 1) !=
      CUFFT_SUCCESS)
    return fail(p, NUFFT_ERR_CUFFT);
  p->fft_ok = true;
  if (cufftSetStream(p->fft, p->stream) != CUFFT_SUCCESS) return fail(p, NUFFT_ERR_CUFFT);
  if (p->opts.debug) {
    for (int i = 0; i < 8; ++i)
      if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return fail(p, NUFFT_ERR_CUDA);
    p->ev_ok = true;
  }
  *out = p;
  return warn;
}

int nufft_setpts(nufft_plan p, int64_t M, const void* x, const void* y, const void* z) {
  if (!p || M < 0) return NUFFT_ERR_BAD_ARG;
  if (M > 0 && (!x || (p->dim > 1 && !y) || (p->dim > 2 && !z))) return NUFFT_ERR_BAD_ARG;
  if (M >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_TOO_BIG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  const Geom& g = p->g;
  int rc = reserve_points(p, M);
  if (rc != NUFFT_OK) return rc;
  PointSet& ps = *p->ps;
  FoldConst fc = make_fold_const(g);
  cudaError_t e = launch_setpts(p->dbl, g, fc, M, x, y, z, p->opts.chkbnds, p->bin_count, p->bin_start,
                                p->sub_first, p->cursor, ps.rec, ps.sub_bin, ps.sub_pt0,
                                ps.sub_cnt, ps.counts, ps.counts + 1, p->small + 0, p->stream,
                                p->ev_ok ? p->ev : nullptr, BatchTable{nullptr, nullptr, nullptr, nullptr, nullptr, 0},
                                g.nbins, Replicas{p->nrep, p->rep_count, p->cursor});
  if (e != cudaSuccess) return NUFFT_ERR_CUDA;
  p->M = M;
  p->last_steps = 1;
  return NUFFT_OK;
}

int nufft_setpts_from(nufft_plan dst, nufft_plan src) {
  if (!dst || !src) return NUFFT_ERR_BAD_ARG;
  if (src->M < 0) return NUFFT_ERR_NOT_SET;
  const Geom& a = dst->g;
  const Geom& b = src->g;
  // the binning depends on the fine grid, the bin extents, the subproblem limits and the precision
  bool same = dst->device == src->device && dst->dbl == src->dbl && a.d == b.d && a.maxsub == b.maxsub &&
              a.sparse_max == b.sparse_max;
  for (int i = 0; i < 3; ++i) same = same && a.n[i] == b.n[i] && a.B[i] == b.B[i];
  if (!same) return NUFFT_ERR_BAD_ARG;
  if (dst == src) return NUFFT_OK;
  dst->ps = src->ps;
  dst->M = src->M;
  dst->last_steps = 0;
  return NUFFT_OK;
}

int nufft_execute(nufft_plan p, void* c, void* f) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  return nufft::plan_execute_as(p, p->type, p->isign, c, f);
}

}  // extern "C"

namespace nufft {

int plan_execute_as(nufft_plan p, int type, int isign, void* c, void* f) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (p->M < 0) return NUFFT_ERR_NOT_SET;
  if (!f || (p->M > 0 && !c)) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  const Geom& g = p->g;
  Sorted s = sorted_of(p);
  ModeGeom mg;
  mg.d = p->dim;
  mg.modeord = p->opts.modeord ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    mg.N[i] = (int)p->N[i];
    mg.n[i] = g.n[i];
  }
  const int dir = isign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD;
  cudaEvent_t* ev = p->ev_ok ? p->ev + 4 : nullptr;
  for (int t = 0; t < p->ntransf; ++t) {
    char* ct = (char*)c + (size_t)t * (size_t)p->M * p->csize;
    char* ft = (char*)f + (size_t)t * (size_t)p->Ntot * p->csize;
    if (type == 1) {
      CUDA_TRY(cudaMemsetAsync(p->grid, 0, (size_t)p->ngrid * p->csize, p->stream));
      if (ev && t == 0) cudaEventRecord(ev[0], p->stream);
      if (p->M > 0) {
        CUDA_TRY(cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream));
        CUDA_TRY(launch_spread(p->dbl, g, p->beta, s, ct, p->grid, p->small + 2, p->spread_cfg, p->stream));
      }
    } else {
      if (ev && t == 0) cudaEventRecord(ev[0], p->stream);
      CUDA_TRY(launch_precorrect(p->dbl, mg, ft, p->grid, p->pk[0], p->pk[1], p->pk[2], p->stream));
    }
    if (ev && t == 0) cudaEventRecord(ev[1], p->stream);
    cufftResult r = p->dbl ? cufftExecZ2Z(p->fft, (cufftDoubleComplex*)p->grid, (cufftDoubleComplex*)p->grid, dir)
                           : cufftExecC2C(p->fft, (cufftComplex*)p->grid, (cufftComplex*)p->grid, dir);
    if (r != CUFFT_SUCCESS) return NUFFT_ERR_CUFFT;
    if (type == 2 && p->M > 0) CUDA_TRY(cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream));
    if (ev && t == 0) cudaEventRecord(ev[2], p->stream);
    if (type == 1) {
      CUDA_TRY(launch_deconv(p->dbl, mg, p->grid, ft, p->pk[0], p->pk[1], p->pk[2], p->stream));
    } else if (p->M > 0) {
      CUDA_TRY(launch_interp(p->dbl, g, p->beta, s, p->grid, ct, p->small + 2, p->interp_cfg, p->stream));
    }
    if (ev && t == 0) cudaEventRecord(ev[3], p->stream);
  }
  p->last_steps = 2;
  return NUFFT_OK;
}

int plan_execute_grad(nufft_plan p, void* c, void* dc, const void* f) {
  if (!p || p->type != 2) return NUFFT_ERR_BAD_ARG;
  if (p->M < 0) return NUFFT_ERR_NOT_SET;
  if (!f || (p->M > 0 && (!c || !dc))) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  const Geom& g = p->g;
  if (p->grad_cfg.blocks == 0) {
    int threads = p->opts.threads > 0 ? p->opts.threads : 256;
    if (grad_config(p->dbl, g, threads, &p->grad_cfg) != cudaSuccess) return NUFFT_ERR_CUDA;
  }
  Sorted s = sorted_of(p);
  ModeGeom mg;
  mg.d = p->dim;
  mg.modeord = p->opts.modeord ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    mg.N[i] = (int)p->N[i];
    mg.n[i] = g.n[i];
  }
  const int dir = p->isign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD;
  const double two_pi = 6.283185307179586476925286766559;
  cudaEvent_t* ev = p->ev_ok ? p->ev + 4 : nullptr;
  for (int t = 0; t < p->ntransf; ++t) {
    char* ct = (char*)c + (size_t)t * (size_t)p->M * p->csize;
    char* dct = (char*)dc + (size_t)t * (size_t)p->dim * (size_t)p->M * p->csize;
    const char* ft = (const char*)f + (size_t)t * (size_t)p->Ntot * p->csize;
    if (ev && t == 0) cudaEventRecord(ev[0], p->stream);
    CUDA_TRY(launch_precorrect(p->dbl, mg, ft, p->grid, p->pk[0], p->pk[1], p->pk[2], p->stream));
    if (ev && t == 0) cudaEventRecord(ev[1], p->stream);
    cufftResult r = p->dbl ? cufftExecZ2Z(p->fft, (cufftDoubleComplex*)p->grid, (cufftDoubleComplex*)p->grid, dir)
                           : cufftExecC2C(p->fft, (cufftComplex*)p->grid, (cufftComplex*)p->grid, dir);
    if (r != CUFFT_SUCCESS) return NUFFT_ERR_CUFFT;
    if (ev && t == 0) cudaEventRecord(ev[2], p->stream);
    if (p->M > 0) {
      CUDA_TRY(cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream));
      GradOut go{};
      for (int d = 0; d < 3; ++d) {
        go.dc[d] = d < p->dim ? dct + (size_t)d * (size_t)p->M * p->csize : nullptr;
        go.scale[d] = d < p->dim ? (2.0 / p->w) * ((double)g.n[d] / two_pi) : 0.0;
      }
      CUDA_TRY(grad_dispatch(p->dbl, g, p->beta, s, p->grid, ct, go, p->small + 2, p->grad_cfg, p->stream, false));
    }
    if (ev && t == 0) cudaEventRecord(ev[3], p->stream);
  }
  p->last_steps = 2;
  return NUFFT_OK;
}

int plan_set_stream(nufft_plan p, cudaStream_t s) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  p->stream = s;
  if (p->fft_ok && cufftSetStream(p->fft, s) != CUFFT_SUCCESS) return NUFFT_ERR_CUFFT;
  return NUFFT_OK;
}

int plan_reserve(nufft_plan p, int64_t mcap) {
  if (!p || mcap < 0) return NUFFT_ERR_BAD_ARG;
  if (mcap >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_TOO_BIG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  return reserve_points(p, mcap);
}

// Device bytes a plan holds: its buffers plus cuFFT's work area.
size_t plan_device_bytes(nufft_plan p) {
  if (!p) return 0;
  size_t rs = p->dbl ? 8 : 4, cs = p->csize;
  size_t b = (size_t)p->ngrid * cs + (3 + 2 * (size_t)p->nrep) * sizeof(int) * (size_t)p->g.nbins + 4 * sizeof(int);
  for (int i = 0; i < 3; ++i) b += (size_t)p->N[i] * rs;
  if (p->ps) b += (size_t)p->ps->Mcap * (p->dbl ? sizeof(RecD) : sizeof(RecF)) + 3 * sizeof(int) * (size_t)p->ps->subcap;
  size_t ws = 0;
  if (p->fft_ok && cufftGetSize(p->fft, &ws) == CUFFT_SUCCESS) b += ws;
  return b;
}

// Upper estimate of plan_device_bytes before the plan exists (default options,
// point capacity mcap); cuFFT's work area is bounded by one more fine grid.
int plan_estimate_bytes(int dim, const int64_t* nmodes, double eps, int prec, int64_t mcap, size_t* bytes,
                        double sigma) {
  if (!bytes || !nmodes || dim < 1 || dim > 3 || mcap < 0 || (prec != NUFFT_C64 && prec != NUFFT_C128))
    return NUFFT_ERR_BAD_ARG;
  int w;
  double beta;
  int64_t n[3] = {1, 1, 1};
  int st = choose_params_impl(dim, nmodes, eps, prec, &w, &beta, n, sigma);
  if (st < 0) return st;
  const bool dbl = prec == NUFFT_C128;
  Geom g;
  g.d = dim;
  g.w = w;
  g.half = w / 2;
  for (int i = 0; i < 3; ++i) g.n[i] = (int)n[i];
  g.maxsub = dbl ? 512 : 1024;
  g.sparse_max = 32;
  g.horner = 0;
  g.kernel = 0;
  nufft_opts o;
  nufft_default_opts(&o);
  choose_bins(g, dbl, o);
  size_t cs = dbl ? 16 : 8, rs = dbl ? 8 : 4;
  size_t ngrid = (size_t)n[0] * (size_t)n[1] * (size_t)n[2];
  size_t b = 2 * ngrid * cs + (3 + 2 * (size_t)replicas_for(g.nbins)) * sizeof(int) * (size_t)g.nbins + 4 * sizeof(int);
  for (int i = 0; i < dim; ++i) b += (size_t)nmodes[i] * rs;
  int64_t subcap = std::min<int64_t>(g.nbins, mcap) + mcap / g.maxsub + 1;
  b += (size_t)mcap * (dbl ? sizeof(RecD) : sizeof(RecF)) + 3 * sizeof(int) * (size_t)subcap;
  *bytes = b;
  return NUFFT_OK;
}

void plan_choose_bins(Geom& g, bool dbl, const nufft_opts& o) { choose_bins(g, dbl, o); }

// Sec. 5.3's piecewise polynomial: on interval t the kernel psi(tau) = phi(2 tau / w),
// tau = t - w/2 + (s + 1)/2, as a polynomial of degree P - 1 = w + 3 in s.  Interpolation at
// the P Chebyshev points of the first kind gives the Chebyshev coefficients
//   c_j = (2 - [j = 0]) / P * sum_k psi(s_k) T_j(s_k),  s_k = cos(pi (k + 1/2) / P),
// and the recurrence T_{j+1} = 2 s T_j - T_{j-1} turns them into monomial coefficients.
// The kernel is analytic on every interval (its square-root branch points sit at the ends of
// the support, where phi = e^-beta), so the monomial form stays well conditioned: the sum of
// |coefficients| of an interval is about 1.
static void horner_fit(int w, double beta, int kernel, double* out) {
  const int P = w + 4;
  const double pi = 3.14159265358979323846;
  std::vector<double> f((size_t)P), c((size_t)P), tm((size_t)P), tj((size_t)P), tn((size_t)P);
  for (int t = 0; t < w; ++t) {
    for (int k = 0; k < P; ++k) {
      const double sk = std::cos(pi * (k + 0.5) / P);
      const double z = (t - 0.5 * w + 0.5 * (sk + 1.0)) * 2.0 / w;
      f[(size_t)k] = kernel_value(z, beta, kernel);
    }
    for (int j = 0; j < P; ++j) {
      double acc = 0.0;
      for (int k = 0; k < P; ++k) acc += f[(size_t)k] * std::cos(pi * j * (k + 0.5) / P);
      c[(size_t)j] = acc * (j == 0 ? 1.0 : 2.0) / P;
    }
    double* a = out + (size_t)t * P;
    for (int m = 0; m < P; ++m) a[m] = 0.0;
    std::fill(tm.begin(), tm.end(), 0.0);  // T_{j-1}
    std::fill(tj.begin(), tj.end(), 0.0);  // T_j
    tj[0] = 1.0;
    for (int j = 0; j < P; ++j) {
      for (int m = 0; m < P; ++m) a[m] += c[(size_t)j] * tj[(size_t)m];
      if (j + 1 == P) break;
      for (int m = 0; m < P; ++m) {
        const double up = m > 0 ? tj[(size_t)m - 1] : 0.0;
        tn[(size_t)m] = (j == 0 ? 1.0 : 2.0) * up - (j == 0 ? 0.0 : tm[(size_t)m]);
      }
      tm = tj;
      tj = tn;
    }
  }
}

const double* horner_table(int w, double beta, int kernel) {
  static std::mutex mu;
  static std::map<std::pair<int, double>, std::vector<double>> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(w + 100 * kernel, beta);
  auto it = cache.find(key);
  if (it == cache.end()) {
    std::vector<double> a((size_t)w * (size_t)(w + 4));
    horner_fit(w, beta, kernel, a.data());
    it = cache.emplace(key, std::move(a)).first;
  }
  return it->second.data();
}

void gl_positive_nodes(int p, double* q, double* wq) {
  std::vector<double> a, b;
  gauss_legendre_positive(p, a, b);
  for (int i = 0; i < p; ++i) {
    q[i] = a[(size_t)i];
    wq[i] = b[(size_t)i];
  }
}

double sigma_from_opts(const nufft_opts& o) { return sigma_of(o); }

int plan_modes(nufft_plan p, int64_t* N, int* dim) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  for (int i = 0; i < 3; ++i) N[i] = p->N[i];
  *dim = p->dim;
  return NUFFT_OK;
}

}  // namespace nufft

extern "C" {

int nufft_execute_grad(nufft_plan p, void* c, void* dc, const void* f) {
  return nufft::plan_execute_grad(p, c, dc, f);
}

int nufft_destroy(nufft_plan p) {
  if (!p) return NUFFT_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  if (p->fft_ok) cufftDestroy(p->fft);
  if (p->ev_ok)
    for (int i = 0; i < 8; ++i) cudaEventDestroy(p->ev[i]);
  void* bufs[] = {p->grid, p->pk[0], p->pk[1], p->pk[2], p->bin_count, p->bin_start, p->sub_first,
                  p->cursor, p->rep_count, p->small};
  for (void* b : bufs)
    if (b) cudaFree(b);
  p->ps.reset();  // freed here unless another plan still shares it
  cudaSetDevice(dev);
  delete p;
  return NUFFT_OK;
}

int nufft_get_status(nufft_plan p) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->small, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (err != 0 && cudaMemset(p->small, 0, sizeof(int)) != cudaSuccess) return NUFFT_ERR_CUDA;
  return err;
}

int nufft_get_timings(nufft_plan p, double* ms, int n) {
  if (!p || !ms || n < 0) return NUFFT_ERR_BAD_ARG;
  if (!p->ev_ok) return 0;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  int k = 0;
  bool missing = false;
  for (int i = 0; i < 6 && k < n; ++i, ++k) {
    float v = 0.f;
    int a = i < 3 ? i : i + 1;  // slots 0-3 setpts, 4-7 execute
    if (cudaEventElapsedTime(&v, p->ev[a], p->ev[a + 1]) != cudaSuccess) {
      v = -1.f;  // a step not run since the plan was made
      missing = true;
    }
    ms[k] = v;
  }
  // an event never recorded fails cudaEventElapsedTime with a non-sticky error that would
  // otherwise be reported by the next launch check of this thread
  if (missing) cudaGetLastError();
  return k;
}

int nufft_plan_info(nufft_plan p, int* w, double* beta, int64_t* n, int* bins, int64_t* nsub) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (w) *w = p->w;
  if (beta) *beta = p->beta;
  for (int i = 0; i < p->dim; ++i) {
    if (n) n[i] = p->g.n[i];
    if (bins) bins[i] = p->g.B[i];
  }
  if (nsub) {
    *nsub = 0;
    if (p->M >= 0) {
      if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
      int v = 0;
      if (cudaMemcpy(&v, p->ps->counts, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NUFFT_ERR_CUDA;
      *nsub = v;
    }
  }
  return NUFFT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// Many independent transforms of one type, dimension, precision and eps with
// their own mode counts.  All transforms share one bin shape (so the spread /
// interp kernels run one tile size), their fine grids sit in one allocation
// grouped by size (one batched cuFFT plan per size), and every step is one
// launch over all transforms: the binning kernels find a point's transform
// from the point offsets, the spread / interp kernels a subproblem's from the
// bin offsets, the correction kernels a row's from the row offsets.  The
// execute sequence is captured once in a CUDA graph and replayed.

struct nufft_batch_s {
  int type = 0, dim = 0, isign = 0, prec = 0;
  bool dbl = false;
  size_t csize = 8;
  nufft_opts opts;
  int B = 0;
  int w = 0;
  double beta = 0;
  Geom g;  // shared: d, w, half, B, T, ntile, maxsub
  std::vector<BatchGeom> hg;
  BatchGeom* bg = nullptr;
  int* boff = nullptr;
  int* poff = nullptr;
  long long* growoff = nullptr;
  long long* mrowoff = nullptr;
  int total_bins = 0;
  long long total_grid = 0, total_modes = 0, total_grow = 0, total_mrow = 0;
  int max_grow = 1, max_mrow = 1;
  void* grid = nullptr;
  void* pk = nullptr;
  struct SizeClass {
    int n[3];
    int count;
    long long goff;
    cufftHandle plan;
    bool ok;
  };
  std::vector<SizeClass> classes;
  int* bin_count = nullptr;
  int* bin_start = nullptr;
  int* sub_first = nullptr;
  int* cursor = nullptr;  // nrep * total_bins
  int* rep_count = nullptr;
  int nrep = 1;
  int* small = nullptr;  // [0] error word, [1] tiled subproblems, [2] work counter, [3] sparse subproblems
  int64_t M = -1, Mcap = 0, subcap = 0;
  void* rec = nullptr;
  int* sub_bin = nullptr;
  int* sub_pt0 = nullptr;
  int* sub_cnt = nullptr;
  std::vector<int> hpoff;
  LaunchCfg cfg{0, 0, 0};
  cudaStream_t stream = nullptr;
  int device = 0;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};  // c, f, rec, sub arrays the graph was built for
};

namespace {

BatchTable table_of(nufft_batch p) {
  return BatchTable{p->bg, p->boff, p->poff, p->growoff, p->mrowoff, p->B};
}

int batch_fail(nufft_batch p, int code) {
  nufft_batch_destroy(p);
  return code;
}

// The execute sequence, enqueued on the plan's stream.
int batch_enqueue(nufft_batch p, void* c, void* f) {
  const BatchTable bt = table_of(p);
  Sorted s{p->rec, p->sub_bin, p->sub_pt0, p->sub_cnt, p->small + 1, p->small + 3, p->small};
  const int dir = p->isign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD;
  const int modeord = p->opts.modeord ? 1 : 0;
  auto ffts = [&]() -> int {
    for (auto& cl : p->classes) {
      char* gp = (char*)p->grid + (size_t)cl.goff * p->csize;
      cufftResult r = p->dbl ? cufftExecZ2Z(cl.plan, (cufftDoubleComplex*)gp, (cufftDoubleComplex*)gp, dir)
                             : cufftExecC2C(cl.plan, (cufftComplex*)gp, (cufftComplex*)gp, dir);
      if (r != CUFFT_SUCCESS) return NUFFT_ERR_CUFFT;
    }
    return NUFFT_OK;
  };
  if (p->type == 1) {
    CUDA_TRY(cudaMemsetAsync(p->grid, 0, (size_t)p->total_grid * p->csize, p->stream));
    if (p->M > 0) {
      CUDA_TRY(cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream));
      CUDA_TRY(launch_spread(p->dbl, p->g, p->beta, s, c, p->grid, p->small + 2, p->cfg, p->stream, bt));
    }
    int r = ffts();
    if (r != NUFFT_OK) return r;
    CUDA_TRY(launch_deconv_batch(p->dbl, p->dim, modeord, p->total_mrow, p->max_mrow, bt, p->grid, f, p->pk, p->stream));
  } else {
    CUDA_TRY(launch_precorrect_batch(p->dbl, p->dim, modeord, p->total_grow, p->max_grow, bt, f, p->grid, p->pk,
                                     p->stream));
    int r = ffts();
    if (r != NUFFT_OK) return r;
    if (p->M > 0) {
      CUDA_TRY(cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream));
      CUDA_TRY(launch_interp(p->dbl, p->g, p->beta, s, p->grid, c, p->small + 2, p->cfg, p->stream, bt));
    }
  }
  return NUFFT_OK;
}

}  // namespace

extern "C" {

int nufft_batch_makeplan(int type, int dim, int B, const int64_t* nmodes, int isign, double eps, int prec,
                         void* stream, const nufft_opts* opts, nufft_batch* out) {
  if (!out) return NUFFT_ERR_BAD_ARG;
  *out = nullptr;
  if ((type != 1 && type != 2) || (isign != 1 && isign != -1) || B < 1 || !nmodes || dim < 1 || dim > 3)
    return NUFFT_ERR_BAD_ARG;
  nufft_batch p = new (std::nothrow) nufft_batch_s();
  if (!p) return NUFFT_ERR_ALLOC;
  p->type = type;
  p->dim = dim;
  p->isign = isign;
  p->prec = prec;
  p->dbl = (prec == NUFFT_C128);
  p->csize = p->dbl ? 16 : 8;
  p->B = B;
  if (opts) p->opts = *opts;
  else nufft_default_opts(&p->opts);
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) return batch_fail(p, NUFFT_ERR_CUDA);
  // per-transform parameters; the widest grid sets the shared bin shape
  std::vector<int64_t> n((size_t)B * 3, 1);
  int warn = NUFFT_OK;
  for (int t = 0; t < B; ++t) {
    int w;
    double beta;
    int st = choose_params_impl(dim, nmodes + (size_t)t * dim, eps, prec, &w, &beta, &n[(size_t)t * 3],
                                sigma_of(p->opts));
    if (st < 0) return batch_fail(p, st);
    warn = st;
    p->w = w;
    p->beta = beta;
    for (int i = 0; i < dim; ++i)
      if (nmodes[(size_t)t * dim + i] > (1 << 29) || n[(size_t)t * 3 + i] > (1 << 30)) return batch_fail(p, NUFFT_ERR_TOO_BIG);
  }
  Geom& g = p->g;
  g.d = dim;
  g.w = p->w;
  g.half = p->w / 2;
  g.maxsub = p->opts.max_subprob > 0 ? std::min(p->opts.max_subprob, 8192) : (p->dbl ? 512 : 1024);
  g.sparse_max = sparse_max_of(p->opts);
  g.horner = p->opts.kerevalmeth == 1 ? 1 : 0;
  g.kernel = p->opts.kernel == 1 ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    int64_t mx = 1;
    for (int t = 0; t < B; ++t) mx = std::max(mx, n[(size_t)t * 3 + i]);
    g.n[i] = (int)mx;
  }
  choose_bins(g, p->dbl, p->opts);
  // size classes (one batched FFT each), grid offsets by class, everything else in transform order
  p->hg.resize(B);
  std::vector<int> cls(B);
  for (int t = 0; t < B; ++t) {
    int k = -1;
    for (size_t c = 0; c < p->classes.size(); ++c)
      if (p->classes[c].n[0] == n[(size_t)t * 3] && p->classes[c].n[1] == n[(size_t)t * 3 + 1] &&
          p->classes[c].n[2] == n[(size_t)t * 3 + 2])
        k = (int)c;
    if (k < 0) {
      nufft_batch_s::SizeClass sc;
      for (int i = 0; i < 3; ++i) sc.n[i] = (int)n[(size_t)t * 3 + i];
      sc.count = 0;
      sc.goff = 0;
      sc.ok = false;
      p->classes.push_back(sc);
      k = (int)p->classes.size() - 1;
    }
    cls[t] = k;
    p->classes[k].count++;
  }
  long long goff = 0;
  for (auto& c : p->classes) {
    c.goff = goff;
    goff += (long long)c.count * c.n[0] * c.n[1] * c.n[2];
  }
  p->total_grid = goff;
  std::vector<int> seen(p->classes.size(), 0);
  std::vector<int> hboff(B + 1, 0);
  std::vector<long long> hgrow(B + 1, 0), hmrow(B + 1, 0);
  long long moff = 0, pkoff = 0;
  int boffc = 0;
  for (int t = 0; t < B; ++t) {
    BatchGeom& tg = p->hg[t];
    Geom gt = g;
    for (int i = 0; i < 3; ++i) gt.n[i] = (int)n[(size_t)t * 3 + i];
    finish_geom(gt);
    int64_t Nt = 1;
    for (int i = 0; i < 3; ++i) {
      tg.n[i] = gt.n[i];
      tg.nb[i] = gt.nb[i];
      tg.ns[i] = gt.ns[i];
      tg.sb[i] = gt.sb[i];
      tg.lsb[i] = gt.lsb[i];
      tg.N[i] = i < dim ? (int)nmodes[(size_t)t * dim + i] : 1;
      Nt *= tg.N[i];
      tg.fs[i] = (double)tg.n[i] / 6.283185307179586476925286766559;
      tg.fs_hi[i] = (float)tg.fs[i];
      tg.fs_lo[i] = (float)(tg.fs[i] - (double)tg.fs_hi[i]);
      tg.pkoff[i] = (int)pkoff;
      pkoff += tg.N[i];
    }
    tg.nbins = gt.nbins;
    tg.boff = boffc;
    hboff[t] = boffc;
    boffc += gt.nbins;
    const auto& c = p->classes[cls[t]];
    tg.goff = c.goff + (long long)seen[cls[t]]++ * c.n[0] * c.n[1] * c.n[2];
    tg.moff = moff;
    moff += Nt;
    tg.growoff = hgrow[t];
    hgrow[t + 1] = hgrow[t] + (long long)tg.n[1] * tg.n[2];
    tg.mrowoff = hmrow[t];
    hmrow[t + 1] = hmrow[t] + (long long)tg.N[1] * tg.N[2];
    p->max_grow = std::max(p->max_grow, tg.n[0]);
    p->max_mrow = std::max(p->max_mrow, tg.N[0]);
  }
  if ((long long)boffc >= (1LL << 31) - 1) return batch_fail(p, NUFFT_ERR_TOO_BIG);
  hboff[B] = boffc;
  p->total_bins = boffc;
  p->total_modes = moff;
  p->total_grow = hgrow[B];
  p->total_mrow = hmrow[B];
  // correction factors of every transform and dimension, one array
  std::vector<double> pkh((size_t)pkoff, 1.0);
  for (int t = 0; t < B; ++t)
    for (int i = 0; i < dim; ++i)
      if (correction_impl(p->hg[t].N[i], p->hg[t].n[i], p->w, p->beta, &pkh[p->hg[t].pkoff[i]], p->opts.kernel) !=
          NUFFT_OK)
        return batch_fail(p, NUFFT_ERR_BAD_ARG);
  const size_t rs = p->dbl ? 8 : 4;
  if (dev_alloc(&p->grid, (size_t)p->total_grid * p->csize) != cudaSuccess ||
      dev_alloc(&p->pk, pkh.size() * rs) != cudaSuccess ||
      dev_alloc(&p->bg, sizeof(BatchGeom) * (size_t)B) != cudaSuccess ||
      dev_alloc(&p->boff, sizeof(int) * (size_t)(B + 1)) != cudaSuccess ||
      dev_alloc(&p->poff, sizeof(int) * (size_t)(B + 1)) != cudaSuccess ||
      dev_alloc(&p->growoff, sizeof(long long) * (size_t)(B + 1)) != cudaSuccess ||
      dev_alloc(&p->mrowoff, sizeof(long long) * (size_t)(B + 1)) != cudaSuccess ||
      dev_alloc(&p->bin_count, sizeof(int) * (size_t)p->total_bins) != cudaSuccess ||
      dev_alloc(&p->bin_start, sizeof(int) * (size_t)p->total_bins) != cudaSuccess ||
      dev_alloc(&p->sub_first, sizeof(int) * (size_t)p->total_bins) != cudaSuccess ||
      dev_alloc(&p->cursor, sizeof(int) * (size_t)p->total_bins * (size_t)(p->nrep = replicas_for(p->total_bins))) !=
          cudaSuccess ||
      dev_alloc(&p->rep_count, sizeof(int) * (size_t)p->total_bins * (size_t)p->nrep) != cudaSuccess ||
      dev_alloc(&p->small, sizeof(int) * 4) != cudaSuccess)
    return batch_fail(p, NUFFT_ERR_ALLOC);
  bool okc = true;
  if (p->dbl) {
    okc &= cudaMemcpy(p->pk, pkh.data(), pkh.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  } else {
    std::vector<float> pf(pkh.begin(), pkh.end());
    okc &= cudaMemcpy(p->pk, pf.data(), pf.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  okc &= cudaMemcpy(p->bg, p->hg.data(), sizeof(BatchGeom) * (size_t)B, cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(p->boff, hboff.data(), sizeof(int) * (size_t)(B + 1), cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(p->growoff, hgrow.data(), sizeof(long long) * (size_t)(B + 1), cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemcpy(p->mrowoff, hmrow.data(), sizeof(long long) * (size_t)(B + 1), cudaMemcpyHostToDevice) == cudaSuccess;
  okc &= cudaMemset(p->small, 0, sizeof(int) * 4) == cudaSuccess;
  if (!okc) return batch_fail(p, NUFFT_ERR_CUDA);
  int threads = p->opts.threads > 0 ? p->opts.threads : 256;
  if (threads % 32 != 0 || threads > 256 || p->opts.kerevalmeth < 0 || p->opts.kerevalmeth > 1 ||
      p->opts.kernel < 0 || p->opts.kernel > 1)
    return batch_fail(p, NUFFT_ERR_BAD_ARG);
  cudaError_t e = (type == 1) ? spread_config(p->dbl, g, threads, &p->cfg) : interp_config(p->dbl, g, threads, &p->cfg);
  if (e != cudaSuccess) return batch_fail(p, NUFFT_ERR_CUDA);
  for (auto& c : p->classes) {
    int nn[3];
    for (int i = 0; i < dim; ++i) nn[i] = c.n[dim - 1 - i];
    const int dist = c.n[0] * c.n[1] * c.n[2];
    if (cufftPlanMany(&c.plan, dim, nn, nullptr, 1, dist, nullptr, 1, dist, p->dbl ? CUFFT_Z2Z : CUFFT_C2C,
                      c.count) != CUFFT_SUCCESS)
      return batch_fail(p, NUFFT_ERR_CUFFT);
    c.ok = true;
    if (cufftSetStream(c.plan, p->stream) != CUFFT_SUCCESS) return batch_fail(p, NUFFT_ERR_CUFFT);
  }
  *out = p;
  return warn;
}

int nufft_batch_setpts(nufft_batch p, const int64_t* offsets, const void* x, const void* y, const void* z) {
  if (!p || !offsets || offsets[0] != 0) return NUFFT_ERR_BAD_ARG;
  for (int t = 0; t < p->B; ++t)
    if (offsets[t + 1] < offsets[t]) return NUFFT_ERR_BAD_ARG;
  const int64_t M = offsets[p->B];
  if (M >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_TOO_BIG;
  if (M > 0 && (!x || (p->dim > 1 && !y) || (p->dim > 2 && !z))) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  p->hpoff.assign(offsets, offsets + p->B + 1);
  // pageable source: the copy is staged before the call returns
  if (cudaMemcpyAsync(p->poff, p->hpoff.data(), sizeof(int) * (size_t)(p->B + 1), cudaMemcpyHostToDevice, p->stream) !=
      cudaSuccess)
    return NUFFT_ERR_CUDA;
  if (M > p->Mcap) {
    cudaFree(p->rec);
    p->rec = nullptr;
    p->Mcap = 0;
    if (dev_alloc(&p->rec, (p->dbl ? sizeof(RecD) : sizeof(RecF)) * (size_t)M) != cudaSuccess) return NUFFT_ERR_ALLOC;
    p->Mcap = M;
  }
  int64_t need = std::min<int64_t>(p->total_bins, M) + M / p->g.maxsub + 1;
  if (need > p->subcap) {
    cudaFree(p->sub_bin);
    cudaFree(p->sub_pt0);
    cudaFree(p->sub_cnt);
    p->sub_bin = p->sub_pt0 = p->sub_cnt = nullptr;
    p->subcap = 0;
    if (dev_alloc(&p->sub_bin, sizeof(int) * (size_t)need) != cudaSuccess ||
        dev_alloc(&p->sub_pt0, sizeof(int) * (size_t)need) != cudaSuccess ||
        dev_alloc(&p->sub_cnt, sizeof(int) * (size_t)need) != cudaSuccess)
      return NUFFT_ERR_ALLOC;
    p->subcap = need;
  }
  FoldConst fc = make_fold_const(p->g);
  cudaError_t e = launch_setpts(p->dbl, p->g, fc, M, x, y, z, p->opts.chkbnds, p->bin_count, p->bin_start,
                                p->sub_first, p->cursor, p->rec, p->sub_bin, p->sub_pt0, p->sub_cnt, p->small + 1,
                                p->small + 3, p->small + 0, p->stream, nullptr, table_of(p), p->total_bins,
                                Replicas{p->nrep, p->rep_count, p->cursor});
  if (e != cudaSuccess) return NUFFT_ERR_CUDA;
  p->M = M;
  return NUFFT_OK;
}

int nufft_batch_execute(nufft_batch p, void* c, void* f) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (p->M < 0) return NUFFT_ERR_NOT_SET;
  if (!f || (p->M > 0 && !c)) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  const void* key[4] = {c, f, p->rec, p->sub_bin};
  bool same = p->gexec != nullptr;
  for (int i = 0; i < 4; ++i) same = same && key[i] == p->gkey[i];
  if (!same) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    // capture the execute sequence once; replay it while the pointers stay the same
    cudaGraph_t graph = nullptr;
    if (p->stream && cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int r = batch_enqueue(p, c, f);
      cudaError_t ce = cudaStreamEndCapture(p->stream, &graph);
      if (r == NUFFT_OK && ce == cudaSuccess && graph &&
          cudaGraphInstantiate(&p->gexec, graph, 0) == cudaSuccess) {
        for (int i = 0; i < 4; ++i) p->gkey[i] = key[i];
      } else {
        p->gexec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    }
    if (!p->gexec) return batch_enqueue(p, c, f);  // no capture on the legacy default stream
  }
  return cudaGraphLaunch(p->gexec, p->stream) == cudaSuccess ? NUFFT_OK : NUFFT_ERR_CUDA;
}

int nufft_batch_destroy(nufft_batch p) {
  if (!p) return NUFFT_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  for (auto& c : p->classes)
    if (c.ok) cufftDestroy(c.plan);
  void* bufs[] = {p->grid, p->pk, p->bg, p->boff, p->poff, p->growoff, p->mrowoff, p->bin_count, p->bin_start,
                  p->sub_first, p->cursor, p->rep_count, p->small, p->rec, p->sub_bin, p->sub_pt0, p->sub_cnt};
  for (void* b : bufs)
    if (b) cudaFree(b);
  cudaSetDevice(dev);
  delete p;
  return NUFFT_OK;
}

int nufft_batch_get_status(nufft_batch p) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->small, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (err != 0 && cudaMemset(p->small, 0, sizeof(int)) != cudaSuccess) return NUFFT_ERR_CUDA;
  return err;
}

}  // extern "C"
