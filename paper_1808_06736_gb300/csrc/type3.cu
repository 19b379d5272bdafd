// Type 3 (non-uniform to non-uniform, Eq. (3)) by the algorithm of Sec. 3.3:
// "a type 1 wrapped around a type 2".
//
// setpts  bounding boxes of sources and targets (a device reduction read by
//         the host), their centres x0, s0 and half-widths X_i, S_i; the fine
//         grid n_i = next235(max(2 sigma X_i S_i / pi + w, 2w)) and dilation
//         gamma_i = n_i / (2 sigma S_i) (Eq. (ng)); the dilated sources
//         x' = (x - x0) / gamma binned onto the n_i grid; the rescaled targets
//         s'' = h gamma (s - s0) set on an inner type-2 plan whose modes are
//         that grid (FFT order); per source the translation phase
//         exp(i isign s0.(x - x0)) and per target the correction
//         prod_i 2 / (w phi^(alpha_i gamma_i (s - s0)_i)) (step 3; the
//         Gauss-Legendre rule of Eq. (quad) with p nodes, no phase winding at
//         non-uniform frequencies) times exp(i isign s.x0) (Eq. (trans)),
//         all phases formed in double precision.
// execute c' = c * phase; spread c' onto the grid (step 1, Eq. (blt3)); the
//         inner type 2 evaluates the grid as a Fourier series at s''
//         (step 2, Eq. (bkt3)); f = correction * result (step 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <new>
#include <utility>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

constexpr int kMinMaxBlocks = 256;
constexpr int kMaxGL = 32;  // p = ceil(1.5 w + 2) <= 26 for w <= 16

struct GLRule {
  double q[kMaxGL];   // positive nodes
  double wf[kMaxGL];  // weight * phi(node)
  float qf[kMaxGL], wff[kMaxGL];  // the same, rounded to float
  int p;
};

template <typename T>
struct CT {
  T x, y;
};

// e^{i a} for a phase formed in double.  complex64: a reduced to [-pi, pi]
// in double, then the float sine and cosine (error ~1e-7, below what float
// coordinates already carry); complex128: the double ones.
template <typename T>
__device__ __forceinline__ CT<T> unit_phase(double a);
template <>
__device__ __forceinline__ CT<float> unit_phase<float>(double a) {
  const double r = a - 6.283185307179586 * rint(a * 0.15915494309189535);
  float sn, cs;
  sincosf((float)r, &sn, &cs);
  return CT<float>{cs, sn};
}
template <>
__device__ __forceinline__ CT<double> unit_phase<double>(double a) {
  double sn, cs;
  sincos(a, &sn, &cs);
  return CT<double>{cs, sn};
}

// 2 / (w phi^(xi)) with phi^(xi) = 2 sum_q w_q phi(q) cos(xi q) over the
// positive Gauss-Legendre nodes (Eq. (quad)); complex64 plans work in float
// (|xi q| < 2 pi w; the FP64 pipe would otherwise bind this kernel)
template <typename T>
__device__ __forceinline__ T corr_factor(double xi, T w, const GLRule& gl);
template <>
__device__ __forceinline__ float corr_factor<float>(double xi, float w, const GLRule& gl) {
  const float xf = (float)xi;
  float ft = 0.0f;
  for (int q = 0; q < gl.p; ++q) ft = fmaf(gl.wff[q], cosf(xf * gl.qf[q]), ft);
  return 1.0f / (w * ft);
}
template <>
__device__ __forceinline__ double corr_factor<double>(double xi, double w, const GLRule& gl) {
  double ft = 0.0;
  for (int q = 0; q < gl.p; ++q) ft += gl.wf[q] * cos(xi * gl.q[q]);
  return 1.0 / (w * ft);
}

// per-dimension min and max of up to three coordinate arrays, one partial per block
template <typename T>
__global__ void k_minmax(int64_t n, int d, const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c,
                         double* __restrict__ part) {
  // min and max are exact in the input precision; partials are widened at the end
  T mn[3] = {T(INFINITY), T(INFINITY), T(INFINITY)}, mx[3] = {-T(INFINITY), -T(INFINITY), -T(INFINITY)};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v[3] = {a[i], d > 1 ? b[i] : T(0), d > 2 ? c[i] : T(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      mn[k] = fmin(mn[k], v[k]);
      mx[k] = fmax(mx[k], v[k]);
    }
  }
  __shared__ T smn[3][32], smx[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[k] = fmin(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
      mx[k] = fmax(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    }
    if (lane == 0) {
      smn[k][wid] = mn[k];
      smx[k][wid] = mx[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      T u = T(INFINITY), v = -T(INFINITY);
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        u = fmin(u, smn[k][q]);
        v = fmax(v, smx[k][q]);
      }
      part[blockIdx.x * 6 + k] = (double)u;
      part[blockIdx.x * 6 + 3 + k] = (double)v;
    }
  }
}

struct Affine {
  double shift[3], scale[3];
};

// sources: x' = (x - x0) / gamma and the translation phase exp(i isign s0.(x - x0))
template <typename T>
__global__ void k_t3_sources(int64_t M, int d, const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z,
                             Affine src, double s0x, double s0y, double s0z, int isign, T* __restrict__ xo,
                             T* __restrict__ yo, T* __restrict__ zo, CT<T>* __restrict__ phase) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    const double u0 = (double)x[j] - src.shift[0];
    const double u1 = d > 1 ? (double)y[j] - src.shift[1] : 0.0;
    const double u2 = d > 2 ? (double)z[j] - src.shift[2] : 0.0;
    xo[j] = (T)(u0 * src.scale[0]);
    if (d > 1) yo[j] = (T)(u1 * src.scale[1]);
    if (d > 2) zo[j] = (T)(u2 * src.scale[2]);
    phase[j] = unit_phase<T>((double)isign * (s0x * u0 + s0y * u1 + s0z * u2));
  }
}

// targets: s'' = h gamma (s - s0) for the inner type 2, and the step-3 factor
//   prod_i 2 / (w phi^(alpha_i gamma_i (s - s0)_i)) * exp(i isign s.x0)
template <typename T>
__global__ void k_t3_targets(int64_t N, int d, const T* __restrict__ s, const T* __restrict__ t,
                             const T* __restrict__ u, Affine tgt, double x0x, double x0y, double x0z, int isign,
                             double w, const double* __restrict__ alpha_gamma, GLRule gl, T* __restrict__ so,
                             T* __restrict__ to, T* __restrict__ uo, CT<T>* __restrict__ corr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const double v[3] = {(double)s[k], d > 1 ? (double)t[k] : 0.0, d > 2 ? (double)u[k] : 0.0};
    T p = T(1);
    for (int i = 0; i < d; ++i) {
      const double sc = v[i] - tgt.shift[i];
      const double so_i = sc * tgt.scale[i];
      if (i == 0) so[k] = (T)so_i;
      if (i == 1) to[k] = (T)so_i;
      if (i == 2) uo[k] = (T)so_i;
      // alpha_i s'_i with s' = gamma (s - s0)
      p *= corr_factor<T>(alpha_gamma[i] * sc, (T)w, gl);
    }
    const CT<T> e = unit_phase<T>((double)isign * (v[0] * x0x + v[1] * x0y + v[2] * x0z));
    corr[k] = CT<T>{p * e.x, p * e.y};
  }
}

template <typename T>
__global__ void k_cmul(int64_t n, const CT<T>* __restrict__ a, const CT<T>* __restrict__ b, CT<T>* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const CT<T> u = a[i], v = b[i];
    out[i] = CT<T>{u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x};
  }
}

int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

struct nufft_plan3_s {
  int dim = 0, isign = 0, prec = 0;
  bool dbl = false;
  size_t cs = 8, rs = 4;
  double eps = 0;
  int w = 0;
  double beta = 0, sigma = 2.0;
  nufft_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t M = -1, N = -1;
  double x0[3] = {0, 0, 0}, s0[3] = {0, 0, 0}, gam[3] = {1, 1, 1};
  int64_t n[3] = {1, 1, 1};
  Geom g;
  LaunchCfg scfg{0, 0, 0};
  void* grid = nullptr;  // n_1 n_2 n_3 complex (step 1's fine grid)
  int64_t gridcap = 0;
  int *bin_count = nullptr, *bin_start = nullptr, *sub_first = nullptr;  // nbins
  int *cursor = nullptr, *rep_count = nullptr;                          // nrep nbins
  int nrep = 1;
  int64_t bincap = 0;
  int* small = nullptr;  // [0] error word, [1] tiled subproblems, [2] work counter, [3] sparse subproblems
  void* rec = nullptr;   // M records
  void* xs[3] = {nullptr, nullptr, nullptr};  // M dilated sources per dimension
  void* phase = nullptr;                      // M complex
  void* cpre = nullptr;                       // M complex
  int64_t Mcap = 0;
  int *sub_bin = nullptr, *sub_pt0 = nullptr, *sub_cnt = nullptr;
  int64_t subcap = 0;
  void* ts[3] = {nullptr, nullptr, nullptr};  // N rescaled targets per dimension
  void* corr = nullptr;                       // N complex
  void* bk = nullptr;                         // N complex
  int64_t Ncap = 0;
  double* part = nullptr;  // min / max partials
  double* dag = nullptr;   // alpha_i gamma_i on the device
  nufft_plan inner = nullptr;
  int64_t inner_n[3] = {0, 0, 0};
};

namespace {

void release(void** b) {
  if (*b) cudaFree(*b);
  *b = nullptr;
}
template <typename P>
void release(P** b) {
  release((void**)b);
}

void free_all(nufft_plan3 p) {
  if (p->inner) nufft_destroy(p->inner);
  p->inner = nullptr;
  void** bufs[] = {&p->grid, (void**)&p->bin_count, (void**)&p->bin_start, (void**)&p->sub_first,
                   (void**)&p->cursor, (void**)&p->rep_count, (void**)&p->small, &p->rec, &p->xs[0], &p->xs[1],
                   &p->xs[2], &p->phase, &p->cpre, (void**)&p->sub_bin, (void**)&p->sub_pt0, (void**)&p->sub_cnt,
                   &p->ts[0], &p->ts[1], &p->ts[2], &p->corr, &p->bk, (void**)&p->part, (void**)&p->dag};
  for (void** b : bufs) release(b);
}

// (re)allocate each of a group of buffers to hold need elements of its size,
// when need exceeds the group's capacity
bool ensure(int64_t& cap, int64_t need, std::initializer_list<std::pair<void**, size_t>> bufs) {
  need = std::max<int64_t>(need, 1);
  if (need <= cap) return true;
  cap = 0;
  for (const auto& b : bufs) {
    release(b.first);
    if (cudaMalloc(b.first, std::max<size_t>(16, (size_t)need * b.second)) != cudaSuccess) return false;
  }
  cap = need;
  return true;
}

template <typename T>
int bounds(nufft_plan3 p, int64_t n, const void* a, const void* b, const void* c, double* lo, double* hi) {
  k_minmax<T><<<kMinMaxBlocks, 256, 0, p->stream>>>(n, p->dim, (const T*)a, (const T*)(b ? b : a),
                                                     (const T*)(c ? c : a), p->part);
  if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
  std::vector<double> h((size_t)kMinMaxBlocks * 6);
  if (cudaMemcpyAsync(h.data(), p->part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess)
    return NUFFT_ERR_CUDA;
  for (int k = 0; k < 3; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
    for (int q = 0; q < kMinMaxBlocks; ++q) {
      lo[k] = std::min(lo[k], h[(size_t)q * 6 + k]);
      hi[k] = std::max(hi[k], h[(size_t)q * 6 + 3 + k]);
    }
  }
  for (int k = 0; k < p->dim; ++k)
    if (!std::isfinite(lo[k]) || !std::isfinite(hi[k])) return NUFFT_ERR_OUT_OF_RANGE;
  return NUFFT_OK;
}

template <typename T>
int setpts_t(nufft_plan3 p, int64_t M, const void* x, const void* y, const void* z, int64_t N, const void* s,
             const void* t, const void* u) {
  const int d = p->dim;
  const double pi = 3.14159265358979323846;
  double xl[3] = {0, 0, 0}, xh[3] = {0, 0, 0}, sl[3] = {0, 0, 0}, sh[3] = {0, 0, 0};
  int rc;
  if (M > 0 && (rc = bounds<T>(p, M, x, y, z, xl, xh)) != NUFFT_OK) return rc;
  if (N > 0 && (rc = bounds<T>(p, N, s, t, u, sl, sh)) != NUFFT_OK) return rc;
  // step 0: centres, half-widths, grid and dilation (Eq. (ng), Eq. (cond1))
  for (int i = 0; i < 3; ++i) {
    p->x0[i] = i < d && M > 0 ? 0.5 * (xl[i] + xh[i]) : 0.0;
    p->s0[i] = i < d && N > 0 ? 0.5 * (sl[i] + sh[i]) : 0.0;
    p->n[i] = 1;
    p->gam[i] = 1.0;
    if (i >= d) continue;
    const double X = M > 0 ? 0.5 * (xh[i] - xl[i]) : 0.0, S = N > 0 ? 0.5 * (sh[i] - sl[i]) : 0.0;
    const double want = std::ceil(2.0 * p->sigma / pi * X * S + p->w);
    if (!(want < 1e9)) return NUFFT_ERR_TOO_BIG;
    const int64_t nn = nufft_next235(std::max<int64_t>((int64_t)want, 2 * (int64_t)p->w));
    if (nn < 0 || nn > (1 << 29)) return NUFFT_ERR_TOO_BIG;
    p->n[i] = nn;
    if (S > 0) p->gam[i] = (double)nn / (2.0 * p->sigma * S);
    else p->gam[i] = X > 0 ? X / (pi * (1.0 - (double)p->w / (double)nn)) : 1.0;
  }
  const int64_t ngrid = p->n[0] * p->n[1] * p->n[2];
  if (ngrid > ((int64_t)1 << 34)) return NUFFT_ERR_TOO_BIG;
  // the spreading grid and its bins
  Geom& g = p->g;
  g.d = d;
  g.w = p->w;
  g.half = p->w / 2;
  for (int i = 0; i < 3; ++i) g.n[i] = (int)p->n[i];
  g.maxsub = p->opts.max_subprob > 0 ? std::min(p->opts.max_subprob, 8192) : (p->dbl ? 512 : 1024);
  g.sparse_max = p->opts.sparse_max < 0 ? 0 : (p->opts.sparse_max == 0 ? 32 : std::min(p->opts.sparse_max, 32));
  g.horner = p->opts.kerevalmeth == 1 ? 1 : 0;
  g.kernel = p->opts.kernel == 1 ? 1 : 0;
  plan_choose_bins(g, p->dbl, p->opts);
  const int threads = p->opts.threads > 0 ? p->opts.threads : 256;
  if (threads % 32 != 0 || threads > 256 || p->opts.kerevalmeth < 0 || p->opts.kerevalmeth > 1 ||
      p->opts.kernel < 0 || p->opts.kernel > 1)
    return NUFFT_ERR_BAD_ARG;
  if (spread_config(p->dbl, g, threads, &p->scfg) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (!ensure(p->gridcap, ngrid, {{&p->grid, p->cs}})) return NUFFT_ERR_ALLOC;
  const int nrep = replicas_for(g.nbins);
  if ((int64_t)nrep * g.nbins > p->bincap * p->nrep || g.nbins > p->bincap) {
    p->bincap = 0;
    int64_t cap = 0;
    if (!ensure(cap, g.nbins, {{(void**)&p->bin_count, sizeof(int)}, {(void**)&p->bin_start, sizeof(int)},
                               {(void**)&p->sub_first, sizeof(int)}}))
      return NUFFT_ERR_ALLOC;
    int64_t rcap = 0;
    if (!ensure(rcap, (int64_t)nrep * g.nbins, {{(void**)&p->cursor, sizeof(int)}, {(void**)&p->rep_count, sizeof(int)}}))
      return NUFFT_ERR_ALLOC;
    p->bincap = g.nbins;
    p->nrep = nrep;
  }
  // sources: dilated coordinates and translation phases
  const size_t recsz = p->dbl ? sizeof(RecD) : sizeof(RecF);
  if (!ensure(p->Mcap, M,
              {{&p->rec, recsz}, {&p->xs[0], p->rs}, {&p->xs[1], p->rs}, {&p->xs[2], p->rs}, {&p->phase, p->cs},
               {&p->cpre, p->cs}}))
    return NUFFT_ERR_ALLOC;
  const int64_t need = std::min<int64_t>(g.nbins, M) + M / g.maxsub + 1;
  if (!ensure(p->subcap, need,
              {{(void**)&p->sub_bin, sizeof(int)}, {(void**)&p->sub_pt0, sizeof(int)}, {(void**)&p->sub_cnt, sizeof(int)}}))
    return NUFFT_ERR_ALLOC;
  if (M > 0) {
    Affine src;
    for (int i = 0; i < 3; ++i) {
      src.shift[i] = p->x0[i];
      src.scale[i] = 1.0 / p->gam[i];
    }
    k_t3_sources<T><<<blocks_for(M), 256, 0, p->stream>>>(
        M, d, (const T*)x, (const T*)(y ? y : x), (const T*)(z ? z : x), src, p->s0[0], p->s0[1], p->s0[2], p->isign,
        (T*)p->xs[0], (T*)p->xs[1], (T*)p->xs[2], (CT<T>*)p->phase);
    if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
  }
  const FoldConst fc = make_fold_const(g);
  if (launch_setpts(p->dbl, g, fc, M, p->xs[0], d > 1 ? p->xs[1] : nullptr, d > 2 ? p->xs[2] : nullptr, 0,
                    p->bin_count, p->bin_start, p->sub_first, p->cursor, p->rec, p->sub_bin, p->sub_pt0, p->sub_cnt,
                    p->small + 1, p->small + 3, p->small + 0, p->stream, nullptr,
                    BatchTable{nullptr, nullptr, nullptr, nullptr, nullptr, 0}, g.nbins,
                    Replicas{p->nrep, p->rep_count, p->cursor}) != cudaSuccess)
    return NUFFT_ERR_CUDA;
  // targets: rescaled frequencies and the step-3 factors
  if (!ensure(p->Ncap, N,
              {{&p->ts[0], p->rs}, {&p->ts[1], p->rs}, {&p->ts[2], p->rs}, {&p->corr, p->cs}, {&p->bk, p->cs}}))
    return NUFFT_ERR_ALLOC;
  if (N > 0) {
    Affine tgt;
    double ag[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
      tgt.shift[i] = p->s0[i];
      tgt.scale[i] = 2.0 * pi / (double)p->n[i] * p->gam[i];
      ag[i] = pi * p->w / (double)p->n[i] * p->gam[i];
    }
    if (cudaMemcpyAsync(p->dag, ag, sizeof(ag), cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
      return NUFFT_ERR_CUDA;
    GLRule gl;
    gl.p = (int)std::ceil(1.5 * p->w + 2.0);
    if (gl.p > kMaxGL) return NUFFT_ERR_BAD_ARG;
    std::vector<double> q((size_t)gl.p), wq((size_t)gl.p);
    gl_positive_nodes(gl.p, q.data(), wq.data());
    for (int j = 0; j < gl.p; ++j) {
      gl.q[j] = q[(size_t)j];
      gl.wf[j] = wq[(size_t)j] * kernel_value(q[(size_t)j], p->beta, p->g.kernel);
      gl.qf[j] = (float)gl.q[j];
      gl.wff[j] = (float)gl.wf[j];
    }
    k_t3_targets<T><<<blocks_for(N), 256, 0, p->stream>>>(
        N, d, (const T*)s, (const T*)(t ? t : s), (const T*)(u ? u : s), tgt, p->x0[0], p->x0[1], p->x0[2], p->isign,
        (double)p->w, p->dag, gl, (T*)p->ts[0], (T*)p->ts[1], (T*)p->ts[2], (CT<T>*)p->corr);
    if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
    // the host arrays ag, q, wq go out of scope: finish the copy first
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  }
  // step 2's plan: a type 2 whose modes are the grid, in FFT order
  if (!p->inner || p->inner_n[0] != p->n[0] || p->inner_n[1] != p->n[1] || p->inner_n[2] != p->n[2]) {
    if (p->inner) nufft_destroy(p->inner);
    p->inner = nullptr;
    nufft_opts o = p->opts;
    o.modeord = 1;
    o.chkbnds = 0;
    o.debug = 0;
    nufft_plan ip = nullptr;
    const int st = nufft_makeplan(2, d, p->n, p->isign, 1, p->eps, p->prec, p->stream, &o, &ip);
    if (st < 0) return st;
    p->inner = ip;
    for (int i = 0; i < 3; ++i) p->inner_n[i] = p->n[i];
  }
  rc = nufft_setpts(p->inner, N, p->ts[0], d > 1 ? p->ts[1] : nullptr, d > 2 ? p->ts[2] : nullptr);
  if (rc < 0) return rc;
  p->M = M;
  p->N = N;
  return NUFFT_OK;
}

template <typename T>
int execute_t(nufft_plan3 p, const void* c, void* f) {
  const int64_t M = p->M, N = p->N;
  if (M > 0) {
    k_cmul<T><<<blocks_for(M), 256, 0, p->stream>>>(M, (const CT<T>*)c, (const CT<T>*)p->phase, (CT<T>*)p->cpre);
    if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
  }
  const size_t gbytes = (size_t)(p->n[0] * p->n[1] * p->n[2]) * p->cs;
  if (cudaMemsetAsync(p->grid, 0, gbytes, p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (M > 0) {
    if (cudaMemsetAsync(p->small + 2, 0, sizeof(int), p->stream) != cudaSuccess) return NUFFT_ERR_CUDA;
    Sorted so{p->rec, p->sub_bin, p->sub_pt0, p->sub_cnt, p->small + 1, p->small + 3, p->small};
    if (launch_spread(p->dbl, p->g, p->beta, so, p->cpre, p->grid, p->small + 2, p->scfg, p->stream) != cudaSuccess)
      return NUFFT_ERR_CUDA;
  }
  if (N == 0) return NUFFT_OK;
  int rc = nufft_execute(p->inner, p->bk, p->grid);
  if (rc < 0) return rc;
  k_cmul<T><<<blocks_for(N), 256, 0, p->stream>>>(N, (const CT<T>*)p->bk, (const CT<T>*)p->corr, (CT<T>*)f);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ERR_CUDA;
}

}  // namespace

extern "C" {

int nufft3_makeplan(int dim, int isign, double eps, int prec, void* stream, const nufft_opts* opts,
                    nufft_plan3* out) {
  if (!out) return NUFFT_ERR_BAD_ARG;
  *out = nullptr;
  if (dim < 1 || dim > 3 || (isign != 1 && isign != -1)) return NUFFT_ERR_BAD_ARG;
  nufft_opts o;
  if (opts) o = *opts;
  else nufft_default_opts(&o);
  const double sigma = sigma_from_opts(o);
  int w;
  double beta;
  int64_t ones[3] = {1, 1, 1}, nn[3];
  int warn = nufft_choose_params_sigma(dim, ones, eps, prec, sigma, &w, &beta, nn);
  if (warn < 0) return warn;
  nufft_plan3 p = new (std::nothrow) nufft_plan3_s();
  if (!p) return NUFFT_ERR_ALLOC;
  p->dim = dim;
  p->isign = isign;
  p->prec = prec;
  p->dbl = prec == NUFFT_C128;
  p->cs = p->dbl ? 16 : 8;
  p->rs = p->dbl ? 8 : 4;
  p->eps = eps;
  p->w = w;
  p->beta = beta;
  p->sigma = sigma;
  p->opts = o;
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->part, sizeof(double) * 6 * kMinMaxBlocks) != cudaSuccess ||
      cudaMalloc(&p->dag, sizeof(double) * 3) != cudaSuccess || cudaMalloc(&p->small, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(p->small, 0, sizeof(int) * 4) != cudaSuccess) {
    free_all(p);
    delete p;
    return NUFFT_ERR_ALLOC;
  }
  *out = p;
  return warn;
}

int nufft3_setpts(nufft_plan3 p, int64_t M, const void* x, const void* y, const void* z, int64_t N, const void* s,
                  const void* t, const void* u) {
  if (!p || M < 0 || N < 0) return NUFFT_ERR_BAD_ARG;
  if (M >= ((int64_t)1 << 31) - 1 || N >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_TOO_BIG;
  if (M > 0 && (!x || (p->dim > 1 && !y) || (p->dim > 2 && !z))) return NUFFT_ERR_BAD_ARG;
  if (N > 0 && (!s || (p->dim > 1 && !t) || (p->dim > 2 && !u))) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  p->M = p->N = -1;
  return p->dbl ? setpts_t<double>(p, M, x, y, z, N, s, t, u) : setpts_t<float>(p, M, x, y, z, N, s, t, u);
}

int nufft3_execute(nufft_plan3 p, const void* c, void* f) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (p->M < 0) return NUFFT_ERR_NOT_SET;
  if ((p->M > 0 && !c) || (p->N > 0 && !f)) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) return NUFFT_ERR_CUDA;
  return p->dbl ? execute_t<double>(p, c, f) : execute_t<float>(p, c, f);
}

int nufft3_plan_info(nufft_plan3 p, int* w, double* beta, int64_t* n, double* gamma) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (w) *w = p->w;
  if (beta) *beta = p->beta;
  for (int i = 0; i < p->dim; ++i) {
    if (n) n[i] = p->n[i];
    if (gamma) gamma[i] = p->gam[i];
  }
  return NUFFT_OK;
}

int nufft3_get_status(nufft_plan3 p) {
  if (!p) return NUFFT_ERR_BAD_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess)
    return NUFFT_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->small, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (err != 0) return err;
  return p->inner ? nufft_get_status(p->inner) : NUFFT_OK;
}

int nufft3_destroy(nufft_plan3 p) {
  if (!p) return NUFFT_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  free_all(p);
  cudaSetDevice(dev);
  delete p;
  return NUFFT_OK;
}

}  // extern "C"
