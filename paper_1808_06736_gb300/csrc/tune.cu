// Autotuner: time launch configurations on the caller's own data and keep
// the fastest.  The tunables are the bin extents (which also fix the
// shared-memory tile, bin + w per dimension), the largest subproblem, the
// threads per block, the threshold below which a subproblem runs one per
// warp (the per-warp path's lanes cooperate on a point's stencil, the tiled
// path gives each thread its own points), the kernel evaluation (the ES
// formula or the piecewise polynomial of Sec. 5.3) and the upsampling factor
// (2, or 5/4 where eps allows: a grid about 4x smaller in 3D for a wider
// kernel).  The search is staged: bin shapes first, then the subproblem size,
// the sparse threshold, the block size, the kernel evaluation and the
// upsampling factor, each stage
// starting from the best configuration so far.  The default configuration is
// always timed first, so the result is never slower than it as measured.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

constexpr size_t kSmemLimit = 200 * 1024;  // below the 227 KB per-block maximum, leaving room for static smem

// Bin shapes tried for this dimension: 1D 256..4096; 2D every pair of
// {8, 16, 32, 64}; 3D every B1 >= B2 >= B3 of {4, 8, 16, 32} (x, the
// contiguous axis, widest).  Shapes whose spread tile does not fit in shared
// memory at width w are left out.
std::vector<std::array<int, 3>> bin_shapes(int dim, bool dbl, int w, int maxsub) {
  std::vector<std::array<int, 3>> all;
  if (dim == 1) {
    for (int b : {256, 512, 1024, 2048, 4096}) all.push_back({b, 1, 1});
  } else if (dim == 2) {
    for (int b0 : {8, 16, 32, 64})
      for (int b1 : {8, 16, 32, 64}) all.push_back({b0, b1, 1});
  } else {
    for (int b0 : {4, 8, 16, 32})
      for (int b1 : {4, 8, 16, 32})
        for (int b2 : {4, 8, 16, 32})
          if (b0 >= b1 && b1 >= b2) all.push_back({b0, b1, b2});
  }
  std::vector<std::array<int, 3>> out;
  for (const auto& b : all) {
    Geom g{};
    g.d = dim;
    g.w = w;
    g.half = w / 2;
    g.maxsub = maxsub;
    for (int i = 0; i < 3; ++i) {
      g.n[i] = i < dim ? (1 << 20) : 1;  // the tile size does not depend on n
      g.B[i] = i < dim ? b[i] : 1;
    }
    finish_geom(g);
    if (spread_smem_bytes(dbl, g, 256) <= kSmemLimit && interp_smem_bytes(dbl, g, 256) <= kSmemLimit) out.push_back(b);
  }
  return out;
}

struct Trial {
  virtual ~Trial() {}
  virtual int make(const nufft_opts& o) = 0;
  virtual int step() = 0;
  virtual void drop() = 0;
};

// Best (minimum) time of reps steps in ms, or -1 when the configuration fails.
double time_trial(Trial& t, const nufft_opts& o, cudaStream_t st, int reps) {
  if (t.make(o) < 0) {
    t.drop();
    return -1.0;
  }
  double best = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    t.drop();
    return -1.0;
  }
  bool ok = t.step() >= 0 && cudaStreamSynchronize(st) == cudaSuccess;  // untimed warm-up
  for (int r = 0; ok && r < reps; ++r) {
    ok = cudaEventRecord(e0, st) == cudaSuccess && t.step() >= 0 && cudaEventRecord(e1, st) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best < 0 || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  t.drop();
  return ok ? best : -1.0;
}

int search(int dim, bool dbl, int w, bool try_sigma54, Trial& t, cudaStream_t st, int reps, nufft_opts* best,
           double* best_ms, double* default_ms) {
  nufft_opts cur;
  nufft_default_opts(&cur);
  double cur_ms = time_trial(t, cur, st, reps);
  if (cur_ms < 0) return NUFFT_ERR_CUDA;
  if (default_ms) *default_ms = cur_ms;
  auto consider = [&](const nufft_opts& o) {
    double ms = time_trial(t, o, st, reps);
    if (ms >= 0 && ms < cur_ms) {
      cur_ms = ms;
      cur = o;
    }
  };
  const int maxsub0 = dbl ? 512 : 1024;
  for (const auto& b : bin_shapes(dim, dbl, w, maxsub0)) {
    nufft_opts o = cur;
    for (int i = 0; i < 3; ++i) o.bin_size[i] = i < dim ? b[i] : 0;
    consider(o);
  }
  for (int ms : {256, 512, 1024, 2048, 4096}) {
    nufft_opts o = cur;
    if (ms == (cur.max_subprob > 0 ? cur.max_subprob : maxsub0)) continue;
    o.max_subprob = ms;
    consider(o);
  }
  for (int sp : {-1, 8, 16}) {
    nufft_opts o = cur;
    o.sparse_max = sp;
    consider(o);
  }
  {
    nufft_opts o = cur;
    o.threads = 128;
    consider(o);
  }
  {  // the other kernel evaluation (Sec. 5.3's piecewise polynomial, or exp and sqrt per value)
    nufft_opts o = cur;
    o.kerevalmeth = 1 - cur.kerevalmeth;
    consider(o);
  }
  if (try_sigma54) {  // smaller grids and FFTs for a wider kernel; its own default bins
    nufft_opts o = cur;
    o.upsampfac = 1.25;
    o.bin_size[0] = o.bin_size[1] = o.bin_size[2] = 0;
    consider(o);
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return NUFFT_OK;
}

struct PlanTrial : Trial {
  int type, dim, isign, prec;
  const int64_t* nmodes;
  double eps;
  int64_t M;
  const void *x, *y, *z, *in;
  void* out;
  cudaStream_t st;
  nufft_plan p = nullptr;
  int make(const nufft_opts& o) override { return nufft_makeplan(type, dim, nmodes, isign, 1, eps, prec, st, &o, &p); }
  int step() override {
    int rc = nufft_setpts(p, M, x, y, z);
    if (rc < 0) return rc;
    return type == 1 ? nufft_execute(p, (void*)in, out) : nufft_execute(p, out, (void*)in);
  }
  void drop() override {
    if (p) nufft_destroy(p);
    p = nullptr;
  }
};

struct BatchTrial : Trial {
  int type, dim, B, isign, prec;
  const int64_t *nmodes, *offsets;
  double eps;
  const void *x, *y, *z, *in;
  void* out;
  cudaStream_t st;
  nufft_batch p = nullptr;
  int make(const nufft_opts& o) override {
    return nufft_batch_makeplan(type, dim, B, nmodes, isign, eps, prec, st, &o, &p);
  }
  int step() override {
    int rc = nufft_batch_setpts(p, offsets, x, y, z);
    if (rc < 0) return rc;
    return type == 1 ? nufft_batch_execute(p, (void*)in, out) : nufft_batch_execute(p, out, (void*)in);
  }
  void drop() override {
    if (p) nufft_batch_destroy(p);
    p = nullptr;
  }
};

}  // namespace

extern "C" {

int nufft_tune_candidates(int dim, int prec, int w, int* bins, int max) {
  if (dim < 1 || dim > 3 || (prec != NUFFT_C64 && prec != NUFFT_C128) || w < 2 || w > 16 || max < 0 ||
      (max > 0 && !bins))
    return NUFFT_ERR_BAD_ARG;
  const bool dbl = prec == NUFFT_C128;
  auto v = bin_shapes(dim, dbl, w, dbl ? 512 : 1024);
  const int n = (int)v.size();
  for (int k = 0; k < std::min(n, max); ++k)
    for (int i = 0; i < 3; ++i) bins[3 * k + i] = v[(size_t)k][(size_t)i];
  return n;
}

int nufft_tune(int type, int dim, const int64_t* nmodes, int isign, double eps, int prec, int64_t M, const void* x,
               const void* y, const void* z, const void* in, void* out, void* stream, int reps, nufft_opts* best,
               double* best_ms, double* default_ms) {
  if (!best || !nmodes || (type != 1 && type != 2) || dim < 1 || dim > 3 || reps < 1 || M < 0 || !in || !out)
    return NUFFT_ERR_BAD_ARG;
  int w;
  double beta;
  int64_t n[3] = {1, 1, 1};
  int st = nufft_choose_params(dim, nmodes, eps, prec, &w, &beta, n);
  if (st < 0) return st;
  const bool s54 = nufft_choose_params_sigma(dim, nmodes, eps, prec, 1.25, nullptr, nullptr, nullptr) == NUFFT_OK;
  PlanTrial t;
  t.type = type;
  t.dim = dim;
  t.isign = isign;
  t.prec = prec;
  t.nmodes = nmodes;
  t.eps = eps;
  t.M = M;
  t.x = x;
  t.y = y;
  t.z = z;
  t.in = in;
  t.out = out;
  t.st = (cudaStream_t)stream;
  return search(dim, prec == NUFFT_C128, w, s54, t, t.st, reps, best, best_ms, default_ms);
}

int nufft_batch_tune(int type, int dim, int B, const int64_t* nmodes, int isign, double eps, int prec,
                     const int64_t* offsets, const void* x, const void* y, const void* z, const void* in, void* out,
                     void* stream, int reps, nufft_opts* best, double* best_ms, double* default_ms) {
  if (!best || !nmodes || !offsets || (type != 1 && type != 2) || dim < 1 || dim > 3 || B < 1 || reps < 1 || !in ||
      !out)
    return NUFFT_ERR_BAD_ARG;
  int w;
  double beta;
  int64_t n[3] = {1, 1, 1};
  int st = nufft_choose_params(dim, nmodes, eps, prec, &w, &beta, n);  // w depends on eps only
  if (st < 0) return st;
  const bool s54 = nufft_choose_params_sigma(dim, nmodes, eps, prec, 1.25, nullptr, nullptr, nullptr) == NUFFT_OK;
  BatchTrial t;
  t.type = type;
  t.dim = dim;
  t.B = B;
  t.isign = isign;
  t.prec = prec;
  t.nmodes = nmodes;
  t.offsets = offsets;
  t.eps = eps;
  t.x = x;
  t.y = y;
  t.z = z;
  t.in = in;
  t.out = out;
  t.st = (cudaStream_t)stream;
  return search(dim, prec == NUFFT_C128, w, s54, t, t.st, reps, best, best_ms, default_ms);
}

}  // extern "C"
