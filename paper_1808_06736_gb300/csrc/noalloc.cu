// nufft_spread_noalloc: type-1 spreading onto a caller-provided fine grid
// that performs no device memory allocation at all.
//
// Who needs this: callers that run where cudaMalloc is not allowed or not
// safe -- code that is already inside a memory-pool or arena regime owned by
// someone else (a framework allocator that must see every byte), real-time
// or interrupt-like paths that cannot afford an allocation's implicit device
// synchronisation, and plugin hosts that forbid their plugins to allocate.
// Such a caller passes its own inputs and output; the binning arrays this
// spreading step needs (bin counts, cursors, point records, subproblem list)
// live in one fixed-size, file-scope device array instead of plan-owned
// allocations.
//
// The array is a `static __device__` object: every GPU on which the library
// is loaded holds kScratchBytes of it until the process exits, and every call
// shares it.  Calls whose device work overlaps (two streams, or a second call
// before the first has finished on another stream) race on it; serialise
// them.  The host-side address of the array is found once per device with
// cudaGetSymbolAddress, during the first call made with that device current;
// make that first call before any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr int kMaxSub = 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_scratch on the current device (set up once per device).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return NUFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return NUFFT_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return NUFFT_OK;
}

// Bin geometry: the largest bins from a fixed list whose spread kernel fits
// in 110 KB of shared memory.
void pick_bins(Geom& g) {
  static const int c3[][3] = {{16, 8, 8}, {8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {4, 4, 4}};
  static const int c2[][3] = {{32, 32, 1}, {32, 16, 1}, {16, 16, 1}, {16, 8, 1}, {8, 8, 1}};
  static const int c1[][3] = {{1024, 1, 1}, {512, 1, 1}, {256, 1, 1}, {128, 1, 1}, {64, 1, 1}};
  const int(*c)[3] = g.d == 3 ? c3 : (g.d == 2 ? c2 : c1);
  for (int k = 0; k < 5; ++k) {
    for (int i = 0; i < 3; ++i) g.B[i] = i < g.d ? std::max(1, std::min(c[k][i], g.n[i])) : 1;
    finish_geom(g);
    if (spread_smem_bytes(false, g, 256) <= 110 * 1024) break;
  }
}

}  // namespace

extern "C" int nufft_spread_noalloc(int dim, const int64_t* n, int w, double beta, int64_t M,
                                    const float* x, const float* y, const float* z, const void* c,
                                    void* grid, void* stream) {
  if (dim < 1 || dim > 3 || !n || w < 2 || w > 16 || !(beta > 0.0) || M < 0 || !grid)
    return NUFFT_ERR_BAD_ARG;
  if (M > 0 && (!x || !c || (dim > 1 && !y) || (dim > 2 && !z))) return NUFFT_ERR_BAD_ARG;
  // point indices and bin ids are 32-bit on the device: bound M and the grid before any
  // size arithmetic (so nothing below can overflow)
  if (M >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_TOO_BIG;
  Geom g;
  g.d = dim;
  g.w = w;
  g.half = w / 2;
  g.maxsub = kMaxSub;
  g.sparse_max = 32;
  g.horner = 0;
  g.kernel = 0;
  int64_t ngrid = 1;
  for (int i = 0; i < 3; ++i) {
    int64_t v = i < dim ? n[i] : 1;
    if (i < dim && (v < 2 * w || v > (1 << 30))) return NUFFT_ERR_BAD_ARG;
    g.n[i] = (int)v;
    if (ngrid > (((int64_t)1 << 31) - 1) / v) return NUFFT_ERR_TOO_BIG;  // grid cells >= 2^31
    ngrid *= v;
  }
  // bin ids (at most one bin per cell) then fit in int, so finish_geom cannot overflow
  pick_bins(g);
  if (g.nbins <= 0) return NUFFT_ERR_TOO_BIG;

  // carve the scratch array; reject sizes that do not fit
  const int64_t subcap = std::min<int64_t>(g.nbins, M) + M / g.maxsub + 1;
  size_t off = 0;
  const size_t o_count = off; off += align256(sizeof(int) * (size_t)g.nbins);
  const size_t o_start = off; off += align256(sizeof(int) * (size_t)g.nbins);
  const size_t o_first = off; off += align256(sizeof(int) * (size_t)g.nbins);
  const size_t o_cursor = off; off += align256(sizeof(int) * (size_t)g.nbins);
  const size_t o_small = off; off += 256;
  const size_t o_subbin = off; off += align256(sizeof(int) * (size_t)subcap);
  const size_t o_subpt0 = off; off += align256(sizeof(int) * (size_t)subcap);
  const size_t o_subcnt = off; off += align256(sizeof(int) * (size_t)subcap);
  const size_t o_rec = off; off += align256(sizeof(RecF) * (size_t)M);
  if (off > kScratchBytes) return NUFFT_ERR_TOO_BIG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NUFFT_ERR_CUDA;
  unsigned char* s = nullptr;
  int st = scratch_address(dev, &s);
  if (st != NUFFT_OK) return st;
  int* bin_count = (int*)(s + o_count);
  int* bin_start = (int*)(s + o_start);
  int* sub_first = (int*)(s + o_first);
  int* cursor = (int*)(s + o_cursor);
  int* small = (int*)(s + o_small);  // [0] error word, [1] tiled / [3] sparse subproblems, [2] work counter
  int* sub_bin = (int*)(s + o_subbin);
  int* sub_pt0 = (int*)(s + o_subpt0);
  int* sub_cnt = (int*)(s + o_subcnt);
  void* rec = s + o_rec;

  cudaStream_t st_ = (cudaStream_t)stream;
  // the scratch keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(small, 0, 4 * sizeof(int), st_) != cudaSuccess) return NUFFT_ERR_CUDA;
  if (cudaMemsetAsync(grid, 0, (size_t)ngrid * 8, st_) != cudaSuccess) return NUFFT_ERR_CUDA;
  FoldConst fc = make_fold_const(g);
  if (launch_setpts(false, g, fc, M, x, y, z, 0, bin_count, bin_start, sub_first, cursor, rec, sub_bin,
                    sub_pt0, sub_cnt, small + 1, small + 3, small + 0, st_, nullptr) != cudaSuccess)
    return NUFFT_ERR_CUDA;
  if (M == 0) return NUFFT_OK;
  LaunchCfg cfg;
  if (spread_config(false, g, 256, &cfg) != cudaSuccess) return NUFFT_ERR_CUDA;
  Sorted so{rec, sub_bin, sub_pt0, sub_cnt, small + 1, small + 3, small};
  if (launch_spread(false, g, beta, so, c, grid, small + 2, cfg, st_) != cudaSuccess) return NUFFT_ERR_CUDA;
  return NUFFT_OK;
}
