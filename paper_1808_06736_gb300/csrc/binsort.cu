// setpts: fold the points onto the fine grid and bin them by a counting sort.
//
// The paper sorts points into boxes of fine-grid cells before spreading or
// interpolating, with an "incomplete" histogram sort: count per box, prefix
// sum into breakpoints, write each point into its box, no order inside a box
// (Sec. 5.1).  Sorted points are then grouped into subproblems of bounded
// size (Sec. 5.2).  Here:
//   k_fold_count  per point: fold, bin id, count (global atomic reduction)
//   k_scan        one block: bin breakpoints (also the scatter cursors) and
//                 subproblem breakpoints
//   k_sublist     per bin: its subproblems (bin, first record, count)
//   k_scatter     per point: folded coordinates relative to the bin origin,
//                 written as one record at the bin's cursor (atomicAdd)
#include <cmath>

#include "nufft_internal.cuh"

namespace nufft {

FoldConst make_fold_const(const Geom& g) {
  FoldConst f;
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < 3; ++i) {
    double s = (double)g.n[i] / two_pi;
    f.s[i] = s;
    f.s_hi[i] = (float)s;
    f.s_lo[i] = (float)(s - (double)f.s_hi[i]);
  }
  return f;
}

namespace {

constexpr double kThreePi = 9.424777960769379715387930149839;

// i mod n for the cell index of a folded point; one add or subtract covers
// every |x| <= 3 pi, the general remainder only runs for points further out.
__device__ __forceinline__ int wrap_cell(long long i, int n) {
  if (i < 0) i += n;
  if (i >= n) i -= n;
  if ((unsigned long long)i >= (unsigned long long)n) {
    i %= n;
    if (i < 0) i += n;
  }
  return (int)i;
}

// u = x n / (2 pi) split as (cell in [0, n), frac in [0, 1)).  The product is
// formed with an FMA error term and the lo part of n/(2 pi), so frac is
// accurate to about 1e-7 cells even where x n / (2 pi) is ~1e3 (a plain
// float product would lose ~3e-5 cells there, i.e. a phase error of
// N_i * 2^-24 rad, the rounding law of Remark r:rounding).
__device__ __forceinline__ void fold(float x, int n, float s_hi, float s_lo, double, int& cell,
                                     float& frac) {
  float p = x * s_hi;
  float e = fmaf(x, s_hi, -p);
  float corr = fmaf(x, s_lo, e);
  float fl = floorf(p);
  float fr = (p - fl) + corr;  // p - fl is exact
  long long i = (long long)fl;
  if (fr < 0.f) {
    fr += 1.f;
    --i;
  }
  if (fr >= 1.f) {
    fr -= 1.f;
    ++i;
  }
  cell = wrap_cell(i, n);
  frac = fr;
}
__device__ __forceinline__ void fold(double x, int n, float, float, double s, int& cell,
                                     double& frac) {
  double p = x * s;
  double fl = floor(p);
  double fr = p - fl;
  long long i = (long long)fl;
  if (fr >= 1.0) {
    fr -= 1.0;
    ++i;
  }
  cell = wrap_cell(i, n);
  frac = fr;
}

template <typename T>
__device__ __forceinline__ T coord(int dim, int j, const T* x, const T* y, const T* z) {
  return dim == 0 ? x[j] : (dim == 1 ? y[j] : z[j]);
}

// Fold one point into its bin id; sets *bad for |x| > 3 pi (or non-finite)
// when chk is on.
template <typename T>
__device__ __forceinline__ int point_bin(const Geom& g, const FoldConst& fc, const T* xv, int chk,
                                         bool* bad) {
  int b[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < g.d) {
      if (chk) *bad |= !(fabs(xv[i]) <= (T)kThreePi);
      int cell;
      T fr;
      fold(xv[i], g.n[i], fc.s_hi[i], fc.s_lo[i], fc.s[i], cell, fr);
      b[i] = cell / g.B[i];
    }
  }
  return bin_id(g, b[0], b[1], b[2]);
}

// Points are handled four per thread per iteration so that twelve independent
// coordinate loads are in flight before the first one is used.
constexpr int kILP = 4;

// For a batch of transforms, the point's transform (found from the point
// offsets) supplies the fine grid and bin layout, and its bins start at the
// transform's first global bin id.
template <typename T>
__device__ __forceinline__ int point_bin_batch(const Geom& g0, const BatchTable& bt, int j, const T* xv, int chk,
                                               bool* bad) {
  const int t = batch_find(bt.poff, bt.B, j);
  const BatchGeom& tg = bt.bg[t];
  Geom g = g0;
  batch_apply(g, tg);
  int b[3] = {0, 0, 0};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < g.d) {
      if (chk) *bad |= !(fabs(xv[i]) <= (T)kThreePi);
      int cell;
      T fr;
      fold(xv[i], g.n[i], tg.fs_hi[i], tg.fs_lo[i], tg.fs[i], cell, fr);
      b[i] = cell / g.B[i];
    }
  }
  return tg.boff + bin_id(g, b[0], b[1], b[2]);
}

// Bin counters come in nrep replicas (a power of two): point j counts in
// replica j mod nrep, so a crowded bin's increments go to nrep addresses
// instead of one (same-address atomics serialise at the L2: a bin holding
// 0.5% of 1e8 clustered points would otherwise take milliseconds alone).
// The replicas are summed per bin before the scan; in crowded bins each
// replica then gets its own scatter cursor inside the bin's range.
template <typename T>
__global__ void k_fold_count(int M, const T* __restrict__ x, const T* __restrict__ y,
                             const T* __restrict__ z, Geom g, FoldConst fc, int chk,
                             int* __restrict__ rep_count, int nrep, int nbins, int* __restrict__ err, BatchTable bt) {
  const int stride = gridDim.x * blockDim.x;
  bool bad = false;
  for (int j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < M; j0 += kILP * stride) {
    T v[kILP][3];
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int j = j0 + u * stride;
      if (j < M) {
        v[u][0] = x[j];
        v[u][1] = g.d > 1 ? y[j] : T(0);
        v[u][2] = g.d > 2 ? z[j] : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int j = j0 + u * stride;
      if (j < M) {
        const int bin = bt.B > 0 ? point_bin_batch(g, bt, j, v[u], chk, &bad) : point_bin(g, fc, v[u], chk, &bad);
        atomicAdd(&rep_count[(size_t)(j & (nrep - 1)) * nbins + bin], 1);  // result unused
      }
    }
  }
  if (chk && bad) atomicCAS(err, 0, NUFFT_ERR_OUT_OF_RANGE);
}

// Exclusive scans of the bin counts (-> breakpoints and scatter cursors) and
// of the per-bin subproblem counts, in one block: the block walks the bins in
// chunks of blockDim (coalesced), carrying the running totals.
// Inclusive block scan of 64-bit values (1024 threads at most).
__device__ __forceinline__ long long block_incl_scan(long long v, long long* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long u = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += t;
    }
    wsum[lane] = u;
  }
  __syncthreads();
  long long r = v + (wid > 0 ? wsum[wid - 1] : 0);
  __syncthreads();  // wsum reused by the next call
  return r;
}

// Per bin: its full chunks of maxsub points and a remainder; the remainder is
// a tiled subproblem when it holds more than smax points and a per-warp
// ("sparse") one otherwise.  Tiled subproblems are numbered in bin order from
// 0 (sub_first); the sparse ones are appended after them by k_sublist.
__device__ __forceinline__ void split_bin(int c, int maxsub, int smax, int* ntiled, int* sparse) {
  const int full = c / maxsub, rem = c - full * maxsub;
  const bool sp = rem > 0 && rem <= smax;
  *ntiled = full + ((rem > 0 && !sp) ? 1 : 0);
  *sparse = sp ? 1 : 0;
}

// One block.  Per round the block stages SCAN_PER * blockDim.x bin counts in
// shared memory (coalesced), each thread scans SCAN_PER consecutive bins: the
// point count (high 32 bits) and the tiled-subproblem count (low 32 bits) of
// its bins go through one 64-bit block scan; the breakpoints are written back
// through shared memory, again coalesced.
constexpr int SCAN_PER = 4;
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(int nbins, int maxsub, int smax, const int* __restrict__ cnt,
                                                       int* __restrict__ start, int* __restrict__ cursor,
                                                       int* __restrict__ sub_first, int* __restrict__ nsub,
                                                       int* __restrict__ nsparse) {
  constexpr int CHUNK = SCAN_THREADS * SCAN_PER;
  __shared__ int s_a[CHUNK];  // counts, then point breakpoints
  __shared__ int s_b[CHUNK];  // subproblem breakpoints
  __shared__ long long wsum[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nbins; base += CHUNK) {
    const int len = min(CHUNK, nbins - base);
    for (int i = threadIdx.x; i < CHUNK; i += blockDim.x) s_a[i] = i < len ? cnt[base + i] : 0;
    __syncthreads();
    const int t0 = threadIdx.x * SCAN_PER;
    int c[SCAN_PER], sc[SCAN_PER];
    long long tot = 0;
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
      c[u] = s_a[t0 + u];
      int sp;
      split_bin(c[u], maxsub, smax, &sc[u], &sp);
      tot += ((long long)c[u] << 32) + sc[u];
    }
    const long long cy = carry;
    long long run = cy + block_incl_scan(tot, wsum) - tot;
#pragma unroll
    for (int u = 0; u < SCAN_PER; ++u) {
      s_a[t0 + u] = (int)(run >> 32);
      s_b[t0 + u] = (int)(run & 0xffffffffLL);
      run += ((long long)c[u] << 32) + sc[u];
    }
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int v = s_a[i];
      start[base + i] = v;
      cursor[base + i] = v;
      sub_first[base + i] = s_b[i];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *nsub = (int)(carry & 0xffffffffLL);
    *nsparse = 0;
  }
}

// Tiled subproblems at sub_first[b] + k; a sparse remainder at nsub + (an
// append position, taken once per warp so neighbouring bins stay close).
__global__ void k_sublist(int nbins, int maxsub, int smax, const int* __restrict__ cnt,
                          const int* __restrict__ start, const int* __restrict__ sub_first,
                          const int* __restrict__ nsub, int* __restrict__ nsparse, int* __restrict__ sub_bin,
                          int* __restrict__ sub_pt0, int* __restrict__ sub_cnt) {
  const int nt = *nsub;
  const int lane = threadIdx.x & 31;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    const int c = cnt[b];
    int ntl, sp;
    split_bin(c, maxsub, smax, &ntl, &sp);
    const int s0 = sub_first[b], p0 = start[b];
    for (int k = 0; k < ntl; ++k) {
      sub_bin[s0 + k] = b;
      sub_pt0[s0 + k] = p0 + k * maxsub;
      sub_cnt[s0 + k] = min(maxsub, c - k * maxsub);
    }
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, sp);
    if (m) {
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(nsparse, __popc(m));
      base = __shfl_sync(act, base, leader);
      if (sp) {
        const int q = nt + base + __popc(m & ((1u << lane) - 1u));
        const int full = c / maxsub;
        sub_bin[q] = b;
        sub_pt0[q] = p0 + full * maxsub;
        sub_cnt[q] = c - full * maxsub;
      }
    }
  }
}

__global__ void k_rep_sum(int nbins, int nrep, const int* __restrict__ rep_count, int* __restrict__ bin_count) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    int t = 0;
    for (int r = 0; r < nrep; ++r) t += rep_count[(size_t)r * nbins + b];
    bin_count[b] = t;
  }
}

// Only crowded bins scatter through their replica cursors; every other bin
// keeps one cursor (replica 0), so its records are written in arrival order
// into one range and its cursor stays hot in L2.
constexpr int kCrowded = 4096;

// Replica r of a crowded bin b starts after replicas 0..r-1 inside the bin's
// range; crowded bins are also marked in a bit mask (zeroed beforehand).
__global__ void k_rep_cursor(int nbins, int nrep, const int* __restrict__ rep_count, const int* __restrict__ bin_count,
                             const int* __restrict__ start, int* __restrict__ rep_cursor, unsigned* __restrict__ crowd) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    int run = start[b];
    if (bin_count[b] <= kCrowded) {
      rep_cursor[b] = run;
      continue;
    }
    atomicOr(&crowd[b >> 5], 1u << (b & 31));
    for (int r = 0; r < nrep; ++r) {
      const int c = rep_count[(size_t)r * nbins + b];
      rep_cursor[(size_t)r * nbins + b] = run;
      run += c;
    }
  }
}

template <typename T>
__global__ void k_scatter(int M, const T* __restrict__ x, const T* __restrict__ y,
                          const T* __restrict__ z, Geom g0, FoldConst fc0, int* __restrict__ rep_cursor, int nrep,
                          int nbins, const unsigned* __restrict__ crowd, int mask_in_smem,
                          typename Traits<T>::Rec* __restrict__ rec, BatchTable bt) {
  // the crowded-bin mask, staged in shared memory when it fits
  extern __shared__ unsigned s_crowd[];
  const int nwords = (nbins + 31) >> 5;
  if (nrep > 1 && mask_in_smem) {
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) s_crowd[i] = crowd[i];
    __syncthreads();
  }
  const unsigned* mask = mask_in_smem ? s_crowd : crowd;
  const int stride = gridDim.x * blockDim.x;
  for (int j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < M; j0 += kILP * stride) {
    T v[kILP][3];
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int j = j0 + u * stride;
      if (j < M) {
        v[u][0] = x[j];
        v[u][1] = g0.d > 1 ? y[j] : T(0);
        v[u][2] = g0.d > 2 ? z[j] : T(0);
      }
    }
    typename Traits<T>::Rec r[kILP];
    int dest[kILP];
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int j = j0 + u * stride;
      if (j < M) {
        Geom g = g0;
        FoldConst fc = fc0;
        int boff = 0;
        if (bt.B > 0) {
          const BatchGeom& tg = bt.bg[batch_find(bt.poff, bt.B, j)];
          batch_apply(g, tg);
          boff = tg.boff;
          for (int i = 0; i < 3; ++i) {
            fc.s[i] = tg.fs[i];
            fc.s_hi[i] = tg.fs_hi[i];
            fc.s_lo[i] = tg.fs_lo[i];
          }
        }
        int bb[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          r[u].v[i] = T(0);
          if (i < g.d) {
            int cell;
            T fr;
            fold(v[u][i], g.n[i], fc.s_hi[i], fc.s_lo[i], fc.s[i], cell, fr);
            bb[i] = cell / g.B[i];
            r[u].v[i] = T(cell - bb[i] * g.B[i]) + fr;
          }
        }
        r[u].idx = j;
        // order inside a bin is arbitrary
        const int bin = boff + bin_id(g, bb[0], bb[1], bb[2]);
        const int rr = (nrep > 1 && ((mask[bin >> 5] >> (bin & 31)) & 1u)) ? (j & (nrep - 1)) : 0;
        dest[u] = atomicAdd(&rep_cursor[(size_t)rr * nbins + bin], 1);
      }
    }
#pragma unroll
    for (int u = 0; u < kILP; ++u) {
      const int j = j0 + u * stride;
      if (j < M) rec[dest[u]] = r[u];
    }
  }
}

}  // namespace

void finish_geom(Geom& g) {
  // super-blocks of about 64 bins (3D 4x4x4, 2D 8x8, 1D 64)
  const int sbd[4][3] = {{1, 1, 1}, {64, 1, 1}, {8, 8, 1}, {4, 4, 4}};
  int nbins = 1, ntile = 1;
  for (int i = 0; i < 3; ++i) {
    if (i >= g.d) {
      g.n[i] = g.n[i] > 0 ? g.n[i] : 1;
      g.B[i] = 1;
    }
    g.T[i] = (i < g.d) ? g.B[i] + g.w : 1;
    g.nb[i] = (g.n[i] + g.B[i] - 1) / g.B[i];
    int sb = sbd[g.d][i];
    while (sb > 1 && sb / 2 >= g.nb[i]) sb /= 2;  // no wider than the grid needs
    g.sb[i] = sb;
    g.lsb[i] = 0;
    while ((1 << g.lsb[i]) < sb) ++g.lsb[i];
    g.ns[i] = (g.nb[i] + sb - 1) / sb;
    nbins *= g.ns[i] * sb;
    ntile *= g.T[i];
  }
  g.nbins = nbins;
  g.ntile = ntile;
  g.qs0 = g.qt1 = g.qtile = 0;
  if (g.d == 3 && (g.w & 1) == 0) {
    int s0 = g.T[0] + 1;
    while ((s0 & 15) != 8) ++s0;
    int t1 = g.T[1];
    while ((t1 & 3) != (g.w & 3)) ++t1;
    g.qs0 = s0;
    g.qt1 = t1;
    g.qtile = s0 * t1 * g.T[2];
  }
}

namespace {

int grid_for(int64_t work, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t setpts_t(const Geom& g, const FoldConst& fc, int M, const void* x, const void* y,
                     const void* z, int chk, int* bin_count, int* bin_start, int* sub_first,
                     int* cursor, void* rec, int* sub_bin, int* sub_pt0, int* sub_cnt, int* nsub,
                     int* nsparse, int* err, cudaStream_t st, cudaEvent_t* ev, const BatchTable& bt,
                     int nbins, const Replicas& rp) {
  const T* xp = (const T*)x;
  const T* yp = g.d > 1 ? (const T*)y : xp;
  const T* zp = g.d > 2 ? (const T*)z : xp;
  const int nrep = rp.nrep > 1 ? rp.nrep : 1;
  int* rep_count = nrep > 1 ? rp.count : bin_count;
  int* rep_cursor = nrep > 1 ? rp.cursor : cursor;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], st);
  if ((e = cudaMemsetAsync(rep_count, 0, sizeof(int) * (size_t)nbins * nrep, st)) != cudaSuccess) return e;
  if (M > 0) {
    k_fold_count<T><<<grid_for(M, 256), 256, 0, st>>>(M, xp, yp, zp, g, fc, chk, rep_count, nrep, nbins, err, bt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (nrep > 1) {
    k_rep_sum<<<grid_for(nbins, 256), 256, 0, st>>>(nbins, nrep, rep_count, bin_count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[1], st);
  const int smax = g.sparse_max < g.maxsub ? g.sparse_max : g.maxsub - 1;
  k_scan<<<1, SCAN_THREADS, 0, st>>>(nbins, g.maxsub, smax, bin_count, bin_start, cursor, sub_first, nsub, nsparse);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_sublist<<<grid_for(nbins, 256), 256, 0, st>>>(nbins, g.maxsub, smax, bin_count, bin_start, sub_first, nsub,
                                                   nsparse, sub_bin, sub_pt0, sub_cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], st);
  // sub_first is free once k_sublist has run: it holds the crowded-bin mask
  unsigned* crowd = reinterpret_cast<unsigned*>(sub_first);
  const size_t mask_bytes = sizeof(unsigned) * (size_t)((nbins + 31) / 32);
  const bool mask_smem = nrep > 1 && mask_bytes <= 32 * 1024;
  if (nrep > 1) {
    if ((e = cudaMemsetAsync(crowd, 0, mask_bytes, st)) != cudaSuccess) return e;
    k_rep_cursor<<<grid_for(nbins, 256), 256, 0, st>>>(nbins, nrep, rep_count, bin_count, bin_start, rep_cursor,
                                                        crowd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (M > 0) {
    k_scatter<T><<<grid_for(M, 256), 256, mask_smem ? mask_bytes : 0, st>>>(
        M, xp, yp, zp, g, fc, rep_cursor, nrep, nbins, crowd, mask_smem ? 1 : 0, (typename Traits<T>::Rec*)rec, bt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[3], st);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_setpts(bool dbl, const Geom& g, const FoldConst& fc, int64_t M, const void* x,
                          const void* y, const void* z, int chkbnds, int* bin_count, int* bin_start,
                          int* sub_first, int* cursor, void* rec, int* sub_bin,
                          int* sub_pt0, int* sub_cnt, int* nsub, int* nsparse, int* err, cudaStream_t st,
                          cudaEvent_t* ev, const BatchTable& bt, int nbins, const Replicas& rp) {
  if (nbins <= 0) nbins = g.nbins;
  if (dbl)
    return setpts_t<double>(g, fc, (int)M, x, y, z, chkbnds, bin_count, bin_start, sub_first, cursor,
                            rec, sub_bin, sub_pt0, sub_cnt, nsub, nsparse, err, st, ev, bt, nbins, rp);
  return setpts_t<float>(g, fc, (int)M, x, y, z, chkbnds, bin_count, bin_start, sub_first, cursor,
                         rec, sub_bin, sub_pt0, sub_cnt, nsub, nsparse, err, st, ev, bt, nbins, rp);
}

}  // namespace nufft
