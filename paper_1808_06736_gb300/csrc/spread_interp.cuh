// Spreading (type 1, Eq. (bl)) and interpolation (type 2, Eq. (interp)) with
// the ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) (Eq. (ES)), one thread
// block per subproblem (a bin, or a chunk of a crowded bin; cf. Sec. 5.2).
//
// Per subproblem a block
//   1. stages the subproblem's point records in shared memory,
//   2. orders them so that the 16 lanes of each half-warp hold points whose
//      stencil corners sit in 16 different shared-memory bank groups
//      ("residue" = tile index of the corner mod 16): points are bucketed by
//      residue and dealt out round-robin over the buckets, so every access of
//      the w^d loop is conflict-free while all buckets still hold points,
//   3. spreads into / gathers from a shared-memory tile that covers the bin
//      plus a halo of floor(w/2) cells below and ceil(w/2) above, so the hot
//      loop never wraps indices (the paper pads its cuboids by w/2 for the
//      same reason, Sec. 5.2),
//   4. (spread) adds the tile into the fine grid with periodic wrapping,
//      (interp) writes each result to the caller's array.
//
// Spreading accumulates in shared memory in fixed point: every contribution
// c_j psi is scaled by K / max_j |c_j| (K <= 2^22 for float, 2^51 for double,
// and K * cnt < 2^31 resp. 2^63 so no cell can overflow), rounded to an
// integer with one FMA against 1.5 * 2^23 (resp. 2^52) and added with an
// integer atomic.  Integer shared-memory atomics are several times faster
// than float ones on this GPU, the rounding error (<= max|c| 2^-23 per
// contribution) is below that of float accumulation of the same sums, and
// the tile result does not depend on the order of the atomics.
#pragma once

#include <cstring>
#include <type_traits>

#include "df.cuh"
#include "nufft_internal.cuh"

namespace nufft {

template <typename T>
struct Fixed;
template <>
struct Fixed<float> {
  using I = int;
  static constexpr double KMAX = 4194304.0;         // 2^22
  static constexpr double IMAX = 2147483647.0;      // 2^31 - 1
  __device__ static __forceinline__ int quant(float v) {  // v in [-2^22, 2^22]
    return __float_as_int(fmaf(v, 1.0f, 12582912.0f)) - 0x4B400000;
  }
  __device__ static __forceinline__ float quant_fma(float a, float b) {
    return fmaf(a, b, 12582912.0f);
  }
  __device__ static __forceinline__ int bits(float r) { return __float_as_int(r) - 0x4B400000; }
  __device__ static __forceinline__ void add(int* p, int v) { atomicAdd(p, v); }
};
template <>
struct Fixed<double> {
  using I = long long;
  static constexpr double KMAX = 2251799813685248.0;  // 2^51
  static constexpr double IMAX = 9.2233720368547e18;  // just below 2^63
  __device__ static __forceinline__ double quant_fma(double a, double b) {
    return fma(a, b, 6755399441055744.0);  // 1.5 * 2^52
  }
  __device__ static __forceinline__ long long bits(double r) {
    return __double_as_longlong(r) - 0x4338000000000000LL;
  }
  __device__ static __forceinline__ void add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
  }
};

// ES kernel value.  Float: kpar = beta log2(e), one exp2.  Double: kpar = beta.
__device__ __forceinline__ float es_eval(float z, float kpar) {
  return exp2f(kpar * (sqrtf(fmaxf(1.0f - z * z, 0.0f)) - 1.0f));
}
__device__ __forceinline__ double es_eval(double z, double kpar) {
  return exp(kpar * (sqrt(fmax(1.0 - z * z, 0.0)) - 1.0));
}

// The stencil of a coordinate u = cell + f starts at ceil(u - w/2), i.e. at
// cell - floor(w/2) + step with step = [f > 0] (w even) or [f > 1/2] (w odd);
// in the tile (origin = bin origin - floor(w/2)) that is local cell + step.
template <int W, typename T>
__device__ __forceinline__ int stencil_step(T f) {
  return (W & 1) ? (f > T(0.5) ? 1 : 0) : (f > T(0) ? 1 : 0);
}
// kernel argument of node t: z = (t - floor(w/2) + step - f) * 2 / w
template <int W, typename T>
__device__ __forceinline__ T node_z(int t, int step, T f) {
  return (T(t - W / 2 + step) - f) * (T(2) / T(W));
}

// Kernel evaluation of a launch: the ES exponent factor kpar and, with horner
// set, the piecewise polynomial of Sec. 5.3 (w intervals, degree w + 3,
// a[t * NC + m] the coefficient of s^m on interval t).  Kernels take it as a
// __grid_constant__ parameter, so in the unrolled Horner loops each coefficient
// is a constant-bank operand of its FMA.  The formula branch evaluates Eq. (ES)
// only: plans with the smooth variant (Remark in Sec. 7) take their kernel
// values from its piecewise polynomial here (make_keval sets horner), which
// keeps a second formula, and the registers it costs, out of these kernels;
// the double-float interpolation and the gradient kernels evaluate the
// variant's formula (cosh_kernel).
template <typename T, int W>
struct KEval {
  static constexpr int NC = W + 4;
  T kpar;
  int horner;
  int cosh_kernel;  // formula of the smooth variant (Remark in Sec. 7) instead of Eq. (ES)
  T a[W * NC];
};

// The ES kernel for the complex128 kernels, evaluated in double-float (df.cuh: square root by a
// Newton step, exponential by Cody-Waite reduction and a degree-13 Taylor series, ~2^-47
// relative) and returned as a double.  The GB300's FP64 pipe, about 1/64 of FP32, would
// otherwise spend some 40 operations on each kernel value's exp and sqrt, as much FP64 work as
// a point's w^3 fixed-point products take in the complex128 spread.
__device__ __forceinline__ double es_eval_dd(double z, double beta) { return df_to(es_eval_df(z, df_of(beta))); }

// Node t of a coordinate with fraction f and stencil step lies at
// tau = t - floor(w/2) + step - f cells, in the unit interval t of the support
// [-w/2, w/2]; its local variable is s = 2 (tau - t + w/2) - 1.
template <int W, typename T>
__device__ __forceinline__ T horner_s(int step, T f) {
  return T(2) * (T(step) - f) + T((W & 1) ? 0 : -1);
}

// kernel value of one node (t not known at compile time)
template <typename T, int W>
__device__ __forceinline__ T kernel_node(const KEval<T, W>& ke, int t, int step, T f) {
  if (ke.horner) {
    constexpr int NC = KEval<T, W>::NC;
    const T x = horner_s<W>(step, f);
    const T* a = ke.a + t * NC;
    T y = a[NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m) y = fma(y, x, a[m]);
    return y;
  }
  if constexpr (sizeof(T) == 8)  // the ES formula in double-float on the FP32 pipe (see es_eval_dd)
    return es_eval_dd(node_z<W>(t, step, f), ke.kpar);
  else
    return es_eval(node_z<W>(t, step, f), ke.kpar);
}

// kernel values of all W nodes of a coordinate
template <typename T, int W>
__device__ __forceinline__ void kernel_row(const KEval<T, W>& ke, int step, T f, T* k) {
  if (ke.horner) {
    constexpr int NC = KEval<T, W>::NC;
    const T x = horner_s<W>(step, f);
#pragma unroll
    for (int t = 0; t < W; ++t) k[t] = ke.a[t * NC + NC - 1];
#pragma unroll
    for (int m = NC - 2; m >= 0; --m)
#pragma unroll
      for (int t = 0; t < W; ++t) k[t] = fma(k[t], x, ke.a[t * NC + m]);
  } else if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int t = 0; t < W; ++t) k[t] = es_eval_dd(node_z<W>(t, step, f), ke.kpar);
  } else {
#pragma unroll
    for (int t = 0; t < W; ++t) k[t] = es_eval(node_z<W>(t, step, f), ke.kpar);
  }
}

// L2 eviction-priority policies: fine-grid lines that neighbouring tiles will
// touch again are kept (evict_last); strengths gathered once per point and
// results scattered once are let go first (evict_first).
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// gather of one strength, read once
__device__ __forceinline__ float2 load_once(const float2* p) {
  float2 v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p), "l"(policy_evict_first()));
  return v;
}
__device__ __forceinline__ double2 load_once(const double2* p) { return *p; }
// scatter of one result, written once
__device__ __forceinline__ void store_once(float2* p, float2 v) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
               "l"(policy_evict_first())
               : "memory");
}
__device__ __forceinline__ void store_once(double2* p, double2 v) { *p = v; }

__device__ __forceinline__ void red_add(float2* p, float a, float b) {
  asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(a), "f"(b),
               "l"(policy_evict_last())
               : "memory");
}
__device__ __forceinline__ void red_add(double2* p, double a, double b) {
  atomicAdd(&p->x, a);
  atomicAdd(&p->y, b);
}

// Asynchronous global -> shared copies of one grid element (Ampere-style
// cp.async; 8-byte copies go through L1, 16-byte ones bypass it).
__device__ __forceinline__ void cp_async_elem(float2* dst, const float2* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* dst, const double2* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrap_idx(int x, int n) {
  if ((unsigned)x >= (unsigned)n) {
    x %= n;
    if (x < 0) x += n;
  }
  return x;
}

// Points are dealt to lanes by the bank group of their stencil corner.
// Interpolation reads 8-byte (float2) tile entries: 16 groups of 8 bytes
// cover the 32 four-byte banks and a half-warp is served in one pass when its
// 16 lanes touch 16 different groups (NRES = 16).  Spreading issues 4-byte
// integer atomics on separate re / im planes: a warp is served in one pass
// when its 32 lanes touch 32 different banks (NRES = 32).
constexpr int NRES_INTERP = 16;
constexpr int NRES_SPREAD = 32;

// Shared-memory layout common to both kernels (after the tile).
// The points' records stay in global memory (read again, from L2, when a
// point is processed); shared memory keeps only the ordering state, so that
// more thread blocks fit on an SM.
template <typename T, int D>
// The spread's gapless order uses res, rank and the first maxsub entries of order
// only, and its shared memory holds just those (3 maxsub); the interpolation's
// aligned order needs all of it (5 maxsub).
struct Stage {
  unsigned short* res;     // [maxsub] bank group of the stencil corner
  unsigned short* rank;    // [maxsub] rank within its group
  unsigned short* order;   // [2 maxsub] processing order by slot (0xFFFF: empty slot)
  unsigned short* rstart;  // [maxsub] first slot of each round
};

template <typename T, int D>
__host__ __device__ inline size_t stage_bytes(int maxsub, bool aligned = true) {
  return (size_t)maxsub * (aligned ? 5 : 3) * sizeof(unsigned short);
}

template <typename T, int D>
__device__ __forceinline__ Stage<T, D> carve_stage(unsigned char* p, int maxsub) {
  Stage<T, D> s;
  s.res = reinterpret_cast<unsigned short*>(p);
  s.rank = s.res + maxsub;
  s.order = s.rank + maxsub;
  s.rstart = s.order + 2 * maxsub;
  return s;
}
constexpr unsigned short kEmptySlot = 0xFFFF;

// Decode a bin index into its per-dimension tile origin (bin origin - floor(w/2)).
__device__ __forceinline__ void tile_origin(const Geom& g, int bin, int* org) {
  int b[3];
  bin_coords(g, bin, b);
  org[0] = b[0] * g.B[0] - g.half;
  org[1] = b[1] * g.B[1] - g.half;
  org[2] = b[2] * g.B[2] - g.half;
}

// Store a record in the stage and count it in its bank group.  hist[] must
// be zero on entry.
template <typename T, int D, int W, int NRES>
__device__ __forceinline__ void stage_point(const Geom& g, const typename Traits<T>::Rec& r, int q,
                                            Stage<T, D>& st, int* hist) {
  int base = 0, stride = 1;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    T v = r.v[d];
    int il = min((int)v, g.B[d] - 1);
    base += (il + stencil_step<W>(v - T(il))) * stride;
    stride *= g.T[d];
  }
  int rr = base & (NRES - 1);
  st.res[q] = (unsigned short)rr;
  st.rank[q] = (unsigned short)atomicAdd(&hist[rr], 1);
}

// Processing order over the bank groups.  Round r takes the r-th point of every group
// that has more than r points, groups in increasing order, so the points of one round
// lie in different bank groups.
//  * ALIGNED = false: rounds follow each other without gaps; the point of group b with
//    rank r lands at sum_g min(size_g, r) + #{g < b : size_g > r}.  Returns cnt.
//  * ALIGNED = true: rounds are packed whole into consecutive groups of NRES slots (a
//    half-warp for the interpolation's 8-byte loads): a round that does not fit in what
//    is left of the current slot group starts the next one, and the slots it leaves stay
//    empty (kEmptySlot).  A slot group then never holds two points of one bank group from
//    one round, which gapless packing does at the tail of uneven groups.  Each gap is
//    smaller than the round that did not fit, so there are fewer than 2 cnt slots.
//    Returns the number of slots.
// The complex64 interpolation takes the aligned order (1.6-2.8 % faster on the 3D benchmark
// workload); the spread (11 % slower aligned), the double-float interpolation (7 % slower)
// and the gradient kernels keep the gapless one.
// Synchronises the block.
template <typename T, int D, int NRES, bool ALIGNED>
__device__ __forceinline__ int bucket_order(int cnt, Stage<T, D>& st, const int* hist, int* s_nslots) {
  __syncthreads();
  int sz[NRES];
  int maxsz = 0;
#pragma unroll
  for (int b = 0; b < NRES; ++b) {
    sz[b] = hist[b];
    maxsz = max(maxsz, sz[b]);
  }
  if constexpr (!ALIGNED) {
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int r = st.rank[q], b = st.res[q];
      int pos = 0;
#pragma unroll
      for (int g = 0; g < NRES; ++g) pos += min(sz[g], r) + ((g < b && sz[g] > r) ? 1 : 0);
      st.order[pos] = (unsigned short)q;
    }
    __syncthreads();
    return cnt;
  }
  // rounds below the smallest group's size hold a point of every group: each fills a slot group
  // exactly (slot NRES r), so only the rounds from minsz on are packed one after another
  int minsz = sz[0];
#pragma unroll
  for (int b = 1; b < NRES; ++b) minsz = min(minsz, sz[b]);
  for (int r = threadIdx.x; r < maxsz; r += blockDim.x) {  // round sizes (maxsz <= cnt)
    int k = 0;
#pragma unroll
    for (int b = 0; b < NRES; ++b) k += sz[b] > r ? 1 : 0;
    st.rstart[r] = (unsigned short)(r < minsz ? NRES * r : k);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int slot = NRES * minsz, fill = 0;  // fill = slot mod NRES
    for (int r = minsz; r < maxsz; ++r) {
      const int k = st.rstart[r];
      if (fill + k > NRES) {
        slot += NRES - fill;
        fill = 0;
      }
      st.rstart[r] = (unsigned short)slot;
      slot += k;
      fill += k;
      if (fill == NRES) fill = 0;
    }
    *s_nslots = slot;
  }
  __syncthreads();
  const int nslots = *s_nslots;
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) st.order[i] = kEmptySlot;
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int r = st.rank[q], b = st.res[q];
    int pos = st.rstart[r];
#pragma unroll
    for (int g = 0; g < NRES; ++g) pos += (g < b && sz[g] > r) ? 1 : 0;
    st.order[pos] = (unsigned short)q;
  }
  __syncthreads();
  return nslots;
}

// Per-point kernel values along one dimension.
template <typename T, int W>
__device__ __forceinline__ void point_weights(T v, int B, const KEval<T, W>& ke, int& ts, T* k) {
  int il = min((int)v, B - 1);
  T f = v - T(il);
  int s = stencil_step<W>(f);
  ts = il + s;
  kernel_row<T, W>(ke, s, f, k);
}

// Add a fixed-point tile (scaled by inv) into the fine grid with periodic
// wrapping.  Warps take tile rows; lanes walk along x.  For complex64 rows
// that do not wrap on a grid with even n_1, neighbouring cells go out as one
// 16-byte vector reduction (red.global.add.v4.f32) from an even grid index.
__device__ __forceinline__ void red_add2(float2* p, float a0, float b0, float a1, float b1) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a0), "f"(b0),
               "f"(a1), "f"(b1), "l"(policy_evict_last())
               : "memory");
}

template <typename T>
__device__ __forceinline__ void flush_tile(const Geom& g, const int* org, const typename Fixed<T>::I* tre,
                                           const typename Fixed<T>::I* tim, T inv,
                                           typename Traits<T>::C* grid) {
  using C = typename Traits<T>::C;
  using I = typename Fixed<T>::I;
  const int T0 = g.T[0];
  const int nrows = g.ntile / T0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const bool pairs = (sizeof(T) == 4) && ((g.n[0] & 1) == 0) && org[0] >= 0 && org[0] + T0 <= g.n[0];
  for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
    const int t1 = row % g.T[1], t2 = row / g.T[1];
    const long long gy = wrap_idx(org[1] + t1, g.n[1]);
    const long long gz = wrap_idx(org[2] + t2, g.n[2]);
    C* grow = grid + (gz * g.n[1] + gy) * (long long)g.n[0];
    const I* ar = tre + row * T0;
    const I* ai = tim + row * T0;
    if (pairs) {
      const int first = org[0] & 1;  // a leading single cell when the row starts at an odd index
      const int nslots = first + (T0 - first + 1) / 2;
      for (int sl = lane; sl < nslots; sl += 32) {
        const int t0 = (first && sl == 0) ? 0 : first + 2 * (sl - first);
        const I a0 = ar[t0], b0 = ai[t0];
        if (t0 + 1 < T0 && !(first && sl == 0)) {
          const I a1 = ar[t0 + 1], b1 = ai[t0 + 1];
          if (a0 != 0 || b0 != 0 || a1 != 0 || b1 != 0)
            red_add2(reinterpret_cast<float2*>(grow + org[0] + t0), float(a0) * float(inv), float(b0) * float(inv),
                     float(a1) * float(inv), float(b1) * float(inv));
        } else if (a0 != 0 || b0 != 0) {
          red_add(grow + org[0] + t0, T(a0) * inv, T(b0) * inv);
        }
      }
    } else {
      for (int t0 = lane; t0 < T0; t0 += 32) {
        const I a = ar[t0], b = ai[t0];
        if (a == 0 && b == 0) continue;
        red_add(grow + wrap_idx(org[0] + t0, g.n[0]), T(a) * inv, T(b) * inv);
      }
    }
  }
}

// ----------------------------------------------------------------- spread
// Fixed-point scales of one complex64 subproblem.  A single scale set by the largest
// strength maxabs rounds every contribution to steps of maxabs / K; when most strengths of
// the subproblem lie below maxabs 2^-10 (one large strength among many small ones), those
// small ones would lose their share to that rounding.  Such subproblems are spread in two
// passes: the strengths above maxabs 2^-10 at K / maxabs, the others at K / (their own
// maximum), each pass flushed on its own.  Counted once per subproblem, after staging;
// s_nsmall and s_msmall must be zero on entry.  Returns the number of passes (1 or 2) and
// the threshold and the small strengths' maximum.
constexpr float kSmallRatio = 1.0f / 1024.0f;
__device__ __forceinline__ int plan_passes(const float2* sc, int cnt, float maxabs, int* s_nsmall, int* s_msmall,
                                           float* thr, float* smax) {
  *thr = maxabs * kSmallRatio;
  int n = 0;
  float m = 0.f;
  if (maxabs > 0.f && maxabs < INFINITY) {
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const float a = fmaxf(fabsf(sc[q].x), fabsf(sc[q].y));
      if (a <= *thr) {
        ++n;
        m = fmaxf(m, a);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0 && n > 0) {
    atomicAdd(s_nsmall, n);
    atomicMax(s_msmall, __float_as_int(m));
  }
  __syncthreads();
  *smax = __int_as_float(*s_msmall);
  return (2 * *s_nsmall > cnt && *smax > 0.f) ? 2 : 1;
}
// scale K / top and its inverse for a pass over strengths of largest magnitude top
__device__ __forceinline__ void pass_scale(double K, float top, float* scale, float* inv) {
  *scale = 0.f;
  *inv = 0.f;
  if (top > 0.f && top < INFINITY) {
    *scale = float(K / (double)top);
    *inv = float((double)top / K);
  } else if (!(top == 0.f)) {
    *inv = NAN;  // non-finite strengths: make the whole tile NaN
  }
}

// float kernels are held to 64 registers so four 256-thread blocks fit an SM
template <typename T>
struct MinBlocks {
  static constexpr int value = sizeof(T) == 4 ? 4 : 2;
};

// Thread 0 takes the next subproblem and puts its geometry in shared memory:
// for a batch, the subproblem's transform, its grid offset and its bin id
// within that transform.  Returns false when the work list is exhausted.
__device__ __forceinline__ void resolve_subproblem(const Geom& g, const Sorted& s, const BatchTable& bt, int sub,
                                                   int* s_sub, int* s_bin, long long* s_goff, Geom* s_geo);
__device__ __forceinline__ void next_subproblem(const Geom& g, const Sorted& s, const BatchTable& bt, int* work,
                                                int* s_sub, int* s_bin, long long* s_goff, Geom* s_geo) {
  resolve_subproblem(g, s, bt, atomicAdd(work, 1), s_sub, s_bin, s_goff, s_geo);
}
// The same for a subproblem id taken from the work counter earlier (a block claims its next id
// while it works on the current one, so the atomic's latency is hidden).
__device__ __forceinline__ void resolve_subproblem(const Geom& g, const Sorted& s, const BatchTable& bt, int sub,
                                                   int* s_sub, int* s_bin, long long* s_goff, Geom* s_geo) {
  *s_sub = sub;
  if (sub < *s.nsub) {
    int bin = s.sub_bin[sub];
    *s_geo = g;
    long long goff = 0;
    if (bt.B > 0) {
      const int t = batch_find(bt.boff, bt.B, bin);
      const BatchGeom tg = bt.bg[t];
      batch_apply(*s_geo, tg);
      bin -= tg.boff;
      goff = tg.goff;
    }
    *s_bin = bin;
    *s_goff = goff;
  }
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) k_spread(Geom g, const __grid_constant__ KEval<T, W> ke, Sorted s,
                                                const typename Traits<T>::C* __restrict__ c,
                                                typename Traits<T>::C* __restrict__ grid,
                                                int* __restrict__ work, BatchTable bt) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  using F = Fixed<T>;
  using I = typename F::I;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[NRES_SPREAD];
  __shared__ int s_sub, s_bin, s_nslots, s_nsmall, s_msmall;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;
  __shared__ I s_maxbits;

  const int ntile = g.ntile, maxsub = g.maxsub;
  I* tre = reinterpret_cast<I*>(smem);
  I* tim = tre + ntile;
  C* sc = reinterpret_cast<C*>(tim + ntile);  // staged strengths
  Stage<T, D> st = carve_stage<T, D>(reinterpret_cast<unsigned char*>(sc + maxsub), maxsub);
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const int T0 = g.T[0], T01 = g.T[0] * g.T[1];

  for (;;) {
    if (threadIdx.x == 0) {
      next_subproblem(g, s, bt, work, &s_sub, &s_bin, &s_goff, &s_geo);
      s_maxbits = 0;
      s_nsmall = 0;
      s_msmall = 0;
    }
    if (threadIdx.x < NRES_SPREAD) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];

    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      tre[t] = 0;
      tim[t] = 0;
    }
    T mloc = T(0);
    // records and strengths in batches of four per thread (independent loads in flight)
    for (int q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
      Rec r[4];
      C cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < cnt) r[u] = rec[p0 + q];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < cnt) cv[u] = load_once(c + r[u].idx);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < cnt) {
          stage_point<T, D, W, NRES_SPREAD>(g, r[u], q, st, hist);
          sc[q] = cv[u];
          mloc = fmax(mloc, fmax(fabs(cv[u].x), fabs(cv[u].y)));
        }
      }
    }
    // non-negative floats order like their bit patterns; NaN (all bits high) wins
    if (!(mloc == mloc)) mloc = T(INFINITY);
    if (sizeof(T) == 4)
      atomicMax(reinterpret_cast<int*>(&s_maxbits), __float_as_int((float)mloc));
    else
      atomicMax(reinterpret_cast<unsigned long long*>(&s_maxbits),
                (unsigned long long)__double_as_longlong((double)mloc));
    const int nslots = bucket_order<T, D, NRES_SPREAD, false>(cnt, st, hist, &s_nslots);

    T maxabs;
    if (sizeof(T) == 4)
      maxabs = (T)__int_as_float((int)s_maxbits);
    else
      maxabs = (T)__longlong_as_double((long long)s_maxbits);
    const double K = fmin(F::KMAX, floor(F::IMAX / (double)cnt) - 1.0);
    // complex64: one or two passes (plan_passes); complex128's 2^51 steps need no split
    float thr = 0.f, smax = 0.f;
    int npass = 1;
    if constexpr (sizeof(T) == 4)
      npass = plan_passes(reinterpret_cast<const float2*>(sc), cnt, (float)maxabs, &s_nsmall, &s_msmall, &thr, &smax);
    for (int pass = 0; pass < npass; ++pass) {
      if (pass == 1) {  // the small strengths, on a zeroed tile
        for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
          tre[t] = 0;
          tim[t] = 0;
        }
        __syncthreads();
      }
      T scale = T(0), inv = T(0);
      const T top = pass == 0 ? maxabs : T(smax);
      if (top > T(0) && top < T(INFINITY)) {
        scale = T(K / (double)top);
        inv = T((double)top / K);
      } else if (!(top == T(0))) {
        inv = T(NAN);  // non-finite strengths: make the whole tile NaN
      }

      // complex128 in 3D: a subproblem of few points (about a hundred per 8x8x8 bin at
      // w = 10) would leave most threads idle through the heavy part, w^3 cells per point, so
      // up to 8 threads share a point, each taking every tpp-th plane of its stencil
      constexpr bool kSplit = sizeof(T) == 8 && D == 3;
      int tpp = 1;
      if constexpr (kSplit) {
        while (tpp < 8 && tpp < W && 2 * tpp * cnt <= (int)blockDim.x) tpp *= 2;
      }
      const int ltpp = kSplit ? __ffs(tpp) - 1 : 0;
      for (int u = threadIdx.x; u < (nslots << ltpp); u += blockDim.x) {
        const int sl = u >> ltpp, part = u & (tpp - 1);
        const int q = st.order[sl];
        if (q == kEmptySlot) continue;
        if (npass == 2 && (fmax(fabs(sc[q].x), fabs(sc[q].y)) > T(thr)) != (pass == 0)) continue;  // not this pass
        const Rec rq = rec[p0 + q];
        T k0[W];
        int ts0, ts1 = 0, ts2 = 0;
        point_weights<T, W>(rq.v[0], g.B[0], ke, ts0, k0);
        T k1[(D > 1) ? W : 1];
        T f2 = T(0);
        int st2 = 0;
        if constexpr (D > 1) point_weights<T, W>(rq.v[1], g.B[1], ke, ts1, k1);
        else k1[0] = T(1);
        if constexpr (D > 2) {
          T v2 = rq.v[2];
          int il2 = min((int)v2, g.B[2] - 1);
          f2 = v2 - T(il2);
          st2 = stencil_step<W>(f2);
          ts2 = il2 + st2;
        }
        const C cv = sc[q];
        const T cr = cv.x * scale, ci = cv.y * scale;
        const int base = ts0 + T0 * ts1 + T01 * ts2;
        constexpr int W1 = (D > 1) ? W : 1;
        constexpr int W2 = (D > 2) ? W : 1;
#pragma unroll 1
        for (int l2 = part; l2 < W2; l2 += tpp) {
          T k2 = T(1);
          if constexpr (D > 2) k2 = kernel_node<T, W>(ke, l2, st2, f2);
          const T cr2 = cr * k2, ci2 = ci * k2;
#pragma unroll
          for (int l1 = 0; l1 < W1; ++l1) {
            const T cr1 = cr2 * k1[l1], ci1 = ci2 * k1[l1];
            I* pr = tre + base + l1 * T0 + l2 * T01;
            I* pi = tim + base + l1 * T0 + l2 * T01;
#pragma unroll
            for (int l0 = 0; l0 < W; ++l0) {
              F::add(pr + l0, F::bits(F::quant_fma(cr1, k0[l0])));
              F::add(pi + l0, F::bits(F::quant_fma(ci1, k0[l0])));
            }
          }
        }
      }
      __syncthreads();

      // add the tile into the fine grid, wrapping periodically; rows of the
      // tile are spread over the warps, a warp's lanes walk along x
      int org[3];
      tile_origin(s_geo, bin, org);
      flush_tile<T>(s_geo, org, tre, tim, inv, grid + s_goff);
      __syncthreads();
    }  // pass
  }
}

// ----------------------------------------------------------------- interp
template <typename T, int D, int W>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) k_interp(Geom g, const __grid_constant__ KEval<T, W> ke, Sorted s,
                                                const typename Traits<T>::C* __restrict__ grid,
                                                typename Traits<T>::C* __restrict__ c,
                                                int* __restrict__ work, BatchTable bt) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[NRES_INTERP];
  __shared__ int s_sub, s_bin, s_nslots;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;

  const int ntile = g.ntile, maxsub = g.maxsub;
  C* tile = reinterpret_cast<C*>(smem);
  Stage<T, D> st = carve_stage<T, D>(reinterpret_cast<unsigned char*>(tile + ntile), maxsub);
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const int T0 = g.T[0], T01 = g.T[0] * g.T[1];

  for (;;) {
    if (threadIdx.x == 0) next_subproblem(g, s, bt, work, &s_sub, &s_bin, &s_goff, &s_geo);
    if (threadIdx.x < NRES_INTERP) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];

    // fetch the tile (bin + halo) from the fine grid, wrapping periodically
    int org[3];
    tile_origin(s_geo, bin, org);
    const int nrows = ntile / T0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int n0 = s_geo.n[0], n1 = s_geo.n[1], n2 = s_geo.n[2];
    const C* gridt = grid + s_goff;
    for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
      const int t1 = row % g.T[1], t2 = row / g.T[1];
      const long long gy = wrap_idx(org[1] + t1, n1);
      const long long gz = wrap_idx(org[2] + t2, n2);
      const C* grow = gridt + (gz * n1 + gy) * (long long)n0;
      for (int t0 = lane; t0 < T0; t0 += 32) cp_async_elem(tile + row * T0 + t0, grow + wrap_idx(org[0] + t0, n0));
    }
    cp_async_commit();
    // records in batches of four per thread while the tile copies are in flight
    for (int q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
      Rec r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < cnt) r[u] = rec[p0 + q];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < cnt) stage_point<T, D, W, NRES_INTERP>(g, r[u], q, st, hist);
      }
    }
    cp_async_wait_all();
    const int nslots = bucket_order<T, D, NRES_INTERP, true>(cnt, st, hist, &s_nslots);

    for (int sl = threadIdx.x; sl < nslots; sl += blockDim.x) {
      const int q = st.order[sl];
      if (q == kEmptySlot) continue;
      const Rec rq = rec[p0 + q];
      T k0[W];
      int ts0, ts1 = 0, ts2 = 0;
      point_weights<T, W>(rq.v[0], g.B[0], ke, ts0, k0);
      T k1[(D > 1) ? W : 1];
      T f2 = T(0);
      int st2 = 0;
      if constexpr (D > 1) point_weights<T, W>(rq.v[1], g.B[1], ke, ts1, k1);
      else k1[0] = T(1);
      if constexpr (D > 2) {
        T v2 = rq.v[2];
        int il2 = min((int)v2, g.B[2] - 1);
        f2 = v2 - T(il2);
        st2 = stencil_step<W>(f2);
        ts2 = il2 + st2;
      }
      const int base = ts0 + T0 * ts1 + T01 * ts2;
      constexpr int W1 = (D > 1) ? W : 1;
      constexpr int W2 = (D > 2) ? W : 1;
      T ar = T(0), ai = T(0);
#pragma unroll 1
      for (int l2 = 0; l2 < W2; ++l2) {
        T br = T(0), bi = T(0);
#pragma unroll
        for (int l1 = 0; l1 < W1; ++l1) {
          const C* rowp = tile + base + l1 * T0 + l2 * T01;
          T sr = T(0), si = T(0);
#pragma unroll
          for (int l0 = 0; l0 < W; ++l0) {
            const C gv = rowp[l0];
            sr = fma(gv.x, k0[l0], sr);
            si = fma(gv.y, k0[l0], si);
          }
          br = fma(sr, k1[l1], br);
          bi = fma(si, k1[l1], bi);
        }
        T k2 = T(1);
        if constexpr (D > 2) k2 = kernel_node<T, W>(ke, l2, st2, f2);
        ar = fma(br, k2, ar);
        ai = fma(bi, k2, ai);
      }
      C out;
      out.x = ar;
      out.y = ai;
      store_once(c + rq.idx, out);
    }
    __syncthreads();
  }
}

// ------------------------------------------------ interp, complex128
// The GB300 runs FP64 at about 1/64 of its FP32 rate, so the complex128
// interpolation runs in double-float arithmetic on the FP32 pipe (df.cuh):
// the kernel values (square root, exponential) and the w^d-term tensor
// contraction; every tile value and weight is a pair (hi, lo) of floats with
// hi + lo equal to the double to ~2^-48.  That is accurate to ~1e-14
// relative, far below the eps >= 1e-11 the complex128 path serves.  The tile
// is scaled by a power of two so its largest value is about 1 (float range;
// the scale is undone exactly on output).
// kernel values along one dimension in double-float (see point_weights)
template <int W>
__device__ __forceinline__ void point_weights_df(double v, int B, DF beta, int cosh_kernel, int& ts, DF* k) {
  const int il = min((int)v, B - 1);
  const double f = v - double(il);
  const int s = stencil_step<W>(f);
  ts = il + s;
  const DF fd = df_of(f);
  const DF scale = DF{2.0f / W, __double2float_rn(2.0 / W - (double)(2.0f / W))};
#pragma unroll
  for (int t = 0; t < W; ++t) {
    // z = (t - floor(w/2) + step - f) 2 / w in double-float
    const DF z = df_mul(df_add(DF{(float)(t - W / 2 + s), 0.0f}, DF{-fd.hi, -fd.lo}), scale);
    k[t] = es_eval_df_z(z, beta, cosh_kernel);
  }
}

__device__ __forceinline__ double2 out_of(DF ar, DF ai, int sh) {
  return make_double2(ldexp((double)ar.hi + (double)ar.lo, sh), ldexp((double)ai.hi + (double)ai.lo, sh));
}
// blocks of 512 threads: a tile of a 16x8x8 bin at w = 10 (135 KB) leaves room for one block
// per SM, and 512 threads at up to 128 registers fill the register file
constexpr int kInterpDfThreads = 512;
// dynamic shared memory above which at most one block fits an SM (228 KB, 1 KB per block reserved)
constexpr size_t kOneBlockSmem = 112 * 1024;
template <int D, int W, bool COSH>
__global__ void __launch_bounds__(kInterpDfThreads, 1) k_interp_df(Geom g, const __grid_constant__ KEval<double, W> ke, Sorted s, const double2* __restrict__ grid,
                                                      double2* __restrict__ c, int* __restrict__ work, BatchTable bt) {
  using Rec = typename Traits<double>::Rec;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[NRES_INTERP];
  __shared__ int s_sub, s_bin, s_maxexp, s_nslots;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;

  const int ntile = g.ntile, maxsub = g.maxsub;
  double2* tile = reinterpret_cast<double2*>(smem);  // then, in place, float4 (re hi, re lo, im hi, im lo)
  float4* tdf = reinterpret_cast<float4*>(smem);
  Stage<double, D> st = carve_stage<double, D>(reinterpret_cast<unsigned char*>(tile + ntile), maxsub);
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const int T0 = g.T[0], T01 = g.T[0] * g.T[1];
  const DF bdf = df_of(ke.kpar);  // beta (the double-float path evaluates the ES formula)

  for (;;) {
    if (threadIdx.x == 0) {
      next_subproblem(g, s, bt, work, &s_sub, &s_bin, &s_goff, &s_geo);
      s_maxexp = -1100;
    }
    if (threadIdx.x < NRES_INTERP) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];

    int org[3];
    tile_origin(s_geo, bin, org);
    const int nrows = ntile / T0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int n0 = s_geo.n[0], n1 = s_geo.n[1], n2 = s_geo.n[2];
    const double2* gridt = grid + s_goff;
    for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
      const int t1 = row % g.T[1], t2 = row / g.T[1];
      const long long gy = wrap_idx(org[1] + t1, n1);
      const long long gz = wrap_idx(org[2] + t2, n2);
      const double2* grow = gridt + (gz * n1 + gy) * (long long)n0;
      for (int t0 = lane; t0 < T0; t0 += 32) cp_async_elem(tile + row * T0 + t0, grow + wrap_idx(org[0] + t0, n0));
    }
    cp_async_commit();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) stage_point<double, D, W, NRES_INTERP>(g, rec[p0 + q], q, st, hist);
    cp_async_wait_all();
    __syncthreads();
    // power-of-two scale: the largest |value| of the tile to [0.5, 1); exponents read from
    // the bit patterns (integer pipe), as is the split below, so the GB300's slow FP64
    // pipe does no per-cell work
    int me = -1100;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const double2 v = tile[t];
      me = max(me, max(df_bexp(v.x), df_bexp(v.y)));
    }
    atomicMax(&s_maxexp, me);
    __syncthreads();
    const int sh = s_maxexp > -1000 ? s_maxexp : 0;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const double2 v = tile[t];
      const DF re = df_split_scaled(v.x, sh), im = df_split_scaled(v.y, sh);
      tdf[t] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    // gapless order: this kernel is bound by its double-float arithmetic, and the aligned
    // order's extra (partly idle) warps cost more than its fewer bank conflicts save
    const int nslots = bucket_order<double, D, NRES_INTERP, false>(cnt, st, hist, &s_nslots);  // synchronises

    // a subproblem of fewer points than threads leaves most threads idle through the w^3 cells
    // of a point: up to 8 threads share a point (3D), each summing every tpp-th plane of its
    // stencil; the partial sums are added with shuffles (warp-uniform trip count)
    int tpp = 1;
    if constexpr (D == 3) {
      while (tpp < 8 && tpp < W && 2 * tpp * nslots <= (int)blockDim.x) tpp *= 2;
    }
    const int ltpp = __ffs(tpp) - 1;
    const int total = nslots << ltpp;
    for (int u0 = threadIdx.x & ~31; u0 < total; u0 += blockDim.x) {
      const int u = u0 + (threadIdx.x & 31);
      const int part = u & (tpp - 1);
      const int q = u < total ? (int)st.order[u >> ltpp] : (int)kEmptySlot;
      const bool act = q != kEmptySlot;
      Rec rq;
      rq.v[0] = rq.v[1] = rq.v[2] = 0.0;
      rq.idx = 0;
      if (act) rq = rec[p0 + q];
      DF k0[W];
      int ts0, ts1 = 0, ts2 = 0;
      point_weights_df<W>(rq.v[0], g.B[0], bdf, COSH, ts0, k0);
      DF k1[(D > 1) ? W : 1];
      double f2 = 0.0;
      int st2 = 0;
      if constexpr (D > 1) {
        point_weights_df<W>(rq.v[1], g.B[1], bdf, COSH, ts1, k1);
      } else {
        k1[0] = DF{1.0f, 0.0f};
      }
      if constexpr (D > 2) {
        const double v2 = rq.v[2];
        const int il2 = min((int)v2, g.B[2] - 1);
        f2 = v2 - double(il2);
        st2 = stencil_step<W>(f2);
        ts2 = il2 + st2;
      }
      const int base = ts0 + T0 * ts1 + T01 * ts2;
      constexpr int W1 = (D > 1) ? W : 1;
      constexpr int W2 = (D > 2) ? W : 1;
      DF ar = {0.f, 0.f}, ai = {0.f, 0.f};
#pragma unroll 1
      for (int l2 = act ? part : W2; l2 < W2; l2 += tpp) {
        DF br = {0.f, 0.f}, bi = {0.f, 0.f};
        // rows one at a time (the row's y value picked from registers): the fully unrolled w^2
        // rows of w cells overflowed the instruction cache (ncu: 1.2 no-instruction stalls per issue)
#pragma unroll 1
        for (int l1 = 0; l1 < W1; ++l1) {
          const DF k1v = df_pick<(D > 1) ? W : 1>(k1, l1);
          const float4* rowp = tdf + base + l1 * T0 + l2 * T01;
          // even and odd nodes in separate accumulators: four independent
          // dependency chains per point instead of two
          DF sr0 = {0.f, 0.f}, si0 = {0.f, 0.f}, sr1 = {0.f, 0.f}, si1 = {0.f, 0.f};
#pragma unroll
          for (int l0 = 0; l0 < W; l0 += 2) {
            const float4 gv = rowp[l0];
            df_mac(sr0, DF{gv.x, gv.y}, k0[l0]);
            df_mac(si0, DF{gv.z, gv.w}, k0[l0]);
            if (l0 + 1 < W) {
              const float4 gu = rowp[l0 + 1];
              df_mac(sr1, DF{gu.x, gu.y}, k0[l0 + 1]);
              df_mac(si1, DF{gu.z, gu.w}, k0[l0 + 1]);
            }
          }
          const DF sr = df_add(df_norm(sr0), df_norm(sr1)), si = df_add(df_norm(si0), df_norm(si1));
          df_mac(br, sr, k1v);
          df_mac(bi, si, k1v);
        }
        DF k2 = {1.0f, 0.0f};
        if constexpr (D > 2) k2 = es_eval_df(node_z<W>(l2, st2, f2), bdf, COSH);
        df_mac(ar, df_norm(br), k2);
        df_mac(ai, df_norm(bi), k2);
      }
      for (int o = 1; o < tpp; o <<= 1) {  // tpp is block-uniform: every lane shuffles
        const DF pr = {__shfl_xor_sync(0xffffffffu, ar.hi, o), __shfl_xor_sync(0xffffffffu, ar.lo, o)};
        const DF pi = {__shfl_xor_sync(0xffffffffu, ai.hi, o), __shfl_xor_sync(0xffffffffu, ai.lo, o)};
        ar = df_add(df_norm(ar), df_norm(pr));
        ai = df_add(df_norm(ai), df_norm(pi));
      }
      if (act && part == 0) store_once(c + rq.idx, out_of(ar, ai, sh));
    }
    __syncthreads();
  }
}

// the tiled interpolation kernel for each precision (complex128: one instance per
// kernel formula, so the ES path carries no code for the smooth variant)
template <typename T, int D, int W>
struct InterpKernel {
  static auto get(bool) { return k_interp<T, D, W>; }
};
template <int D, int W>
struct InterpKernel<double, D, W> {
  static auto get(bool cosh) { return cosh ? k_interp_df<D, W, true> : k_interp_df<D, W, false>; }
};

// ------------------------------------------------- sparse subproblems
// Subproblems of at most 32 points (low point density: most bins hold a few
// points or none) skip the shared-memory tile, whose zeroing, flushing or
// loading would cost far more than their w^d contributions per point.  One
// warp takes one such subproblem: lane j holds point j; per pass the warp
// handles PP = max(1, 32 / w^d) points, its lanes computing the per-dimension
// ES weights into a small per-warp buffer, then each lane owns one stencil
// cell of one point (lanes along x first, so a warp's accesses fall in
// contiguous rows of the fine grid) and adds to / gathers from the fine grid
// directly, wrapping periodically.
template <int W, int D>
struct Sparse {
  static constexpr int CP = (D == 1) ? W : (D == 2 ? W * W : W * W * W);  // cells per point
  static constexpr int PP = CP >= 32 ? 1 : 32 / CP;                      // points per pass
  static constexpr int NW = PP * W * D;                                  // weights per pass (<= 48)
  static constexpr int WB = 64;                                          // weight buffer per warp
};

// The subproblem's geometry for a batch: its transform's grid, bin id and offset.
__device__ __forceinline__ void sparse_geometry(const Geom& g, const BatchTable& bt, int& bin, Geom& gg,
                                                long long& goff) {
  gg = g;
  goff = 0;
  if (bt.B > 0) {
    const int t = batch_find(bt.boff, bt.B, bin);
    const BatchGeom tg = bt.bg[t];
    batch_apply(gg, tg);
    bin -= tg.boff;
    goff = tg.goff;
  }
}

// Weights of the points jb .. jb+PP-1 (records held by lanes jb + p) into wb,
// entry p*W*D + d*W + t.  Every lane takes part in the shuffles.
template <typename T, int D, int W>
__device__ __forceinline__ void sparse_weights(const typename Traits<T>::Rec& r, int jb, const Geom& gg,
                                               const KEval<T, W>& ke, T* wb) {
  using S = Sparse<W, D>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int e0 = 0; e0 < S::NW; e0 += 32) {
    const int e = e0 + lane;
    const int p = e / (W * D), dd = (e / W) % D, t = e % W;
    const int src = (jb + p) & 31;
    const T v0 = __shfl_sync(0xffffffffu, r.v[0], src);
    const T v1 = __shfl_sync(0xffffffffu, r.v[1], src);
    const T v2 = __shfl_sync(0xffffffffu, r.v[2], src);
    if (e < S::NW) {
      const T v = dd == 0 ? v0 : (dd == 1 ? v1 : v2);
      const int il = min((int)v, gg.B[dd] - 1);
      const T f = v - T(il);
      wb[e] = kernel_node<T, W>(ke, t, stencil_step<W>(f), f);
    }
  }
  __syncwarp();
}

// Fine-grid index of stencil cell `cell` of the point whose record is v, and
// the cell's weight from wb (point slot p).
template <typename T, int D, int W>
__device__ __forceinline__ long long sparse_cell(const T* v, const int* org, const Geom& gg, const T* wb, int p,
                                                 int cell, T& wt) {
  const int i0 = cell % W, i1 = (cell / W) % W, i2 = cell / (W * W);
  const int ii[3] = {i0, i1, i2};
  long long idx = 0, stride = 1;
  wt = T(1);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int il = min((int)v[d], gg.B[d] - 1);
    const int a = org[d] + il + stencil_step<W>(v[d] - T(il));
    idx += (long long)wrap_idx(a + ii[d], gg.n[d]) * stride;
    stride *= gg.n[d];
    wt *= wb[p * W * D + d * W + ii[d]];
  }
  return idx;
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_spread_sparse(Geom g, const __grid_constant__ KEval<T, W> ke, Sorted s,
                                                       const typename Traits<T>::C* __restrict__ c,
                                                       typename Traits<T>::C* __restrict__ grid, BatchTable bt) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  using S = Sparse<W, D>;
  __shared__ T wbuf[8][S::WB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nt = *s.nsub, nsp = *s.nsparse;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  T* wb = wbuf[wid];
  for (int i = blockIdx.x * 8 + wid; i < nsp; i += gridDim.x * 8) {
    const int sub = nt + i;
    int bin = s.sub_bin[sub];
    const int p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];
    Geom gg;
    long long goff;
    sparse_geometry(g, bt, bin, gg, goff);
    int org[3];
    tile_origin(gg, bin, org);
    Rec r;
    r.v[0] = r.v[1] = r.v[2] = T(0);
    C cv;
    cv.x = cv.y = T(0);
    if (lane < cnt) {
      r = rec[p0 + lane];
      cv = load_once(c + r.idx);
    }
    C* gt = grid + goff;
    for (int jb = 0; jb < cnt; jb += S::PP) {
      sparse_weights<T, D, W>(r, jb, gg, ke, wb);
      if (S::PP > 1) {
        const int p = lane / S::CP, cell = lane - p * S::CP;
        const int src = (jb + p) & 31;
        T v[3];
        v[0] = __shfl_sync(0xffffffffu, r.v[0], src);
        v[1] = __shfl_sync(0xffffffffu, r.v[1], src);
        v[2] = __shfl_sync(0xffffffffu, r.v[2], src);
        const T cx = __shfl_sync(0xffffffffu, cv.x, src), cy = __shfl_sync(0xffffffffu, cv.y, src);
        if (p < S::PP && jb + p < cnt) {
          T wt;
          const long long q = sparse_cell<T, D, W>(v, org, gg, wb, p, cell, wt);
          red_add(gt + q, cx * wt, cy * wt);
        }
      } else {
        const T v[3] = {__shfl_sync(0xffffffffu, r.v[0], jb), __shfl_sync(0xffffffffu, r.v[1], jb),
                        __shfl_sync(0xffffffffu, r.v[2], jb)};
        const T cx = __shfl_sync(0xffffffffu, cv.x, jb), cy = __shfl_sync(0xffffffffu, cv.y, jb);
        for (int cell = lane; cell < S::CP; cell += 32) {
          T wt;
          const long long q = sparse_cell<T, D, W>(v, org, gg, wb, 0, cell, wt);
          red_add(gt + q, cx * wt, cy * wt);
        }
      }
      __syncwarp();
    }
  }
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_interp_sparse(Geom g, const __grid_constant__ KEval<T, W> ke, Sorted s,
                                                       const typename Traits<T>::C* __restrict__ grid,
                                                       typename Traits<T>::C* __restrict__ c, BatchTable bt) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  using S = Sparse<W, D>;
  __shared__ T wbuf[8][S::WB];
  __shared__ C part[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nt = *s.nsub, nsp = *s.nsparse;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  T* wb = wbuf[wid];
  for (int i = blockIdx.x * 8 + wid; i < nsp; i += gridDim.x * 8) {
    const int sub = nt + i;
    int bin = s.sub_bin[sub];
    const int p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];
    Geom gg;
    long long goff;
    sparse_geometry(g, bt, bin, gg, goff);
    int org[3];
    tile_origin(gg, bin, org);
    Rec r;
    r.v[0] = r.v[1] = r.v[2] = T(0);
    r.idx = 0;
    if (lane < cnt) r = rec[p0 + lane];
    const C* gt = grid + goff;
    for (int jb = 0; jb < cnt; jb += S::PP) {
      sparse_weights<T, D, W>(r, jb, gg, ke, wb);
      if (S::PP > 1) {
        const int p = lane / S::CP, cell = lane - p * S::CP;
        const int src = (jb + p) & 31;
        T v[3];
        v[0] = __shfl_sync(0xffffffffu, r.v[0], src);
        v[1] = __shfl_sync(0xffffffffu, r.v[1], src);
        v[2] = __shfl_sync(0xffffffffu, r.v[2], src);
        C acc;
        acc.x = acc.y = T(0);
        if (p < S::PP && jb + p < cnt) {
          T wt;
          const long long q = sparse_cell<T, D, W>(v, org, gg, wb, p, cell, wt);
          const C gv = __ldg(gt + q);
          acc.x = gv.x * wt;
          acc.y = gv.y * wt;
        }
        part[wid][lane] = acc;
        const int dst = __shfl_sync(0xffffffffu, r.idx, (jb + lane) & 31);
        __syncwarp();
        if (lane < S::PP && jb + lane < cnt) {
          C sum;
          sum.x = sum.y = T(0);
          for (int k = 0; k < S::CP; ++k) {
            sum.x += part[wid][lane * S::CP + k].x;
            sum.y += part[wid][lane * S::CP + k].y;
          }
          store_once(c + dst, sum);
        }
      } else {
        const T v[3] = {__shfl_sync(0xffffffffu, r.v[0], jb), __shfl_sync(0xffffffffu, r.v[1], jb),
                        __shfl_sync(0xffffffffu, r.v[2], jb)};
        T sr = T(0), si = T(0);
        for (int cell = lane; cell < S::CP; cell += 32) {
          T wt;
          const long long q = sparse_cell<T, D, W>(v, org, gg, wb, 0, cell, wt);
          const C gv = __ldg(gt + q);
          sr = fma(gv.x, wt, sr);
          si = fma(gv.y, wt, si);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        const int dst = __shfl_sync(0xffffffffu, r.idx, jb);
        if (lane == 0) {
          C out;
          out.x = sr;
          out.y = si;
          store_once(c + dst, out);
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace nufft

#include "spread_interp_q.cuh"
#include "spread_dw.cuh"

namespace nufft {

// shared-memory bytes of each kernel
template <typename T, int D>
inline size_t interp_bytes(const Geom& g) {
  return (size_t)g.ntile * sizeof(typename Traits<T>::C) + stage_bytes<T, D>(g.maxsub);
}

template <typename T>
inline T kernel_param(double beta);
template <>
inline float kernel_param<float>(double beta) {
  return (float)(beta * 1.4426950408889634073599246810019);
}
template <>
inline double kernel_param<double>(double beta) {
  return beta;
}

// the launch's kernel evaluation parameters (the table for g.horner)
template <typename T, int W>
inline KEval<T, W> make_keval(const Geom& g, double beta) {
  KEval<T, W> ke;
  ke.kpar = kernel_param<T>(beta);
  ke.cosh_kernel = g.kernel == 1 ? 1 : 0;
  ke.horner = (g.horner || ke.cosh_kernel) ? 1 : 0;
  const double* a = ke.horner ? horner_table(W, beta, ke.cosh_kernel) : nullptr;
  for (int i = 0; i < W * KEval<T, W>::NC; ++i) ke.a[i] = a ? T(a[i]) : T(0);
  return ke;
}

// The bank-grouped kernels (spread_interp_q.cuh) run 3D complex64 transforms of even w.
template <typename T, int D, int W>
constexpr bool kQuad = std::is_same<T, float>::value && D == 3 && (W % 2) == 0;

template <int W>
cudaError_t run_spread_q(const Geom& g, double beta, const Sorted& s, const void* c, void* grid, int* work,
                         const LaunchCfg& cfg, cudaStream_t st, bool configure_only, const BatchTable& bt) {
  auto kern = k_spread_q<W>;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, cfg.threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;  // blocks per SM; caller scales
    return cudaSuccess;
  }
  const KEval<float, W> ke = make_keval<float, W>(g, beta);
  // the tensor map covers the plan's own grid only; batches and foreign grids flush per cell
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const int use_map = (cfg.tmap != nullptr && bt.B == 0) ? 1 : 0;
  if (use_map) memcpy(&map, cfg.tmap, sizeof(map));
  kern<<<cfg.blocks, cfg.threads, cfg.smem, st>>>(g, ke, s, reinterpret_cast<const float2*>(c),
                                                  reinterpret_cast<float2*>(grid), work, bt, map, use_map);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_spread_sparse<float, 3, W><<<2 * cfg.blocks, 256, 0, st>>>(g, ke, s, reinterpret_cast<const float2*>(c),
                                                                reinterpret_cast<float2*>(grid), bt);
  return cudaGetLastError();
}

template <int W>
cudaError_t run_interp_q(const Geom& g, double beta, const Sorted& s, const void* grid, void* c, int* work,
                         const LaunchCfg& cfg, cudaStream_t st, bool configure_only, const BatchTable& bt) {
  auto kern = k_interp_q<W>;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, cfg.threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;
    return cudaSuccess;
  }
  const KEval<float, W> ke = make_keval<float, W>(g, beta);
  // the tensor map covers the plan's own grid only; batches and foreign grids take per-cell copies
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const int use_map = (cfg.tmap != nullptr && bt.B == 0) ? 1 : 0;
  if (use_map) memcpy(&map, cfg.tmap, sizeof(map));
  kern<<<cfg.blocks, cfg.threads, cfg.smem, st>>>(g, ke, s, reinterpret_cast<const float2*>(grid),
                                                  reinterpret_cast<float2*>(c), work, bt, map, use_map);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_interp_sparse<float, 3, W><<<2 * cfg.blocks, 256, 0, st>>>(g, ke, s, reinterpret_cast<const float2*>(grid),
                                                                reinterpret_cast<float2*>(c), bt);
  return cudaGetLastError();
}

// The complex128 spread with 32-bit words (spread_dw.cuh) serves w <= kDwMaxW; wider kernels
// (eps below about 1e-11) keep 64-bit words, whose finer resolution those tolerances need.
template <int D, int W>
cudaError_t run_spread_dw(const Geom& g, double beta, const Sorted& s, const void* c, void* grid, int* work,
                          const LaunchCfg& cfg, cudaStream_t st, bool configure_only, const BatchTable& bt) {
  // blocks of DWords::kThreads threads when the tile leaves room for one block per SM, two blocks
  // of 256 threads otherwise
  auto kern = g.kernel == 1 ? k_spread_dw<D, W, true> : k_spread_dw<D, W, false>;
  const int threads = cfg.smem > kOneBlockSmem ? DWords::kThreads : 256;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;  // blocks per SM; caller scales
    return cudaSuccess;
  }
  const KEval<double, W> ke = make_keval<double, W>(g, beta);
  kern<<<cfg.blocks, threads, cfg.smem, st>>>(g, ke, s, reinterpret_cast<const double2*>(c),
                                              reinterpret_cast<double2*>(grid), work, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_spread_sparse<double, D, W><<<2 * cfg.blocks, 256, 0, st>>>(g, ke, s, reinterpret_cast<const double2*>(c),
                                                                 reinterpret_cast<double2*>(grid), bt);
  return cudaGetLastError();
}

template <typename T, int D, int W>
cudaError_t run_spread(const Geom& g, double beta, const Sorted& s, const void* c, void* grid,
                       int* work, const LaunchCfg& cfg, cudaStream_t st, bool configure_only,
                       const BatchTable& bt) {
  if constexpr (kQuad<T, D, W>) {
    if (quad_layout(g)) return run_spread_q<W>(g, beta, s, c, grid, work, cfg, st, configure_only, bt);
  }
  if constexpr (std::is_same<T, double>::value && W <= kDwMaxW)
    return run_spread_dw<D, W>(g, beta, s, c, grid, work, cfg, st, configure_only, bt);
  auto kern = k_spread<T, D, W>;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, cfg.threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;  // blocks per SM; caller scales
    return cudaSuccess;
  }
  kern<<<cfg.blocks, cfg.threads, cfg.smem, st>>>(
      g, make_keval<T, W>(g, beta), s, reinterpret_cast<const typename Traits<T>::C*>(c),
      reinterpret_cast<typename Traits<T>::C*>(grid), work, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_spread_sparse<T, D, W><<<2 * cfg.blocks, 256, 0, st>>>(
      g, make_keval<T, W>(g, beta), s, reinterpret_cast<const typename Traits<T>::C*>(c),
      reinterpret_cast<typename Traits<T>::C*>(grid), bt);
  return cudaGetLastError();
}

template <typename T, int D, int W>
cudaError_t run_interp(const Geom& g, double beta, const Sorted& s, const void* grid, void* c,
                       int* work, const LaunchCfg& cfg, cudaStream_t st, bool configure_only,
                       const BatchTable& bt) {
  if constexpr (kQuad<T, D, W>) {
    if (quad_layout(g)) return run_interp_q<W>(g, beta, s, grid, c, work, cfg, st, configure_only, bt);
  }
  auto kern = InterpKernel<T, D, W>::get(g.kernel == 1);
  // the complex128 (double-float) interpolation: blocks of kInterpDfThreads when its tile leaves
  // room for one block per SM, two blocks of 256 threads otherwise
  const int threads = std::is_same<T, double>::value ? (cfg.smem > kOneBlockSmem ? kInterpDfThreads : 256)
                                                     : cfg.threads;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;
    return cudaSuccess;
  }
  kern<<<cfg.blocks, threads, cfg.smem, st>>>(
      g, make_keval<T, W>(g, beta), s, reinterpret_cast<const typename Traits<T>::C*>(grid),
      reinterpret_cast<typename Traits<T>::C*>(c), work, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_interp_sparse<T, D, W><<<2 * cfg.blocks, 256, 0, st>>>(
      g, make_keval<T, W>(g, beta), s, reinterpret_cast<const typename Traits<T>::C*>(grid),
      reinterpret_cast<typename Traits<T>::C*>(c), bt);
  return cudaGetLastError();
}

// w -> template dispatch for one (precision, dimension)
#define NUFFT_W_CASES(FN, T, D)                                             \
  switch (g.w) {                                                            \
    case 2: return FN<T, D, 2>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 3: return FN<T, D, 3>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 4: return FN<T, D, 4>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 5: return FN<T, D, 5>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 6: return FN<T, D, 6>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 7: return FN<T, D, 7>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 8: return FN<T, D, 8>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 9: return FN<T, D, 9>(g, beta, s, a, b, work, cfg, st, conf, bt);      \
    case 10: return FN<T, D, 10>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 11: return FN<T, D, 11>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 12: return FN<T, D, 12>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 13: return FN<T, D, 13>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 14: return FN<T, D, 14>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 15: return FN<T, D, 15>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    case 16: return FN<T, D, 16>(g, beta, s, a, b, work, cfg, st, conf, bt);    \
    default: return cudaErrorInvalidValue;                                  \
  }

#define NUFFT_DEFINE_SI(P, T, D)                                                                   \
  cudaError_t spread_##P##_d##D(const Geom& g, double beta, const Sorted& s, const void* a,       \
                                void* b, int* work, const LaunchCfg& cfg, cudaStream_t st,         \
                                bool conf, const BatchTable& bt) {                                 \
    NUFFT_W_CASES(run_spread, T, D)                                                                \
  }                                                                                                \
  cudaError_t interp_##P##_d##D(const Geom& g, double beta, const Sorted& s, const void* a,       \
                                void* b, int* work, const LaunchCfg& cfg, cudaStream_t st,         \
                                bool conf, const BatchTable& bt) {                                 \
    NUFFT_W_CASES(run_interp, T, D)                                                                \
  }

}  // namespace nufft
