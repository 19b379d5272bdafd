// Complex128 spreading (Eq. (bl) with the ES kernel, Eq. (ES), or its smooth variant) with its
// per-cell arithmetic on the FP32 pipe: the GB300's FP64 rate is about 1/64 of FP32, and the
// tiled complex128 spread spends 2 w^d multiply-adds per point on it.
//
// Each contribution v = c_j psi(l) K / max|c| (K = 2^52) is formed in double-float: the
// kernel values along the three dimensions are pairs (hi, lo) of floats (df.cuh, ~2^-47
// relative), the row weight c_j psi_3 psi_2 is a pair, and the product with the x value comes
// out as ph + e (ph the rounded product of the high parts, e its error term plus the two cross
// terms).  The contribution is then cut into three 32-bit integer words
//     v ~ x2 2^42 + x1 2^21 + x0,
// each obtained exactly from float operations: adding 1.5 2^23 to a float of magnitude below
// 2^22 rounds it to an integer that sits in the low bits of the result's bit pattern, and the
// remainder left by the rounding is again a float, exactly:
//     x2 = round(ph 2^-42),                  r2 = ph - x2 2^42        (|r2| <= 2^41, exact)
//     x1 = round(r2 2^-21) + round(e 2^-21),  r1, re the remainders   (|r1|, |re| <= 2^20)
//     x0 = round(r1 + re).
// The words' sum is v to within one unit or |v| 2^-46.  A cell of the shared tile holds six
// 32-bit words (x2, x1, x0 of the real and the imaginary part), added with 32-bit shared-memory
// atomics: six per cell against two 64-bit ones before, which this GPU runs 3.7-6 times slower
// than 32-bit ones.  Integer sums do not depend on the order of the atomics.  Word bounds for a
// chunk of c <= 512 points at K = 2^52: |sum x2| <= c 2^10, |sum x1| <= c (2^20 + 2^9),
// |sum x0| <= c 2^21 < 2^31.  The resolution max|c| 2^-52 is finer than the 2^-51 of the int64
// words this replaces; the double-float products (2^-46 of each contribution) set the accuracy.
#pragma once

namespace nufft {

struct DWords {
  static constexpr float M = 12582912.0f;  // 1.5 2^23
  static constexpr int B = 0x4B400000;     // its bit pattern
  static constexpr int kChunk = 512;       // points per flush
  static constexpr double K = 4503599627370496.0;  // 2^52
  static constexpr int kPlanes = 6;                // int words per tile cell
  static constexpr int kThreads = 512;             // threads per block (one block per SM)
};

// Words of v = a b (a, b normalised double-float pairs, |a b| <= 2^52 (1 + 2^-20)): x2 weighs
// 2^42, x1 2^21, x0 1.
__device__ __forceinline__ void dw_split(DF a, DF b, int& x2, int& x1, int& x0) {
  constexpr float M = DWords::M;
  const float ph = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -ph);  // exact error of ph
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float t2 = __fmaf_rn(ph, 0x1p-42f, M);                           // M + x2
  const float r2 = __fadd_rn(ph, __fmaf_rn(t2, -0x1p42f, M * 0x1p42f));  // ph - x2 2^42
  const float t1 = __fmaf_rn(r2, 0x1p-21f, M);                           // M + round(r2 2^-21)
  const float r1 = __fadd_rn(r2, __fmaf_rn(t1, -0x1p21f, M * 0x1p21f));
  const float te = __fmaf_rn(e, 0x1p-21f, M);                            // M + round(e 2^-21)
  const float re = __fadd_rn(e, __fmaf_rn(te, -0x1p21f, M * 0x1p21f));
  const float t0 = __fadd_rn(__fadd_rn(r1, re), M);                      // M + round(r1 + re)
  x2 = __float_as_int(t2) - DWords::B;
  x1 = __float_as_int(t1) + __float_as_int(te) - 2 * DWords::B;
  x0 = __float_as_int(t0) - DWords::B;
}
__device__ __forceinline__ long long dw_value(int x2, int x1, int x0) {
  return ((long long)x2 << 42) + ((long long)x1 << 21) + (long long)x0;
}

// Add a six-word tile (scaled by inv) into the fine grid with periodic wrapping.  Planes:
// x2 re, x2 im, x1 re, x1 im, x0 re, x0 im, each ntile ints.
__device__ __forceinline__ void flush_tile_dw(const Geom& g, const int* org, const int* tile, double inv,
                                              double2* grid) {
  const int T0 = g.T[0], ntile = g.ntile;
  const int nrows = ntile / T0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
    const int t1 = row % g.T[1], t2 = row / g.T[1];
    const long long gy = wrap_idx(org[1] + t1, g.n[1]);
    const long long gz = wrap_idx(org[2] + t2, g.n[2]);
    double2* grow = grid + (gz * g.n[1] + gy) * (long long)g.n[0];
    for (int t0 = lane; t0 < T0; t0 += 32) {
      const int c = row * T0 + t0;
      const long long vr = dw_value(tile[c], tile[2 * ntile + c], tile[4 * ntile + c]);
      const long long vi = dw_value(tile[ntile + c], tile[3 * ntile + c], tile[5 * ntile + c]);
      if (vr == 0 && vi == 0) continue;
      red_add(grow + wrap_idx(org[0] + t0, g.n[0]), (double)vr * inv, (double)vi * inv);
    }
  }
}

// Tiled complex128 spread: the structure of k_spread (persistent blocks pulling subproblems,
// strengths staged in shared memory, points in bank-group order, up to 8 threads per point of
// a small subproblem) with the six-word accumulation above, in blocks of 512 threads: the tile of
// a 16x8x8 bin at w = 10 takes most of an SM's shared memory, so one block runs per SM.  Kernel values are evaluated with
// the formula in double-float (COSH: the smooth variant), whatever the plan's kerevalmeth, as
// in the complex128 interpolation.  A subproblem of more than 512 points runs in chunks of 512
// points, each accumulated on a zeroed tile and flushed on its own.
template <int D, int W, bool COSH>
__global__ void __launch_bounds__(DWords::kThreads, 1) k_spread_dw(Geom g, const __grid_constant__ KEval<double, W> ke, Sorted s,
                                                      const double2* __restrict__ c, double2* __restrict__ grid,
                                                      int* __restrict__ work, BatchTable bt) {
  using Rec = RecD;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[NRES_SPREAD];
  __shared__ int s_sub, s_bin, s_nslots;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;
  __shared__ unsigned long long s_maxbits;

  const int ntile = g.ntile, maxsub = g.maxsub;
  int* tile = reinterpret_cast<int*>(smem);  // six planes of ntile ints
  int* p2r = tile;
  int* p2i = tile + ntile;
  int* p1r = tile + 2 * ntile;
  int* p1i = tile + 3 * ntile;
  int* p0r = tile + 4 * ntile;
  int* p0i = tile + 5 * ntile;
  double2* sc = reinterpret_cast<double2*>(smem + ((DWords::kPlanes * (size_t)ntile * 4 + 15) & ~(size_t)15));
  Stage<double, D> st = carve_stage<double, D>(reinterpret_cast<unsigned char*>(sc + maxsub), maxsub);
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const int T0 = g.T[0], T01 = g.T[0] * g.T[1];
  const DF bdf = df_of(ke.kpar);  // beta

  for (;;) {
    if (threadIdx.x == 0) {
      next_subproblem(g, s, bt, work, &s_sub, &s_bin, &s_goff, &s_geo);
      s_maxbits = 0;
    }
    if (threadIdx.x < NRES_SPREAD) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];

    double mloc = 0.0;
    for (int q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
      Rec r[4];
      double2 cv[4];
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
          stage_point<double, D, W, NRES_SPREAD>(g, r[u], q, st, hist);
          sc[q] = cv[u];
          mloc = fmax(mloc, fmax(fabs(cv[u].x), fabs(cv[u].y)));
        }
      }
    }
    // non-negative doubles order like their bit patterns; NaN (all bits high) wins
    if (!(mloc == mloc)) mloc = INFINITY;
    atomicMax(&s_maxbits, (unsigned long long)__double_as_longlong(mloc));
    const int nslots = bucket_order<double, D, NRES_SPREAD, false>(cnt, st, hist, &s_nslots);  // synchronises
    const double maxabs = __longlong_as_double((long long)s_maxbits);
    int org[3];
    tile_origin(s_geo, bin, org);

    for (int c0 = 0; c0 < nslots; c0 += DWords::kChunk) {
      const int c1 = min(nslots, c0 + DWords::kChunk);
      {  // zero the six planes
        int4* t4 = reinterpret_cast<int4*>(tile);
        const int n4 = (DWords::kPlanes * ntile) >> 2;
        for (int t = threadIdx.x; t < n4; t += blockDim.x) t4[t] = make_int4(0, 0, 0, 0);
        for (int t = 4 * n4 + threadIdx.x; t < DWords::kPlanes * ntile; t += blockDim.x) tile[t] = 0;
      }
      __syncthreads();
      double scale = 0.0, inv = 0.0;
      if (maxabs > 0.0 && maxabs < INFINITY) {
        scale = DWords::K / maxabs;
        inv = maxabs / DWords::K;
      } else if (!(maxabs == 0.0)) {
        inv = NAN;  // non-finite strengths: make the whole tile NaN
      }

      // a chunk of few points (about a hundred per 8x8x8 bin at w = 10) would leave most threads
      // idle through the w^3 cells of a point, so up to 8 threads share a point, each taking
      // every tpp-th plane of its stencil (3D)
      int tpp = 1;
      if constexpr (D == 3) {
        while (tpp < 8 && tpp < W && 2 * tpp * (c1 - c0) <= (int)blockDim.x) tpp *= 2;
      }
      const int ltpp = __ffs(tpp) - 1;
      for (int u = threadIdx.x; u < ((c1 - c0) << ltpp); u += blockDim.x) {
        const int sl = c0 + (u >> ltpp), part = u & (tpp - 1);
        const int q = st.order[sl];
        if (q == kEmptySlot) continue;
        const Rec rq = rec[p0 + q];
        DF k0[W];
        int ts0, ts1 = 0, ts2 = 0;
        point_weights_df<W>(rq.v[0], g.B[0], bdf, COSH, ts0, k0);
        DF k1[(D > 1) ? W : 1];
        if constexpr (D > 1) point_weights_df<W>(rq.v[1], g.B[1], bdf, COSH, ts1, k1);
        else k1[0] = DF{1.0f, 0.0f};
        DF f2d = {0.0f, 0.0f};
        int st2 = 0;
        if constexpr (D > 2) {
          const double v2 = rq.v[2];
          const int il2 = min((int)v2, g.B[2] - 1);
          const double f2 = v2 - double(il2);
          st2 = stencil_step<W>(f2);
          ts2 = il2 + st2;
          f2d = df_of(f2);
        }
        const double2 cv = sc[q];
        const DF cr = df_of(cv.x * scale), ci = df_of(cv.y * scale);
        const int base = ts0 + T0 * ts1 + T01 * ts2;
        constexpr int W1 = (D > 1) ? W : 1;
        constexpr int W2 = (D > 2) ? W : 1;
#pragma unroll 1
        for (int l2 = part; l2 < W2; l2 += tpp) {
          DF k2 = {1.0f, 0.0f};
          if constexpr (D > 2) {
            const DF sc2 = DF{2.0f / W, __double2float_rn(2.0 / W - (double)(2.0f / W))};
            const DF z = df_mul(df_add(DF{(float)(l2 - W / 2 + st2), 0.0f}, DF{-f2d.hi, -f2d.lo}), sc2);
            k2 = es_eval_df_z(z, bdf, COSH);
          }
          const DF cr2 = df_mul(cr, k2), ci2 = df_mul(ci, k2);
          // rows one at a time (the row's y value picked from registers): the fully unrolled w^2
          // rows of w cells overflowed the instruction cache (ncu: 1.1 no-instruction stalls per issue)
#pragma unroll 1
          for (int l1 = 0; l1 < W1; ++l1) {
            const DF k1v = df_pick<(D > 1) ? W : 1>(k1, l1);
            const DF cr1 = df_mul(cr2, k1v), ci1 = df_mul(ci2, k1v);
            const int o = base + l1 * T0 + l2 * T01;
#pragma unroll
            for (int l0 = 0; l0 < W; ++l0) {
              int r2, i2, r1, i1, r0, i0;
              dw_split(cr1, k0[l0], r2, r1, r0);
              dw_split(ci1, k0[l0], i2, i1, i0);
              atomicAdd(p2r + o + l0, r2);
              atomicAdd(p2i + o + l0, i2);
              atomicAdd(p1r + o + l0, r1);
              atomicAdd(p1i + o + l0, i1);
              atomicAdd(p0r + o + l0, r0);
              atomicAdd(p0i + o + l0, i0);
            }
          }
        }
      }
      __syncthreads();
      flush_tile_dw(s_geo, org, tile, inv, grid + s_goff);
      __syncthreads();
    }
  }
}

}  // namespace nufft
