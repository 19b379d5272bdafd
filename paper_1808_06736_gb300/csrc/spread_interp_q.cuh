// Bank-grouped spreading and interpolation for 3D grids and even kernel widths
// (the production path of the 3D complex64 transforms: Eq. (bl) and Eq. (interp)
// with the ES kernel, Eq. (ES), one thread block per subproblem as in
// spread_interp.cuh).
//
// Several lanes share one point, each taking an interleaved subset of its
// w^2 stencil rows (rho = l1 + w l2):
//   * spreading: 4 lanes per point (rows rho = 4i + q, q = lane mod 4), 8
//     points per warp, 32-bit integer shared atomics on separate re / im planes;
//   * interpolation: 2 lanes per point (rows rho = 2i + q), 8 points per
//     half-warp, 8-byte loads of (re, im) pairs, the two partial sums added
//     with one shuffle.
// The tile is laid out with a row stride qs0 = 8 (mod 16) and qt1 = w (mod 4)
// rows per plane (Geom::qs0, qt1), so that a stencil row rho starts rho qs0
// (mod 32) cells after the stencil corner.  The q lanes of one point then sit
// on banks corner + q qs0 + l0, i.e. on the 4 (spread) or 2 (interp) cosets of
// the corner's residue mod 8 in the 32 banks (16 double banks), and the points
// of a warp (half-warp) are conflict-free when their corners differ mod 8.
// Points are dealt out in rounds over the 8 residue classes of their corner
// (its x position in the tile mod 8): the interpolation packs rounds whole into
// groups of 8 slots (a half-warp), the spread packs them without gaps.
// Compared with one point per lane and 32 classes this cuts the class-imbalance
// tail that put two points of one class into a warp.
//
// The tile's x-origin is the bin origin - floor(w/2), rounded down to an even
// grid index (so the interpolation can fetch it with one TMA copy whose x
// offset is 16-byte aligned); xsh = 0 or 1 is the shift.
#pragma once

#include <cuda.h>

// included by spread_interp.cuh after the helpers it uses
namespace nufft {

__host__ __device__ constexpr int qgcd(int a, int b) { return b == 0 ? a : qgcd(b, a % b); }
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Kernel values for the bank-grouped kernels.  The ES formula, Eq. (ES), with the PTX
// approximate square root and base-2 exponential (one special-function operation each):
// phi = 2^(kpar (s - 1)), s = sqrt(max(1 - z^2, 0)), kpar = beta log2(e).  The argument of
// the exponential lies in [-kpar, 0] (about [-20, 0] for w <= 8 in complex64), so the result
// is a normal float; both instructions are accurate to a few units in the last place, about
// the rounding of s itself (whose absolute error kpar amplifies to ~1e-6 relative in phi).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <int W>
__device__ __forceinline__ float es_node_q(const KEval<float, W>& ke, int t, int step, float f) {
  if (ke.horner) return kernel_node<float, W>(ke, t, step, f);  // Sec. 5.3's polynomial
  const float z = node_z<W>(t, step, f);
  return ex2_approx(fmaf(ke.kpar, sqrt_approx(fmaxf(fmaf(-z, z, 1.0f), 0.0f)), -ke.kpar));
}
// Shared-memory accesses by 32-bit shared-window address (constant offsets fold into the
// instruction): the fixed-point add of the spread (no value returned) and the (re, im) load
// of the interpolation.
__device__ __forceinline__ void red_shared(unsigned addr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ float2 ld_shared_f2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// the cell of a coordinate v in a bin of extent B: stencil step and start (cell + step), fraction
template <int W>
__device__ __forceinline__ void coord_cell(float v, int B, int& step, int& start, float& f) {
  const int il = min((int)v, B - 1);
  f = v - float(il);
  step = stencil_step<W>(f);
  start = il + step;
}

// Stage a record in bank-grouped order: its class is the x position of its stencil
// corner in the tile mod 8.  hist[8] must be zero on entry.
template <int W>
__device__ __forceinline__ void stage_point_q(const Geom& g, const RecF& r, int q, int xsh, Stage<float, 3>& st,
                                              int* hist) {
  const float v = r.v[0];
  const int il = min((int)v, g.B[0] - 1);
  const int xl = il + stencil_step<W>(v - float(il)) + xsh;
  const int cls = xl & 7;
  st.res[q] = (unsigned short)cls;
  st.rank[q] = (unsigned short)atomicAdd(&hist[cls], 1);
}

// Add a bank-grouped fixed-point tile (scaled by inv) into the fine grid, wrapping
// periodically.  Tile cell (tx, ty, tz) -> grid (ox + tx, org1 + ty, org2 + tz), ox the
// even x-origin; cells tx < T0 + xsh, ty < T1 carry data.  Rows that do not wrap go out as
// 16-byte vector reductions of two cells from an even grid index.
__device__ __forceinline__ void flush_tile_q(const Geom& g, int ox, int xsh, const int* org, const int* tre,
                                             const int* tim, float inv, float2* grid) {
  const int S0 = g.qs0, T1 = g.T[1], QT1 = g.qt1;
  const int tx = g.T[0] + xsh;  // cells per row that carry data
  const int nrows = T1 * g.T[2];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const bool pairs = ((g.n[0] & 1) == 0) && ox >= 0 && ox + tx <= g.n[0];
  const int npair = (tx + 1) >> 1;
  for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
    const int t1 = row % T1, t2 = row / T1;
    const long long gy = wrap_idx(org[1] + t1, g.n[1]);
    const long long gz = wrap_idx(org[2] + t2, g.n[2]);
    float2* grow = grid + (gz * g.n[1] + gy) * (long long)g.n[0];
    const int* ar = tre + (t2 * QT1 + t1) * S0;
    const int* ai = tim + (t2 * QT1 + t1) * S0;
    if (pairs) {
      for (int k = lane; k < npair; k += 32) {
        const int t0 = 2 * k;
        const int a0 = ar[t0], b0 = ai[t0];
        const int a1 = t0 + 1 < tx ? ar[t0 + 1] : 0, b1 = t0 + 1 < tx ? ai[t0 + 1] : 0;
        if ((a0 | b0 | a1 | b1) == 0) continue;
        if (t0 + 1 < tx)
          red_add2(grow + ox + t0, float(a0) * inv, float(b0) * inv, float(a1) * inv, float(b1) * inv);
        else
          red_add(grow + ox + t0, float(a0) * inv, float(b0) * inv);
      }
    } else {
      for (int t0 = lane; t0 < tx; t0 += 32) {
        const int a = ar[t0], b = ai[t0];
        if ((a | b) == 0) continue;
        red_add(grow + wrap_idx(ox + t0, g.n[0]), float(a) * inv, float(b) * inv);
      }
    }
  }
}

// x-origin (even) and shift of a subproblem's tile
__device__ __forceinline__ int tile_xsh(const int* org) { return org[0] & 1; }

// ------------------------------------------------------ TMA tile fetch
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with this parity to complete, at most about 2^31 SM cycles (~1 s);
// false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One tiled TMA load of a 3D box (x in floats, 16-byte aligned) into shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// contiguous bulk copy of nbytes (a multiple of 16) from global to shared memory (both
// addresses 16-byte aligned), completing on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned nbytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(nbytes), "r"(smem_u32(bar))
               : "memory");
}

// bulk tensor reduce-add of a 3D box of floats from shared memory into global memory
// (x in floats, 16-byte aligned, not negative), in the current bulk group
__device__ __forceinline__ void tma_reduce_add_3d(const void* src, const CUtensorMap* map, int x, int y, int z) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<unsigned long long>(map)),
      "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread: wait until the bulk operations it committed have read their shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and until they have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Flush of a tile that lies inside the grid: the fixed-point planes are converted in place to
// (re, im) float pairs (each thread holds a run of up to kFlushCells consecutive cells in
// registers across one barrier) and added to the grid by one bulk tensor reduction of the whole
// box.  Cells that hold 0 give exactly 0 (also when inv is NaN, as in the per-cell flush).  The
// caller waits (bulk_wait_read) before the tile is written again.
constexpr int kFlushCells = 19;
__device__ __forceinline__ void flush_tile_tma(int* tre, int qtile, float inv, const CUtensorMap* map, int x, int y,
                                               int z) {
  int re[kFlushCells], im[kFlushCells];
  const int c0 = threadIdx.x * kFlushCells;  // odd run length: the runs of a warp fall in distinct banks
#pragma unroll
  for (int k = 0; k < kFlushCells; ++k) {
    const int c = c0 + k;
    re[k] = c < qtile ? tre[c] : 0;
    im[k] = c < qtile ? tre[qtile + c] : 0;
  }
  __syncthreads();
  float2* t2 = reinterpret_cast<float2*>(tre);
#pragma unroll
  for (int k = 0; k < kFlushCells; ++k) {
    const int c = c0 + k;
    if (c < qtile) t2[c] = make_float2(re[k] ? float(re[k]) * inv : 0.f, im[k] ? float(im[k]) * inv : 0.f);
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma_reduce_add_3d(t2, map, x, y, z);
    bulk_commit();
  }
}

// ------------------------------------------------------------ quad spread
// Shared memory (spread_q_bytes): re and im planes of qtile ints (128-byte aligned), the staged
// strengths (maxsub float2), the gapless point order (3 maxsub shorts).

// One pass of a subproblem's points over the tile (the main loop of k_spread_q).
template <int W>
__device__ __forceinline__ void spread_pass_q(const Geom& g, const KEval<float, W>& ke, const RecF* __restrict__ rec,
                                              int p0, const Stage<float, 3>& st, const float2* sc, int nslots,
                                              int npass, int pass, float thr, float scale, int xsh, unsigned tre_s,
                                              int qtile) {
  constexpr bool kPar = (W % 4) == 2;
  constexpr int YSTEP = kPar ? 2 : 4, ZSTEP = kPar ? 2 : 1;
  constexpr int NA = W / YSTEP, NB = W / ZSTEP;  // y and z nodes per lane
  constexpr int NS = (W + 3) / 4;                // nodes per lane of a shared row (t = q mod 4)
  const int S0 = g.qs0, S01 = g.qs0 * g.qt1;
  const int lane = threadIdx.x & 31, p = lane >> 2, q = lane & 3;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int qb = lane & ~3;  // first lane of this point's quad
  const int yq0 = kPar ? (q & 1) : q, zq0 = kPar ? (q >> 1) : 0;
  const int loff = yq0 * S0 + zq0 * S01;
  const int ngroups = (nslots + 7) >> 3;
  for (int gi = wid; gi < ngroups; gi += nw) {  // warp-uniform trip count: shuffles below see all lanes
    const int sl = gi * 8 + p;
    int qi = sl < nslots ? (int)st.order[sl] : (int)kEmptySlot;
    if (npass == 2 && qi != kEmptySlot) {  // this pass's strengths only
      const float2 cq = sc[qi];
      if ((fmaxf(fabsf(cq.x), fabsf(cq.y)) > thr) != (pass == 0)) qi = kEmptySlot;
    }
    const bool act = qi != kEmptySlot;
    RecF r;
    r.v[0] = r.v[1] = r.v[2] = 0.f;
    if (act) r = rec[p0 + qi];
    int sx, sy, sz, ts0, ts1, ts2;
    float fx, fy, fz;
    coord_cell<W>(r.v[0], g.B[0], sx, ts0, fx);
    coord_cell<W>(r.v[1], g.B[1], sy, ts1, fy);
    coord_cell<W>(r.v[2], g.B[2], sz, ts2, fz);
    // x values: lane q evaluates nodes t = q (mod 4), the quad exchanges them
    float kq[NS], k0[W];
#pragma unroll
    for (int u = 0; u < NS; ++u) kq[u] = (q + 4 * u < W) ? es_node_q<W>(ke, q + 4 * u, sx, fx) : 0.f;
#pragma unroll
    for (int t = 0; t < W; ++t) k0[t] = __shfl_sync(0xffffffffu, kq[t / 4], qb + (t & 3));
    float K2[NB];
    if constexpr (kPar) {
#pragma unroll
      for (int b = 0; b < NB; ++b) K2[b] = es_node_q<W>(ke, zq0 + ZSTEP * b, sz, fz);
    } else {  // every z node: evaluated t = q (mod 4) and exchanged like x
#pragma unroll
      for (int u = 0; u < NS; ++u) kq[u] = (q + 4 * u < W) ? es_node_q<W>(ke, q + 4 * u, sz, fz) : 0.f;
#pragma unroll
      for (int t = 0; t < W; ++t) K2[t] = __shfl_sync(0xffffffffu, kq[t / 4], qb + (t & 3));
    }
    if (!act) continue;
    float K1[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) K1[a] = es_node_q<W>(ke, yq0 + YSTEP * a, sy, fy);
    const float2 cv = sc[qi];
    const float cr = cv.x * scale, ci = cv.y * scale;
    const unsigned pr = tre_s + 4u * (unsigned)(ts0 + xsh + S0 * ts1 + S01 * ts2 + loff);
    const unsigned pi = pr + 4u * (unsigned)qtile;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float cr2 = cr * K2[b], ci2 = ci * K2[b];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const float cr1 = cr2 * K1[a], ci1 = ci2 * K1[a];
        const unsigned off = 4u * (unsigned)(YSTEP * a * S0 + ZSTEP * b * S01);
#pragma unroll
        for (int l0 = 0; l0 < W; ++l0) {
          red_shared(pr + off + 4u * l0, Fixed<float>::bits(Fixed<float>::quant_fma(cr1, k0[l0])));
          red_shared(pi + off + 4u * l0, Fixed<float>::bits(Fixed<float>::quant_fma(ci1, k0[l0])));
        }
      }
    }
  }
}

template <int W>
__global__ void __launch_bounds__(256, 4) k_spread_q(Geom g, const __grid_constant__ KEval<float, W> ke, Sorted s,
                                                    const float2* __restrict__ c, float2* __restrict__ grid,
                                                    int* __restrict__ work, BatchTable bt,
                                                    const __grid_constant__ CUtensorMap tmap, int use_tmap) {
  // Lane q of a point's quad takes the stencil rows (l1, l2) with
  //   w = 2 (mod 4): l1 = q&1 (mod 2), l2 = q>>1 (mod 2)  -- w/2 x w/2 rows;
  //   w = 0 (mod 4): l1 = q (mod 4), every l2             -- w/4 x w rows.
  // Its row offset yq0 qs0 + zq0 qs01 is 0, 8, 16 or 24 banks (mod 32) from lane 0's, and
  // the remaining row offsets (multiples of ystep, zstep) are the same for the four lanes.
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[8];
  __shared__ int s_sub, s_bin, s_nslots, s_maxbits, s_nsmall, s_msmall;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;

  const int qtile = g.qtile, maxsub = g.maxsub;
  // the tile starts 128-byte aligned: the source of the bulk tensor reduction
  int* tre = reinterpret_cast<int*>(smem + ((128u - (smem_u32(smem) & 127u)) & 127u));
  int* tim = tre + qtile;
  float2* sc = reinterpret_cast<float2*>(tim + qtile);
  Stage<float, 3> st = carve_stage<float, 3>(reinterpret_cast<unsigned char*>(sc + maxsub), maxsub);
  const RecF* __restrict__ rec = reinterpret_cast<const RecF*>(s.rec);
  const unsigned tre_s = smem_u32(tre);

  // tiles flushed by one bulk reduction: whole tile inside the grid, the plan's own grid
  const bool tma_ok = use_tmap && bt.B == 0 && qtile <= kFlushCells * (int)blockDim.x;
  for (;;) {
    if (threadIdx.x == 0) {
      next_subproblem(g, s, bt, work, &s_sub, &s_bin, &s_goff, &s_geo);
      s_maxbits = 0;
      s_nsmall = 0;
      s_msmall = 0;
    }
    if (threadIdx.x < 8) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) {
      if (tma_ok && threadIdx.x == 0) bulk_wait_all();
      break;
    }
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];
    int org[3];
    tile_origin(s_geo, bin, org);
    const int xsh = tile_xsh(org);

    float mloc = 0.f;
    for (int q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
      RecF r[4];
      float2 cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q0 + u * blockDim.x;
        if (k < cnt) r[u] = rec[p0 + k];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q0 + u * blockDim.x;
        if (k < cnt) cv[u] = load_once(c + r[u].idx);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q0 + u * blockDim.x;
        if (k < cnt) {
          stage_point_q<W>(g, r[u], k, xsh, st, hist);
          sc[k] = cv[u];
          mloc = fmaxf(mloc, fmaxf(fabsf(cv[u].x), fabsf(cv[u].y)));
        }
      }
    }
    if (!(mloc == mloc)) mloc = INFINITY;  // NaN strengths make the tile NaN below
    atomicMax(&s_maxbits, __float_as_int(mloc));
    // gapless rounds: the kernel is bound by instruction issue, so the empty slots of round-aligned
    // packing cost more than the conflicts it saves (measured: 12.48 -> 12.00 ms on 1e8 points)
    const int nslots = bucket_order<float, 3, 8, false>(cnt, st, hist, &s_nslots);

    // the tile is zeroed only now, so the previous tile's bulk reduction reads it while this
    // subproblem's points are staged and ordered; plan_passes' barrier orders the zeros
    // before the main loop
    if (tma_ok && threadIdx.x == 0) bulk_wait_read();
    __syncthreads();
    for (int t = threadIdx.x; t < qtile; t += blockDim.x) {
      tre[t] = 0;
      tim[t] = 0;
    }
    const float maxabs = __int_as_float(s_maxbits);
    const double K = fmin(Fixed<float>::KMAX, floor(Fixed<float>::IMAX / (double)cnt) - 1.0);
    float thr, smax;
    const int npass = plan_passes(sc, cnt, maxabs, &s_nsmall, &s_msmall, &thr, &smax);
    for (int pass = 0; pass < npass; ++pass) {
      if (pass == 1) {  // the small strengths, on a zeroed tile
        if (tma_ok && threadIdx.x == 0) bulk_wait_read();
        __syncthreads();
        for (int t = threadIdx.x; t < qtile; t += blockDim.x) {
          tre[t] = 0;
          tim[t] = 0;
        }
        __syncthreads();
      }
      float scale, inv;
      pass_scale(K, pass == 0 ? maxabs : smax, &scale, &inv);
      spread_pass_q<W>(g, ke, rec, p0, st, sc, nslots, npass, pass, thr, scale, xsh, tre_s, qtile);
      __syncthreads();
      const int ox = org[0] - xsh;
      if (tma_ok && ox >= 0 && ox + g.T[0] + xsh <= s_geo.n[0] && org[1] >= 0 && org[1] + g.T[1] <= s_geo.n[1] &&
          org[2] >= 0 && org[2] + g.T[2] <= s_geo.n[2])
        flush_tile_tma(tre, qtile, inv, &tmap, 2 * ox, org[1], org[2]);
      else
        flush_tile_q(s_geo, ox, xsh, org, tre, tim, inv, grid + s_goff);
      __syncthreads();
    }  // pass
  }
}

// ------------------------------------------------------ paired interpolation
// Shared memory (interp_q_bytes): the tile (qtile float2, 128-byte aligned for TMA) and the
// aligned point order (5 maxsub shorts).

template <int W>
__global__ void __launch_bounds__(256, 4) k_interp_q(Geom g, const __grid_constant__ KEval<float, W> ke, Sorted s,
                                                    const float2* __restrict__ grid, float2* __restrict__ c,
                                                    int* __restrict__ work, BatchTable bt,
                                                    const __grid_constant__ CUtensorMap tmap, int use_tmap) {
  constexpr int NM = W / 2;  // stencil rows of one plane per lane
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[8];
  __shared__ int s_sub, s_bin, s_nslots;
  __shared__ long long s_goff;
  __shared__ Geom s_geo;
  __shared__ __align__(8) unsigned long long s_bar;

  const int qtile = g.qtile, maxsub = g.maxsub, S0 = g.qs0, QT1 = g.qt1, S01 = g.qs0 * g.qt1;
  unsigned char* abase = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
  float2* tile = reinterpret_cast<float2*>(abase);
  const unsigned tile_s = smem_u32(tile);
  Stage<float, 3> st = carve_stage<float, 3>(reinterpret_cast<unsigned char*>(tile + qtile), maxsub);
  const RecF* __restrict__ rec = reinterpret_cast<const RecF*>(s.rec);
  const int lane = threadIdx.x & 31, p = lane >> 1, q = lane & 1;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned tile_bytes = (unsigned)qtile * 8u;
  unsigned phase = 0;
  if (use_tmap && threadIdx.x == 0) mbar_init(&s_bar);
  // wrapping tiles fetched by row copies (the plan's own grid, even n0): see below
  const int ntx_max = (g.T[0] + 2) & ~1;
  int next = 0;  // thread 0: the subproblem id claimed for the next iteration
  if (threadIdx.x == 0) next = atomicAdd(work, 1);

  for (;;) {
    if (threadIdx.x == 0) {
      resolve_subproblem(g, s, bt, next, &s_sub, &s_bin, &s_goff, &s_geo);
      next = atomicAdd(work, 1);  // in flight while this subproblem is worked on
    }
    if (threadIdx.x < 8) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s_bin, p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];
    int org[3];
    tile_origin(s_geo, bin, org);
    const int xsh = tile_xsh(org), ox = org[0] - xsh, tx = g.T[0] + xsh;
    const int n0 = s_geo.n[0], n1 = s_geo.n[1], n2 = s_geo.n[2];
    // one TMA box when the used part of the tile lies inside the grid (no periodic wrap)
    const bool by_tma = use_tmap && ox >= 0 && ox + tx <= n0 && org[1] >= 0 && org[1] + g.T[1] <= n1 &&
                        org[2] >= 0 && org[2] + g.T[2] <= n2;
    // A tile that wraps: one bulk copy per row, or two where the row crosses the grid's x edge,
    // of its cells [0, ntx) (data cells rounded up to even: ox and n0 even, so every piece starts
    // 16-byte aligned and holds whole pairs of cells), all completing on the tile's mbarrier.
    const bool by_rows = !by_tma && use_tmap && (n0 & 1) == 0 && ntx_max <= n0;
    if (by_tma) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&s_bar, tile_bytes);
        tma_load_3d(tile, &tmap, 2 * ox, org[1], org[2], &s_bar);
      }
    } else if (by_rows) {
      const int ntx = (tx + 1) & ~1, nrows = g.T[1] * g.T[2];
      if (threadIdx.x == 0) mbar_expect_tx(&s_bar, 8u * (unsigned)(ntx * nrows));
      __syncthreads();  // the expected bytes are posted before any copy can complete
      const float2* gridt = grid + s_goff;
      fence_proxy_async_smem();
      for (int row = threadIdx.x; row < nrows; row += blockDim.x) {
        const int t1 = row % g.T[1], t2 = row / g.T[1];
        const long long gy = wrap_idx(org[1] + t1, n1);
        const long long gz = wrap_idx(org[2] + t2, n2);
        const float2* grow = gridt + (gz * n1 + gy) * (long long)n0;
        float2* trow = tile + (t2 * QT1 + t1) * S0;
        if (ox >= 0 && ox + ntx <= n0) {
          bulk_load(trow, grow + ox, 8u * ntx, &s_bar);
        } else {
          const int a = ox < 0 ? -ox : n0 - ox;  // cells before the edge
          bulk_load(trow, grow + (ox < 0 ? ox + n0 : ox), 8u * a, &s_bar);
          bulk_load(trow + a, grow, 8u * (ntx - a), &s_bar);
        }
      }
    } else {
      const float2* gridt = grid + s_goff;
      const int nrows = g.T[1] * g.T[2];
      for (int row = wid; row < nrows; row += nw) {
        const int t1 = row % g.T[1], t2 = row / g.T[1];
        const long long gy = wrap_idx(org[1] + t1, n1);
        const long long gz = wrap_idx(org[2] + t2, n2);
        const float2* grow = gridt + (gz * n1 + gy) * (long long)n0;
        float2* trow = tile + (t2 * QT1 + t1) * S0;
        for (int t0 = lane; t0 < tx; t0 += 32) cp_async_elem(trow + t0, grow + wrap_idx(ox + t0, n0));
      }
      cp_async_commit();
    }
    // records while the tile is in flight
    for (int q0 = threadIdx.x; q0 < cnt; q0 += 4 * blockDim.x) {
      RecF r[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q0 + u * blockDim.x;
        if (k < cnt) r[u] = rec[p0 + k];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = q0 + u * blockDim.x;
        if (k < cnt) stage_point_q<W>(g, r[u], k, xsh, st, hist);
      }
    }
    if (by_tma || by_rows) {
      const bool ok = mbar_wait_bounded(&s_bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {  // the copy never completed: report and stop this block
        if (threadIdx.x == 0) {
          if (s.err) atomicCAS(s.err, 0, NUFFT_ERR_CUDA);
          mbar_wait_bounded(&s_bar, phase ^ 1u);  // give the copy in flight one more bounded chance
        }
        return;
      }
    } else {
      cp_async_wait_all();
    }
    const int nslots = bucket_order<float, 3, 8, true>(cnt, st, hist, &s_nslots);

    const int ngroups = (nslots + 15) >> 4;
    for (int gi = wid; gi < ngroups; gi += nw) {  // warp-uniform trip count: the shuffles see all lanes
      const int sl = gi * 16 + p;
      const int qi = sl < nslots ? (int)st.order[sl] : (int)kEmptySlot;
      const bool act = qi != kEmptySlot;
      RecF r;
      r.v[0] = r.v[1] = r.v[2] = 0.f;
      r.idx = 0;
      if (act) r = rec[p0 + qi];
      int sx, sy, sz, ts0, ts1, ts2;
      float fx, fy, fz;
      coord_cell<W>(r.v[0], g.B[0], sx, ts0, fx);
      coord_cell<W>(r.v[1], g.B[1], sy, ts1, fy);
      coord_cell<W>(r.v[2], g.B[2], sz, ts2, fz);
      // x and z values: lane q evaluates the nodes t = q (mod 2) of both, the pair exchanges them
      float kx[NM], kz[NM], k0[W], k2[W];
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        kx[m] = es_node_q<W>(ke, 2 * m + q, sx, fx);
        kz[m] = es_node_q<W>(ke, 2 * m + q, sz, fz);
      }
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const float ox = __shfl_xor_sync(0xffffffffu, kx[m], 1), oz = __shfl_xor_sync(0xffffffffu, kz[m], 1);
        k0[2 * m] = q == 0 ? kx[m] : ox;
        k0[2 * m + 1] = q == 0 ? ox : kx[m];
        k2[2 * m] = q == 0 ? kz[m] : oz;
        k2[2 * m + 1] = q == 0 ? oz : kz[m];
      }
      float ar = 0.f, ai = 0.f;
      if (act) {
        // this lane's y nodes 2m + q
        float K1[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) K1[m] = es_node_q<W>(ke, 2 * m + q, sy, fy);
        const unsigned tb = tile_s + 8u * (unsigned)(ts0 + xsh + S0 * (ts1 + q) + S01 * ts2);
#pragma unroll
        for (int l2 = 0; l2 < W; ++l2) {
          float br = 0.f, bi = 0.f;
#pragma unroll
          for (int m = 0; m < NM; ++m) {
            const unsigned rowp = tb + 8u * (unsigned)(2 * m * S0 + l2 * S01);
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int l0 = 0; l0 < W; ++l0) {
              const float2 v = ld_shared_f2(rowp + 8u * l0);
              sr = fmaf(v.x, k0[l0], sr);
              si = fmaf(v.y, k0[l0], si);
            }
            br = fmaf(sr, K1[m], br);
            bi = fmaf(si, K1[m], bi);
          }
          ar = fmaf(br, k2[l2], ar);
          ai = fmaf(bi, k2[l2], ai);
        }
      }
      ar += __shfl_xor_sync(0xffffffffu, ar, 1);
      ai += __shfl_xor_sync(0xffffffffu, ai, 1);
      if (act && q == 0) store_once(c + r.idx, make_float2(ar, ai));
    }
    __syncthreads();
  }
}

}  // namespace nufft
