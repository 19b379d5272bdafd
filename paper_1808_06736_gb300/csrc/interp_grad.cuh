// Interpolation with the gradient in the point (type 2): besides
//   c_j = sum_l b_l psi(x_j - l h)                  (Eq. (interp))
// the kernels return
//   dc_j / dx_{j,d} = sum_l b_l d/dx_d psi(x_j - l h),
// the exact derivative of the type-2 approximation, with the derivative of
// the ES kernel (Eq. (ES)) phi'(z) = -beta z / sqrt(1 - z^2) phi(z).  The
// paper notes (Remark in Sec. 7) that phi' is unbounded near z = +-1; the
// factor 1 / sqrt(1 - z^2) is capped at 1e3 here, which only touches points
// within ~5e-7 w/2 cells of a stencil edge, where phi itself is e^-beta.
// With opts.kernel = 1 the plan uses the Remark's smooth variant instead,
// whose derivative is bounded (es_eval_d).
// The error of the derivative is a few times that of the values (aliased
// frequencies near n are weighted by |k + m n| instead of |k|).
//
// Same block structure as k_interp (tile + halo in shared memory, bank-aware
// point order) and as k_interp_sparse for subproblems of at most 32 points;
// the inner loops carry 1 + d complex accumulators instead of one.
#pragma once

#include "spread_interp.cuh"

namespace nufft {

template <typename T>
struct GradOutT {
  typename Traits<T>::C* dc[3];  // derivative in x_1, x_2, x_3 (M values each)
  T scale[3];                    // (2 / w) n_d / (2 pi) = -d z / d x_d
};

// k = phi(z) and dk = -phi'(z).  ES: phi' = -beta z / sqrt(1 - z^2) phi(z), the root capped
// below at 1e-3.  The smooth variant 2 e^-beta cosh(beta s), s = sqrt(1 - z^2) (Remark in
// Sec. 7): phi = a + b with a = e^{beta (s - 1)}, b = e^{-beta (s + 1)}, and
// -phi' = beta z (a - b) / s = 2 beta z e^-beta sinh(beta s) / s, bounded (-> 2 beta^2 z e^-beta
// as s -> 0); for small beta s the quotient is taken from its series 2 beta e^-beta (1 + (beta s)^2 / 6).
__device__ __forceinline__ void es_eval_d(float z, float kpar, float beta, int cosh_kernel, float& k, float& dk) {
  const float s = sqrtf(fmaxf(1.0f - z * z, 0.0f));
  if (!cosh_kernel) {
    k = exp2f(kpar * (s - 1.0f));
    dk = k * beta * z / fmaxf(s, 1e-3f);
    return;
  }
  const float a = exp2f(kpar * (s - 1.0f)), b = exp2f(-kpar * (s + 1.0f));
  k = a + b;
  const float bs = beta * s;
  const float q = bs > 0.05f ? (a - b) / s : 2.0f * beta * exp2f(-kpar) * (1.0f + bs * bs * (1.0f / 6.0f));
  dk = beta * z * q;
}
__device__ __forceinline__ void es_eval_d(double z, double kpar, double beta, int cosh_kernel, double& k,
                                          double& dk) {
  const double s = sqrt(fmax(1.0 - z * z, 0.0));
  if (!cosh_kernel) {
    k = exp(kpar * (s - 1.0));
    dk = k * beta * z / fmax(s, 1e-3);
    return;
  }
  const double a = exp(kpar * (s - 1.0)), b = exp(-kpar * (s + 1.0));
  k = a + b;
  const double bs = beta * s;
  const double q = bs > 1e-3 ? (a - b) / s : 2.0 * beta * exp(-kpar) * (1.0 + bs * bs * (1.0 / 6.0));
  dk = beta * z * q;
}

template <typename T>
__device__ __forceinline__ T beta_of(T kpar);
template <>
__device__ __forceinline__ float beta_of<float>(float kpar) {
  return kpar * 0.69314718055994530942f;  // kpar = beta log2(e) for float
}
template <>
__device__ __forceinline__ double beta_of<double>(double kpar) {
  return kpar;
}

template <typename T, int W>
__device__ __forceinline__ void point_weights_d(T v, int B, T kpar, T beta, int cosh_kernel, int& ts, T* k, T* dk) {
  const int il = min((int)v, B - 1);
  const T f = v - T(il);
  const int s = stencil_step<W>(f);
  ts = il + s;
#pragma unroll
  for (int t = 0; t < W; ++t) es_eval_d(node_z<W>(t, s, f), kpar, beta, cosh_kernel, k[t], dk[t]);
}

// float: two blocks per SM (128 registers); double: one (the 1 + d complex
// accumulators and 2w weights per dimension need the registers)
template <typename T>
struct MinBlocksGrad {
  static constexpr int value = sizeof(T) == 4 ? 2 : 1;
};

template <typename T, int D, int W>
__global__ void __launch_bounds__(256, MinBlocksGrad<T>::value) k_interp_grad(Geom g, T kpar, Sorted s,
                                                const typename Traits<T>::C* __restrict__ grid,
                                                typename Traits<T>::C* __restrict__ c, GradOutT<T> go,
                                                int* __restrict__ work) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int hist[NRES_INTERP];
  __shared__ int s_sub, s_nslots;

  const int ntile = g.ntile, maxsub = g.maxsub;
  C* tile = reinterpret_cast<C*>(smem);
  Stage<T, D> st = carve_stage<T, D>(reinterpret_cast<unsigned char*>(tile + ntile), maxsub);
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const int T0 = g.T[0], T01 = g.T[0] * g.T[1];
  const T beta = beta_of<T>(kpar);

  for (;;) {
    if (threadIdx.x == 0) s_sub = atomicAdd(work, 1);
    if (threadIdx.x < NRES_INTERP) hist[threadIdx.x] = 0;
    __syncthreads();
    const int sub = s_sub;
    if (sub >= *s.nsub) break;
    const int bin = s.sub_bin[sub], p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];

    int org[3];
    tile_origin(g, bin, org);
    const int nrows = ntile / T0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < nrows; row += nw) {
      const int t1 = row % g.T[1], t2 = row / g.T[1];
      const long long gy = wrap_idx(org[1] + t1, g.n[1]);
      const long long gz = wrap_idx(org[2] + t2, g.n[2]);
      const C* grow = grid + (gz * g.n[1] + gy) * (long long)g.n[0];
      for (int t0 = lane; t0 < T0; t0 += 32) cp_async_elem(tile + row * T0 + t0, grow + wrap_idx(org[0] + t0, g.n[0]));
    }
    cp_async_commit();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) stage_point<T, D, W, NRES_INTERP>(g, rec[p0 + q], q, st, hist);
    cp_async_wait_all();
    const int nslots = bucket_order<T, D, NRES_INTERP, false>(cnt, st, hist, &s_nslots);

    for (int sl = threadIdx.x; sl < nslots; sl += blockDim.x) {
      const int q = st.order[sl];
      if (q == kEmptySlot) continue;
      const Rec rq = rec[p0 + q];
      T k0[W], d0[W];
      int ts0, ts1 = 0, ts2 = 0;
      point_weights_d<T, W>(rq.v[0], g.B[0], kpar, beta, g.kernel, ts0, k0, d0);
      T k1[(D > 1) ? W : 1], d1[(D > 1) ? W : 1];
      T f2 = T(0);
      int st2 = 0;
      if constexpr (D > 1) {
        point_weights_d<T, W>(rq.v[1], g.B[1], kpar, beta, g.kernel, ts1, k1, d1);
      } else {
        k1[0] = T(1);
        d1[0] = T(0);
      }
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
      C a = {T(0), T(0)}, ax = {T(0), T(0)}, ay = {T(0), T(0)}, az = {T(0), T(0)};
#pragma unroll 1
      for (int l2 = 0; l2 < W2; ++l2) {
        C b = {T(0), T(0)}, bx = {T(0), T(0)}, by = {T(0), T(0)};
#pragma unroll
        for (int l1 = 0; l1 < W1; ++l1) {
          const C* rowp = tile + base + l1 * T0 + l2 * T01;
          C r = {T(0), T(0)}, rx = {T(0), T(0)};
#pragma unroll
          for (int l0 = 0; l0 < W; ++l0) {
            const C gv = rowp[l0];
            r.x = fma(gv.x, k0[l0], r.x);
            r.y = fma(gv.y, k0[l0], r.y);
            rx.x = fma(gv.x, d0[l0], rx.x);
            rx.y = fma(gv.y, d0[l0], rx.y);
          }
          b.x = fma(r.x, k1[l1], b.x);
          b.y = fma(r.y, k1[l1], b.y);
          bx.x = fma(rx.x, k1[l1], bx.x);
          bx.y = fma(rx.y, k1[l1], bx.y);
          if constexpr (D > 1) {
            by.x = fma(r.x, d1[l1], by.x);
            by.y = fma(r.y, d1[l1], by.y);
          }
        }
        T k2 = T(1), d2 = T(0);
        if constexpr (D > 2) es_eval_d(node_z<W>(l2, st2, f2), kpar, beta, g.kernel, k2, d2);
        a.x = fma(b.x, k2, a.x);
        a.y = fma(b.y, k2, a.y);
        ax.x = fma(bx.x, k2, ax.x);
        ax.y = fma(bx.y, k2, ax.y);
        ay.x = fma(by.x, k2, ay.x);
        ay.y = fma(by.y, k2, ay.y);
        az.x = fma(b.x, d2, az.x);
        az.y = fma(b.y, d2, az.y);
      }
      store_once(c + rq.idx, a);
      store_once(go.dc[0] + rq.idx, C{ax.x * go.scale[0], ax.y * go.scale[0]});
      if constexpr (D > 1) store_once(go.dc[1] + rq.idx, C{ay.x * go.scale[1], ay.y * go.scale[1]});
      if constexpr (D > 2) store_once(go.dc[2] + rq.idx, C{az.x * go.scale[2], az.y * go.scale[2]});
    }
    __syncthreads();
  }
}

// Sparse subproblems (<= 32 points): one warp each, lanes over stencil cells.
template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_interp_grad_sparse(Geom g, T kpar, Sorted s,
                                                            const typename Traits<T>::C* __restrict__ grid,
                                                            typename Traits<T>::C* __restrict__ c, GradOutT<T> go) {
  using C = typename Traits<T>::C;
  using Rec = typename Traits<T>::Rec;
  using S = Sparse<W, D>;
  __shared__ T wbuf[8][2 * S::WB];
  __shared__ C part[8][D + 1][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nt = *s.nsub, nsp = *s.nsparse;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(s.rec);
  const T beta = beta_of<T>(kpar);
  T* wb = wbuf[wid];
  T* db = wbuf[wid] + S::WB;
  for (int i = blockIdx.x * 8 + wid; i < nsp; i += gridDim.x * 8) {
    const int sub = nt + i;
    const int bin = s.sub_bin[sub], p0 = s.sub_pt0[sub], cnt = s.sub_cnt[sub];
    int org[3];
    tile_origin(g, bin, org);
    Rec r;
    r.v[0] = r.v[1] = r.v[2] = T(0);
    r.idx = 0;
    if (lane < cnt) r = rec[p0 + lane];
    for (int jb = 0; jb < cnt; jb += S::PP) {
      // weights and derivative weights of points jb .. jb+PP-1
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
          const int il = min((int)v, g.B[dd] - 1);
          const T f = v - T(il);
          es_eval_d(node_z<W>(t, stencil_step<W>(f), f), kpar, beta, g.kernel, wb[e], db[e]);
        }
      }
      __syncwarp();
      const int p = S::PP > 1 ? lane / S::CP : 0;
      const int src = (jb + p) & 31;
      T v[3];
      v[0] = __shfl_sync(0xffffffffu, r.v[0], src);
      v[1] = __shfl_sync(0xffffffffu, r.v[1], src);
      v[2] = __shfl_sync(0xffffffffu, r.v[2], src);
      C acc[D + 1];
#pragma unroll
      for (int k = 0; k <= D; ++k) acc[k] = C{T(0), T(0)};
      const bool live = S::PP > 1 ? (p < S::PP && jb + p < cnt) : true;
      if (live) {
        for (int cell = (S::PP > 1 ? lane - p * S::CP : lane); cell < S::CP; cell += (S::PP > 1 ? S::CP : 32)) {
          const int ii[3] = {cell % W, (cell / W) % W, cell / (W * W)};
          long long idx = 0, stride = 1;
          T wv[3], dv[3];
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const int il = min((int)v[d], g.B[d] - 1);
            const int a = org[d] + il + stencil_step<W>(v[d] - T(il));
            idx += (long long)wrap_idx(a + ii[d], g.n[d]) * stride;
            stride *= g.n[d];
            wv[d] = wb[p * W * D + d * W + ii[d]];
            dv[d] = db[p * W * D + d * W + ii[d]];
          }
          const C gv = __ldg(grid + idx);
          T wt = T(1);
#pragma unroll
          for (int d = 0; d < D; ++d) wt *= wv[d];
          acc[0].x = fma(gv.x, wt, acc[0].x);
          acc[0].y = fma(gv.y, wt, acc[0].y);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            T wd = dv[d];
#pragma unroll
            for (int e = 0; e < D; ++e)
              if (e != d) wd *= wv[e];
            acc[d + 1].x = fma(gv.x, wd, acc[d + 1].x);
            acc[d + 1].y = fma(gv.y, wd, acc[d + 1].y);
          }
          if (S::PP > 1) break;  // one cell per lane
        }
      }
      if (S::PP > 1) {
#pragma unroll
        for (int k = 0; k <= D; ++k) part[wid][k][lane] = acc[k];
        const int dst = __shfl_sync(0xffffffffu, r.idx, (jb + lane) & 31);
        __syncwarp();
        if (lane < S::PP && jb + lane < cnt) {
#pragma unroll
          for (int k = 0; k <= D; ++k) {
            C sum = {T(0), T(0)};
            for (int q = 0; q < S::CP; ++q) {
              sum.x += part[wid][k][lane * S::CP + q].x;
              sum.y += part[wid][k][lane * S::CP + q].y;
            }
            if (k == 0) store_once(c + dst, sum);
            else store_once(go.dc[k - 1] + dst, C{sum.x * go.scale[k - 1], sum.y * go.scale[k - 1]});
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k <= D; ++k)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, o);
            acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, o);
          }
        const int dst = __shfl_sync(0xffffffffu, r.idx, jb);
        if (lane == 0) {
          store_once(c + dst, acc[0]);
#pragma unroll
          for (int k = 1; k <= D; ++k)
            store_once(go.dc[k - 1] + dst, C{acc[k].x * go.scale[k - 1], acc[k].y * go.scale[k - 1]});
        }
      }
      __syncwarp();
    }
  }
}

template <typename T, int D, int W>
cudaError_t run_interp_grad(const Geom& g, double beta, const Sorted& s, const void* grid, void* c,
                            const GradOut& gov, int* work, const LaunchCfg& cfg, cudaStream_t st, bool configure_only) {
  auto kern = k_interp_grad<T, D, W>;
  if (configure_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, cfg.threads, cfg.smem);
    if (e != cudaSuccess) return e;
    const_cast<LaunchCfg&>(cfg).blocks = nb;
    return cudaSuccess;
  }
  using C = typename Traits<T>::C;
  GradOutT<T> go;
  for (int i = 0; i < 3; ++i) {
    go.dc[i] = reinterpret_cast<C*>(gov.dc[i]);
    go.scale[i] = (T)gov.scale[i];
  }
  kern<<<cfg.blocks, cfg.threads, cfg.smem, st>>>(g, kernel_param<T>(beta), s, reinterpret_cast<const C*>(grid),
                                                 reinterpret_cast<C*>(c), go, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.sparse_max <= 0) return e;
  k_interp_grad_sparse<T, D, W><<<2 * cfg.blocks, 256, 0, st>>>(g, kernel_param<T>(beta), s,
                                                                reinterpret_cast<const C*>(grid),
                                                                reinterpret_cast<C*>(c), go);
  return cudaGetLastError();
}

#define NUFFT_GRAD_W_CASES(T, D)                                                          \
  switch (g.w) {                                                                          \
    case 2: return run_interp_grad<T, D, 2>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 3: return run_interp_grad<T, D, 3>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 4: return run_interp_grad<T, D, 4>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 5: return run_interp_grad<T, D, 5>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 6: return run_interp_grad<T, D, 6>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 7: return run_interp_grad<T, D, 7>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 8: return run_interp_grad<T, D, 8>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 9: return run_interp_grad<T, D, 9>(g, beta, s, grid, c, go, work, cfg, st, conf);    \
    case 10: return run_interp_grad<T, D, 10>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 11: return run_interp_grad<T, D, 11>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 12: return run_interp_grad<T, D, 12>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 13: return run_interp_grad<T, D, 13>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 14: return run_interp_grad<T, D, 14>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 15: return run_interp_grad<T, D, 15>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    case 16: return run_interp_grad<T, D, 16>(g, beta, s, grid, c, go, work, cfg, st, conf);  \
    default: return cudaErrorInvalidValue;                                                \
  }

#define NUFFT_DEFINE_GRAD(P, T, D)                                                                          \
  cudaError_t interp_grad_##P##_d##D(const Geom& g, double beta, const Sorted& s, const void* grid, void* c, \
                                     const GradOut& go, int* work, const LaunchCfg& cfg, cudaStream_t st,     \
                                     bool conf) {                                                             \
    NUFFT_GRAD_W_CASES(T, D)                                                                                  \
  }

}  // namespace nufft
