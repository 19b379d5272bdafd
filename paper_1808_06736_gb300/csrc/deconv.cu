// Diagonal correction between the fine grid and the mode array.
//
// Type 1, step 3 (Eq. (pb1), Eq. (pk)): f_k = p_{k_1} ... p_{k_d} b^_{k mod n}
//   for k in I_N -- truncation to the central modes, correction and reordering
//   in one pass (k_deconv, one thread per output mode).
// Type 2, step 1 (Sec. 3.2): b^_{k mod n} = p_k f_k for k in I_N and 0 on the
//   rest of the fine grid (a memset of the grid at full write bandwidth, then
//   k_precorrect, one thread per mode; the batched variant writes every cell
//   once, one thread per fine-grid cell).
// p_{k_i} = 2 / (w phi^(alpha_i k_i)) come from the host (Eq. (pk1)) as one
// array per dimension indexed by k_i + floor(N_i / 2).
#include "nufft_internal.cuh"

namespace nufft {
namespace {

// mode array position -> k (modeord 0: increasing k; 1: FFT order)
__device__ __forceinline__ int pos_to_k(int m, int N, int modeord) {
  if (modeord == 0) return m - N / 2;
  return (m < N - N / 2) ? m : m - N;
}
// k -> mode array position
__device__ __forceinline__ int k_to_pos(int k, int N, int modeord) {
  if (modeord == 0) return k + N / 2;
  return k >= 0 ? k : k + N;
}

// One row (fixed k_2, k_3) of the deconvolution: threads walk k_1.
template <typename T>
__device__ __forceinline__ void deconv_row(const ModeGeom& m, int m2, int m3,
                                           const typename Traits<T>::C* __restrict__ grid,
                                           typename Traits<T>::C* __restrict__ f, const T* __restrict__ p1,
                                           const T* __restrict__ p2, const T* __restrict__ p3) {
  using C = typename Traits<T>::C;
  const int k2 = pos_to_k(m2, m.N[1], m.modeord), k3 = pos_to_k(m3, m.N[2], m.modeord);
  const int l2 = k2 < 0 ? k2 + m.n[1] : k2, l3 = k3 < 0 ? k3 + m.n[2] : k3;
  const T p23 = p2[k2 + m.N[1] / 2] * p3[k3 + m.N[2] / 2];
  const C* grow = grid + ((long long)l3 * m.n[1] + l2) * (long long)m.n[0];
  C* frow = f + ((long long)m3 * m.N[1] + m2) * (long long)m.N[0];
  for (int m1 = blockIdx.x * blockDim.x + threadIdx.x; m1 < m.N[0]; m1 += gridDim.x * blockDim.x) {
    const int k1 = pos_to_k(m1, m.N[0], m.modeord);
    const int l1 = k1 < 0 ? k1 + m.n[0] : k1;
    const T p = p23 * p1[k1 + m.N[0] / 2];
    const C b = grow[l1];
    C o;
    o.x = b.x * p;
    o.y = b.y * p;
    frow[m1] = o;
  }
}

// One fine-grid row (fixed l_2, l_3) of the pre-correction: threads walk l_1.
template <typename T>
__device__ __forceinline__ void precorrect_row(const ModeGeom& m, int l2, int l3,
                                               const typename Traits<T>::C* __restrict__ f,
                                               typename Traits<T>::C* __restrict__ grid, const T* __restrict__ p1,
                                               const T* __restrict__ p2, const T* __restrict__ p3) {
  using C = typename Traits<T>::C;
  // fine-grid index l <-> mode k = l (l < N - N/2) or l - n (l >= n - N/2)
  const int k2 = l2 < m.N[1] - m.N[1] / 2 ? l2 : l2 - m.n[1];
  const int k3 = l3 < m.N[2] - m.N[2] / 2 ? l3 : l3 - m.n[2];
  const bool in23 = (k2 >= -(m.N[1] / 2)) && (k3 >= -(m.N[2] / 2));
  C* grow = grid + ((long long)l3 * m.n[1] + l2) * (long long)m.n[0];
  const C zero = {T(0), T(0)};
  if (!in23) {
    for (int l1 = blockIdx.x * blockDim.x + threadIdx.x; l1 < m.n[0]; l1 += gridDim.x * blockDim.x) grow[l1] = zero;
    return;
  }
  const T p23 = p2[k2 + m.N[1] / 2] * p3[k3 + m.N[2] / 2];
  const C* frow = f + ((long long)k_to_pos(k3, m.N[2], m.modeord) * m.N[1] + k_to_pos(k2, m.N[1], m.modeord)) *
                          (long long)m.N[0];
  for (int l1 = blockIdx.x * blockDim.x + threadIdx.x; l1 < m.n[0]; l1 += gridDim.x * blockDim.x) {
    const int k1 = l1 < m.N[0] - m.N[0] / 2 ? l1 : l1 - m.n[0];
    C o = zero;
    if (k1 >= -(m.N[0] / 2)) {
      const T p = p23 * p1[k1 + m.N[0] / 2];
      const C v = frow[k_to_pos(k1, m.N[0], m.modeord)];
      o.x = v.x * p;
      o.y = v.y * p;
    }
    grow[l1] = o;
  }
}

template <typename T>
__global__ void k_deconv(ModeGeom m, const typename Traits<T>::C* __restrict__ grid,
                         typename Traits<T>::C* __restrict__ f, const T* __restrict__ p1,
                         const T* __restrict__ p2, const T* __restrict__ p3) {
  const int nrows = m.N[1] * m.N[2];
  for (int row = blockIdx.y; row < nrows; row += gridDim.y) deconv_row<T>(m, row % m.N[1], row / m.N[1], grid, f, p1, p2, p3);
}

// Scatter of the corrected modes into a zeroed fine grid: one thread per
// mode, rows of k_1 (the grid's zero padding is a memset beforehand).
template <typename T>
__device__ __forceinline__ void scatter_row(const ModeGeom& m, int m2, int m3,
                                            const typename Traits<T>::C* __restrict__ f,
                                            typename Traits<T>::C* __restrict__ grid, const T* __restrict__ p1,
                                            const T* __restrict__ p2, const T* __restrict__ p3) {
  using C = typename Traits<T>::C;
  const int k2 = pos_to_k(m2, m.N[1], m.modeord), k3 = pos_to_k(m3, m.N[2], m.modeord);
  const int l2 = k2 < 0 ? k2 + m.n[1] : k2, l3 = k3 < 0 ? k3 + m.n[2] : k3;
  const T p23 = p2[k2 + m.N[1] / 2] * p3[k3 + m.N[2] / 2];
  C* grow = grid + ((long long)l3 * m.n[1] + l2) * (long long)m.n[0];
  const C* frow = f + ((long long)m3 * m.N[1] + m2) * (long long)m.N[0];
  for (int m1 = blockIdx.x * blockDim.x + threadIdx.x; m1 < m.N[0]; m1 += gridDim.x * blockDim.x) {
    const int k1 = pos_to_k(m1, m.N[0], m.modeord);
    const int l1 = k1 < 0 ? k1 + m.n[0] : k1;
    const T p = p23 * p1[k1 + m.N[0] / 2];
    const C v = frow[m1];
    C o;
    o.x = v.x * p;
    o.y = v.y * p;
    grow[l1] = o;
  }
}

template <typename T>
__global__ void k_precorrect(ModeGeom m, const typename Traits<T>::C* __restrict__ f,
                             typename Traits<T>::C* __restrict__ grid, const T* __restrict__ p1,
                             const T* __restrict__ p2, const T* __restrict__ p3) {
  const int nrows = m.N[1] * m.N[2];
  for (int row = blockIdx.y; row < nrows; row += gridDim.y) scatter_row<T>(m, row % m.N[1], row / m.N[1], f, grid, p1, p2, p3);
}

// Batched: rows of all transforms in one launch; a row's transform comes from
// the per-transform first-row table.
__device__ __forceinline__ ModeGeom batch_modegeom(const BatchGeom& tg, int d, int modeord) {
  ModeGeom m;
  m.d = d;
  m.modeord = modeord;
  for (int i = 0; i < 3; ++i) {
    m.N[i] = tg.N[i];
    m.n[i] = tg.n[i];
  }
  return m;
}

template <typename T>
__global__ void k_deconv_batch(int d, int modeord, long long nrows, BatchTable bt, const typename Traits<T>::C* __restrict__ grid,
                               typename Traits<T>::C* __restrict__ f, const T* __restrict__ pk) {
  for (long long row = blockIdx.y; row < nrows; row += gridDim.y) {
    const int t = batch_find(bt.mrowoff, bt.B, row);
    const BatchGeom& tg = bt.bg[t];
    const ModeGeom m = batch_modegeom(tg, d, modeord);
    const int r = (int)(row - tg.mrowoff);
    deconv_row<T>(m, r % m.N[1], r / m.N[1], grid + tg.goff, f + tg.moff, pk + tg.pkoff[0], pk + tg.pkoff[1],
                  pk + tg.pkoff[2]);
  }
}

template <typename T>
__global__ void k_precorrect_batch(int d, int modeord, long long nrows, BatchTable bt,
                                   const typename Traits<T>::C* __restrict__ f, typename Traits<T>::C* __restrict__ grid,
                                   const T* __restrict__ pk) {
  for (long long row = blockIdx.y; row < nrows; row += gridDim.y) {
    const int t = batch_find(bt.growoff, bt.B, row);
    const BatchGeom& tg = bt.bg[t];
    const ModeGeom m = batch_modegeom(tg, d, modeord);
    const int r = (int)(row - tg.growoff);
    precorrect_row<T>(m, r % m.n[1], r / m.n[1], f + tg.moff, grid + tg.goff, pk + tg.pkoff[0], pk + tg.pkoff[1],
                      pk + tg.pkoff[2]);
  }
}

// x: chunks of a row; y: rows (grid-stride), about 8 resident blocks per SM
dim3 row_grid(int len, int rows, int slabs, int threads) {
  int bx = (len + threads - 1) / threads;
  if (bx > 65535) bx = 65535;
  long long r = (long long)rows * slabs;
  int by = (int)((152LL * 8 + bx - 1) / bx);
  if (by < 1) by = 1;
  if (by > r) by = (int)r;
  if (by > 65535) by = 65535;
  return dim3(bx, by, 1);
}

template <typename T>
cudaError_t deconv_t(const ModeGeom& m, const void* grid, void* f, const void* p1, const void* p2,
                     const void* p3, cudaStream_t st) {
  k_deconv<T><<<row_grid(m.N[0], m.N[1], m.N[2], 256), 256, 0, st>>>(
      m, (const typename Traits<T>::C*)grid, (typename Traits<T>::C*)f, (const T*)p1, (const T*)p2,
      (const T*)p3);
  return cudaGetLastError();
}
template <typename T>
cudaError_t precorrect_t(const ModeGeom& m, const void* f, void* grid, const void* p1,
                         const void* p2, const void* p3, cudaStream_t st) {
  const size_t bytes = (size_t)m.n[0] * m.n[1] * m.n[2] * sizeof(typename Traits<T>::C);
  cudaError_t e = cudaMemsetAsync(grid, 0, bytes, st);
  if (e != cudaSuccess) return e;
  k_precorrect<T><<<row_grid(m.N[0], m.N[1], m.N[2], 256), 256, 0, st>>>(
      m, (const typename Traits<T>::C*)f, (typename Traits<T>::C*)grid, (const T*)p1, (const T*)p2,
      (const T*)p3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t deconv_batch_t(int d, int modeord, long long nrows, int maxlen, const BatchTable& bt, const void* grid,
                           void* f, const void* pk, cudaStream_t st) {
  int bx = (maxlen + 255) / 256;
  long long by = (152LL * 8 + bx - 1) / bx;
  if (by > nrows) by = nrows;
  if (by > 65535) by = 65535;
  if (by < 1) by = 1;
  k_deconv_batch<T><<<dim3(bx, (unsigned)by, 1), 256, 0, st>>>(d, modeord, nrows, bt, (const typename Traits<T>::C*)grid,
                                                               (typename Traits<T>::C*)f, (const T*)pk);
  return cudaGetLastError();
}
template <typename T>
cudaError_t precorrect_batch_t(int d, int modeord, long long nrows, int maxlen, const BatchTable& bt, const void* f,
                               void* grid, const void* pk, cudaStream_t st) {
  int bx = (maxlen + 255) / 256;
  long long by = (152LL * 8 + bx - 1) / bx;
  if (by > nrows) by = nrows;
  if (by > 65535) by = 65535;
  if (by < 1) by = 1;
  k_precorrect_batch<T><<<dim3(bx, (unsigned)by, 1), 256, 0, st>>>(d, modeord, nrows, bt, (const typename Traits<T>::C*)f,
                                                                   (typename Traits<T>::C*)grid, (const T*)pk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_deconv_batch(bool dbl, int d, int modeord, long long nrows, int maxlen, const BatchTable& bt,
                                const void* grid, void* f, const void* pk, cudaStream_t st) {
  return dbl ? deconv_batch_t<double>(d, modeord, nrows, maxlen, bt, grid, f, pk, st)
             : deconv_batch_t<float>(d, modeord, nrows, maxlen, bt, grid, f, pk, st);
}
cudaError_t launch_precorrect_batch(bool dbl, int d, int modeord, long long nrows, int maxlen, const BatchTable& bt,
                                    const void* f, void* grid, const void* pk, cudaStream_t st) {
  return dbl ? precorrect_batch_t<double>(d, modeord, nrows, maxlen, bt, f, grid, pk, st)
             : precorrect_batch_t<float>(d, modeord, nrows, maxlen, bt, f, grid, pk, st);
}

cudaError_t launch_deconv(bool dbl, const ModeGeom& m, const void* grid, void* f, const void* p1,
                          const void* p2, const void* p3, cudaStream_t st) {
  return dbl ? deconv_t<double>(m, grid, f, p1, p2, p3, st) : deconv_t<float>(m, grid, f, p1, p2, p3, st);
}
cudaError_t launch_precorrect(bool dbl, const ModeGeom& m, const void* f, void* grid, const void* p1,
                              const void* p2, const void* p3, cudaStream_t st) {
  return dbl ? precorrect_t<double>(m, f, grid, p1, p2, p3, st)
             : precorrect_t<float>(m, f, grid, p1, p2, p3, st);
}

}  // namespace nufft
