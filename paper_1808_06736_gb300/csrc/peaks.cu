// Microbenchmarks of the GPU units that bound the spread and interp kernels,
// for their rooflines: FP32 and FP64 FMA throughput, the special-function
// unit (exp2 and reciprocal square root, the ES kernel's two operations),
// and 32-bit shared-memory atomic adds with conflict-free addresses (the
// spread kernel's fixed-point accumulation).  Each kernel runs a fixed number
// of independent dependency chains per thread on a grid of resident blocks
// and writes one value per block so the work cannot be removed.
#include <cuda_runtime.h>

#include "nufft_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma(int iters, T a, T b, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == T(-1.2345)) out[blockIdx.x] = s;  // never true for the inputs used; keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_sfu(int iters, float* out) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 0.5f + 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = exp2f(-rsqrtf(v[c]));  // stays in (0.36, 1)
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s < 0.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_smem_atomic(int iters, int* out) {
  constexpr int kTile = 4096;
  __shared__ int t[kTile];
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) t[i] = 0;
  __syncthreads();
  // lane-consecutive addresses: the 32 lanes of a warp hit 32 different banks
  for (int i = 0; i < iters; ++i) atomicAdd(&t[(threadIdx.x + i * kThreads) & (kTile - 1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = t[0];
}

// milliseconds of the second of two identical launches
template <typename F>
int time_launch(cudaStream_t st, F launch, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NUFFT_ERR_CUDA;
  }
  launch();
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? NUFFT_OK : NUFFT_ERR_CUDA;
}

}  // namespace

extern "C" int nufft_measure_peaks(void* stream, double* out, int n) {
  if (!out || n < 4) return NUFFT_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NUFFT_ERR_CUDA;
  const int blocks = sms * 8;  // 2048 threads per SM
  void* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * (size_t)blocks) != cudaSuccess) return NUFFT_ERR_ALLOC;
  const double threads = (double)blocks * kThreads;
  float ms = 0.f;
  int rc = NUFFT_OK;
  const int it32 = 4096, it64 = 256, itsfu = 1024, itat = 4096;
  // FP32: 2 flops per FMA
  if ((rc = time_launch(st, [&] { k_fma<float><<<blocks, kThreads, 0, st>>>(it32, 0.999f, 1e-3f, (float*)sink); }, &ms)) !=
      NUFFT_OK)
    goto done;
  out[0] = threads * it32 * kChains * 2.0 / (ms * 1e-3) / 1e12;
  if ((rc = time_launch(st, [&] { k_fma<double><<<blocks, kThreads, 0, st>>>(it64, 0.999, 1e-3, (double*)sink); }, &ms)) !=
      NUFFT_OK)
    goto done;
  out[1] = threads * it64 * kChains * 2.0 / (ms * 1e-3) / 1e12;
  // SFU: one exp2 and one reciprocal square root per step
  if ((rc = time_launch(st, [&] { k_sfu<<<blocks, kThreads, 0, st>>>(itsfu, (float*)sink); }, &ms)) != NUFFT_OK) goto done;
  out[2] = threads * itsfu * kChains * 2.0 / (ms * 1e-3) / 1e9;
  if ((rc = time_launch(st, [&] { k_smem_atomic<<<blocks, kThreads, 0, st>>>(itat, (int*)sink); }, &ms)) != NUFFT_OK)
    goto done;
  out[3] = threads * itat / (ms * 1e-3);
done:
  cudaFree(sink);
  return rc;
}
