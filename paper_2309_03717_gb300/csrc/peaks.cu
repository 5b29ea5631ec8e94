// peaks.cu -- measured issue rates of the units the pair kernels are bound by:
// FP32 FMA, FP64 FMA, MUFU reciprocal square root, FP32 / FP64 shared-memory
// atomic adds to scattered bins, and global float4 vector reductions into an
// L2-resident buffer (the forward kernels' deposits).  These are the denominators of the ALU
// roofline the benchmark reports.  Every loop has a fixed trip count and every
// index is masked into its buffer.
#include <cuda_runtime.h>

#include "../../include/c8r.h"

namespace {

constexpr int kChains = 8;

__global__ void k_peak_ffma(float* out, int iters, float a, float b) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_peak_dfma(double* out, int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_peak_rsqrt(float* out, int iters) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1.0f + threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = rsqrtf(acc[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// scattered bins: a per-thread LCG picks one of 4096 words for every add
template <typename T>
__global__ void k_peak_satom(T* out, int iters) {
  __shared__ T sm[4096];
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) sm[i] = T(0);
  __syncthreads();
  unsigned h = threadIdx.x * 2654435761u + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
    h = h * 1664525u + 1013904223u;
    atomicAdd(&sm[(h >> 10) & 4095], T(1));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) out[(size_t)blockIdx.x * 4096 + i] = sm[i];
}

// global vector reductions (atomicAdd on float4, fire-and-forget) to
// scattered 16-byte elements of an L2-resident buffer of `mask + 1` elements:
// the unit the forward kernels deposit with
__global__ void k_peak_gred4(float4* buf, unsigned mask, int iters) {
  unsigned h = threadIdx.x * 2654435761u + blockIdx.x * 40503u;
  for (int i = 0; i < iters; ++i) {
    h = h * 1664525u + 1013904223u;
    atomicAdd(buf + ((h >> 7) & mask), make_float4(1.0f, 1.0f, 1.0f, 0.0f));
  }
}

}  // namespace

extern "C" int c8r_measure_peaks(int device, double* out_rates) {
  if (!out_rates) return C8R_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return C8R_EINVAL;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int threads = 256, blocks = sms * 8;
  void* buf = nullptr;
  const size_t bytes = sizeof(double) * (size_t)blocks * 4096;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) return C8R_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto launch, double ops) {
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  };
  const double lanes = (double)blocks * threads;
  out_rates[0] = timed([&] { k_peak_ffma<<<blocks, threads>>>((float*)buf, 4096, 0.999f, 1e-3f); },
                       lanes * kChains * 4096);
  out_rates[1] = timed([&] { k_peak_dfma<<<blocks, threads>>>((double*)buf, 256, 0.999, 1e-3); },
                       lanes * kChains * 256);
  out_rates[2] = timed([&] { k_peak_rsqrt<<<blocks, threads>>>((float*)buf, 1024); }, lanes * kChains * 1024);
  out_rates[3] = timed([&] { k_peak_satom<float><<<blocks, threads>>>((float*)buf, 1024); }, lanes * 1024);
  out_rates[4] = timed([&] { k_peak_satom<double><<<blocks, threads>>>((double*)buf, 512); }, lanes * 512);
  // 2^21 float4 elements = 32 MB (the buffer holds blocks x 4096 doubles >= 32 MB on 152 SMs)
  unsigned mask = (1u << 21) - 1;
  while ((size_t)(mask + 1) * sizeof(float4) > bytes) mask >>= 1;
  cudaMemset(buf, 0, bytes);
  out_rates[5] = timed([&] { k_peak_gred4<<<blocks, threads>>>((float4*)buf, mask, 256); }, lanes * 256);
  cudaError_t e = cudaDeviceSynchronize();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return e == cudaSuccess ? C8R_OK : C8R_ECUDA;
}
