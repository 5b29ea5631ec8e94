// kernels_mixed.cu -- instantiation of the mixed-precision forward,
// arrival-listing and adjoint kernels (FP32 field arithmetic, float-float
// arrival times).
#include "pair_mixed.cuh"

namespace c8r {

cudaError_t launch_forward_mixed(int formalism, bool lin, const void* tiles, int64_t n_tiles, const AntRec* ants,
                                 int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count,
                                 int* err, cudaStream_t st) {
  if (lin) return launch_forward_mixed_lin(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
  return forward_mixed<false>(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
}

// accumulator [n_ant][n_bins] float4 -> traces [n_ant][3][n_bins] (added or
// stored); `replicas` copies of the accumulator, `stride` elements apart, are summed
__global__ void k_acc_to_traces_f32(const float4* acc, int64_t n_ant_bins, int n_bins, float* out, int add,
                                    int replicas, int64_t stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ant_bins) return;
  const int64_t a = i / n_bins;
  const int k = (int)(i - a * n_bins);
  float4 v = acc[i];
  for (int r = 1; r < replicas; ++r) {
    const float4 u = acc[i + r * stride];
    v.x += u.x;
    v.y += u.y;
    v.z += u.z;
  }
  float* o = out + a * 3 * n_bins + k;
  if (add) {
    o[0] += v.x;
    o[n_bins] += v.y;
    o[2 * n_bins] += v.z;
  } else {
    o[0] = v.x;
    o[n_bins] = v.y;
    o[2 * n_bins] = v.z;
  }
}

// accumulator with a row of box edges [n_ant][2][n_bins] float4 -> traces:
// out[k] = direct[k] + sum_{j <= k} edge[j], each summed over the `replicas`
// copies of the accumulator (`stride` elements apart).  One CTA per antenna
// walks the bins in chunks of its size: an inclusive scan of the chunk (FP64,
// warp shuffles, then the warp totals) plus the carry of the chunks before.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_acc_scan_to_traces(const float4* acc, int n_bins, float* out,
                                                                      int add, int replicas, int64_t stride) {
  __shared__ double warp_tot[3][kScanThreads / 32];
  const int a = blockIdx.x;
  const float4* direct = acc + (size_t)a * 2 * n_bins;
  const float4* edge = direct + n_bins;
  float* o = out + (size_t)a * 3 * n_bins;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double carry[3] = {0.0, 0.0, 0.0};
  for (int base = 0; base < n_bins; base += blockDim.x) {
    const int k = base + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (k < n_bins) {
      for (int r = 0; r < replicas; ++r) {
        const float4 e = edge[k + r * stride];
        v[0] += e.x;
        v[1] += e.y;
        v[2] += e.z;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v[c], d);
        if (lane >= d) v[c] += u;
      }
      if (lane == 31) warp_tot[c][wid] = v[c];
    }
    __syncthreads();
    double tot[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      for (int w = 0; w < nw; ++w) {
        const double t = warp_tot[c][w];
        if (w < wid) v[c] += t;
        tot[c] += t;
      }
    }
    if (k < n_bins) {
      double d[3] = {0.0, 0.0, 0.0};
      for (int q = 0; q < replicas; ++q) {
        const float4 u = direct[k + q * stride];
        d[0] += u.x;
        d[1] += u.y;
        d[2] += u.z;
      }
      const float r[3] = {(float)(d[0] + carry[0] + v[0]), (float)(d[1] + carry[1] + v[1]),
                          (float)(d[2] + carry[2] + v[2])};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (add)
          o[(size_t)c * n_bins + k] += r[c];
        else
          o[(size_t)c * n_bins + k] = r[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] += tot[c];
    __syncthreads();  // warp_tot is rewritten by the next chunk
  }
}

__global__ void k_acc_to_traces_f64(const Acc4D* acc, int64_t n_ant_bins, int n_bins, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ant_bins) return;
  const int64_t a = i / n_bins;
  const int k = (int)(i - a * n_bins);
  const Acc4D v = acc[i];
  double* o = out + a * 3 * n_bins + k;
  o[0] = v.x;
  o[n_bins] = v.y;
  o[2 * n_bins] = v.z;
}

cudaError_t launch_acc_to_traces(int precision, const void* acc, int n_ant, int n_bins, int rows, void* out, int add,
                                 cudaStream_t st, int replicas) {
  const int64_t n = (int64_t)n_ant * n_bins;
  if (n <= 0) return cudaSuccess;
  const int64_t stride = n * rows;  // accumulator elements per copy
  if (rows == 2) {
    k_acc_scan_to_traces<<<(unsigned)n_ant, kScanThreads, 0, st>>>(static_cast<const float4*>(acc), n_bins,
                                                                     static_cast<float*>(out), add, replicas, stride);
    return cudaGetLastError();
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == C8R_FP64)
    k_acc_to_traces_f64<<<blocks, 256, 0, st>>>(static_cast<const Acc4D*>(acc), n, n_bins, static_cast<double*>(out));
  else
    k_acc_to_traces_f32<<<blocks, 256, 0, st>>>(static_cast<const float4*>(acc), n, n_bins, static_cast<float*>(out),
                                                  add, replicas, stride);
  return cudaGetLastError();
}

// traces [n_ant][3][n_bins] (float or double) -> bin-major [n_ant][n_bins] of
// (x, y, z, 0), the layout the adjoint gathers one bin of from
template <typename T, typename T4>
__global__ void k_traces_to_bin_major(const T* g, int64_t n_ant_bins, int n_bins, T4* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ant_bins) return;
  const int64_t a = i / n_bins;
  const int k = (int)(i - a * n_bins);
  const T* s = g + a * 3 * n_bins + k;
  T4 v;
  v.x = s[0];
  v.y = s[n_bins];
  v.z = s[2 * (size_t)n_bins];
  v.w = T(0);
  out[i] = v;
}

cudaError_t launch_traces_to_bin_major(int precision, const void* g, int n_ant, int n_bins, void* out,
                                       cudaStream_t st) {
  const int64_t n = (int64_t)n_ant * n_bins;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == C8R_FP64)
    k_traces_to_bin_major<double, Acc4D><<<blocks, 256, 0, st>>>(static_cast<const double*>(g), n, n_bins,
                                                                 static_cast<Acc4D*>(out));
  else
    k_traces_to_bin_major<float, float4><<<blocks, 256, 0, st>>>(static_cast<const float*>(g), n, n_bins,
                                                                 static_cast<float4*>(out));
  return cudaGetLastError();
}

// running sums over the bins of a bin-major gradient, in FP64, stored as
// float-float: out[a][k] = sum_{j < k} g[a][j], k = 0 .. n_bins (one CTA per antenna)
__device__ __forceinline__ PrefixFF prefix_ff(double x, double y, double z) {
  PrefixFF p;
  p.hx = (float)x;
  p.hy = (float)y;
  p.hz = (float)z;
  p.lx = (float)(x - (double)p.hx);
  p.ly = (float)(y - (double)p.hy);
  p.lz = (float)(z - (double)p.hz);
  p.hpad = p.lpad = 0.0f;
  return p;
}
__global__ void __launch_bounds__(kScanThreads) k_bin_running_sums(const float4* g, int n_bins, PrefixFF* out) {
  __shared__ double warp_tot[3][kScanThreads / 32];
  const int a = blockIdx.x;
  const float4* row = g + (size_t)a * n_bins;
  PrefixFF* o = out + (size_t)a * (n_bins + 1);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double carry[3] = {0.0, 0.0, 0.0};
  if (threadIdx.x == 0) o[0] = prefix_ff(0.0, 0.0, 0.0);
  for (int base = 0; base < n_bins; base += blockDim.x) {
    const int k = base + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (k < n_bins) {
      const float4 e = row[k];
      v[0] = e.x;
      v[1] = e.y;
      v[2] = e.z;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v[c], d);
        if (lane >= d) v[c] += u;
      }
      if (lane == 31) warp_tot[c][wid] = v[c];
    }
    __syncthreads();
    double tot[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      for (int w = 0; w < nw; ++w) {
        const double t = warp_tot[c][w];
        if (w < wid) v[c] += t;
        tot[c] += t;
      }
    }
    if (k < n_bins) o[k + 1] = prefix_ff(carry[0] + v[0], carry[1] + v[1], carry[2] + v[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] += tot[c];
    __syncthreads();
  }
}

cudaError_t launch_bin_running_sums(const void* g, int n_ant, int n_bins, PrefixFF* out, cudaStream_t st) {
  if (n_ant <= 0 || n_bins <= 0) return cudaSuccess;
  k_bin_running_sums<<<(unsigned)n_ant, kScanThreads, 0, st>>>(static_cast<const float4*>(g), n_bins, out);
  return cudaGetLastError();
}

cudaError_t launch_arrivals_mixed(int formalism, const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                  const MedParams& M, int32_t* branch, int32_t* bin, float* frac, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n * (int64_t)n_ant + 255) / 256);
  if (M.kind == C8R_EXPONENTIAL_RAY) {
    if (formalism == C8R_ENDPOINT)
      k_arrivals<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL_RAY>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch,
                                                                                     bin, frac);
    else
      k_arrivals<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL_RAY>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin,
                                                                                frac);
    return cudaGetLastError();
  }
  if (M.kind == C8R_EXPONENTIAL_SPHERICAL) {
    if (formalism == C8R_ENDPOINT)
      k_arrivals<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL_SPHERICAL>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M,
                                                                                           branch, bin, frac);
    else
      k_arrivals<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL_SPHERICAL>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M,
                                                                                      branch, bin, frac);
    return cudaGetLastError();
  }
  const bool ex = M.kind == C8R_EXPONENTIAL;
  if (formalism == C8R_ENDPOINT) {
    if (ex)
      k_arrivals<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch,
                                                                                 bin, frac);
    else
      k_arrivals<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin,
                                                                             frac);
  } else {
    if (ex)
      k_arrivals<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin,
                                                                            frac);
    else
      k_arrivals<OpsMixed<C8R_ZHS, C8R_UNIFORM>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin,
                                                                        frac);
  }
  return cudaGetLastError();
}

cudaError_t launch_backward_mixed(int formalism, bool lin, BwdArgs& a, const FwdShape& shape, int sm_count,
                                  cudaStream_t st) {
  if (lin) return launch_backward_mixed_lin(formalism, a, shape, sm_count, st);
  return backward_mixed<false>(formalism, a, shape, sm_count, st);
}

}  // namespace c8r
