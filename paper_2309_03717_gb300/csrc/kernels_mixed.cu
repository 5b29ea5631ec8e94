// kernels_mixed.cu -- instantiation of the mixed-precision forward,
// arrival-listing and adjoint kernels (FP32 field arithmetic, float-float
// arrival times).
#include "pair_mixed.cuh"

namespace c8r {

cudaError_t launch_forward_mixed(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                                 const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                                 cudaStream_t st) {
  FwdArgs a{tiles, n_tiles, ants, n_ant, shape.a_tile, acc, err, FwdGrid{}, M};
  auto go = [&](auto ops) {
    using O = decltype(ops);
    const int64_t ctas = forward_grid(a, shape, sm_count * forward_blocks_per_sm<O>(shape.a_tile), sizeof(float4));
    return launch_forward_ops<O>(a, ctas, st);
  };
  const bool ex = M.kind == C8R_EXPONENTIAL;
  if (formalism == C8R_ENDPOINT)
    return ex ? go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>{}) : go(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>{});
  return ex ? go(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL>{}) : go(OpsMixed<C8R_ZHS, C8R_UNIFORM>{});
}

// accumulator [n_ant][n_bins] float4 -> traces [n_ant][3][n_bins] (added or stored)
__global__ void k_acc_to_traces_f32(const float4* acc, int64_t n_ant_bins, int n_bins, float* out, int add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ant_bins) return;
  const int64_t a = i / n_bins;
  const int k = (int)(i - a * n_bins);
  const float4 v = acc[i];
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

cudaError_t launch_acc_to_traces(int precision, const void* acc, int n_ant, int n_bins, void* out, int add,
                                 cudaStream_t st) {
  const int64_t n = (int64_t)n_ant * n_bins;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == C8R_FP64)
    k_acc_to_traces_f64<<<blocks, 256, 0, st>>>(static_cast<const Acc4D*>(acc), n, n_bins, static_cast<double*>(out));
  else
    k_acc_to_traces_f32<<<blocks, 256, 0, st>>>(static_cast<const float4*>(acc), n, n_bins, static_cast<float*>(out),
                                                  add);
  return cudaGetLastError();
}

cudaError_t launch_arrivals_mixed(int formalism, const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                  const MedParams& M, int32_t* branch, int32_t* bin, float* frac, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n * (int64_t)n_ant + 255) / 256);
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

cudaError_t launch_backward_mixed(const BwdArgs& a, int blocks, cudaStream_t st) {
  const size_t smem = sizeof(float) * (3 * (size_t)a.n_ant + 1);
  const bool ex = a.M.kind == C8R_EXPONENTIAL;
  if (ex) {
    auto k = k_backward<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, 256, smem, st>>>(a);
  } else {
    auto k = k_backward<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace c8r
