// kernels_mixed.cu -- instantiation of the mixed-precision forward,
// arrival-listing and adjoint kernels (FP32 field arithmetic, float-float
// arrival times).
#include "pair_mixed.cuh"

namespace c8r {

cudaError_t launch_forward_mixed(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                                 const MedParams& M, void* traces, const FwdShape& shape, int sm_count, int* err,
                                 cudaStream_t st) {
  FwdArgs a{tiles, n_tiles, 0, ants, n_ant, shape.a_tile, traces, err, M};
  dim3 grid;
  forward_grid(a, shape, sm_count, grid);
  const int threads = forward_threads(shape.a_tile);
  const size_t smem = fwd_layout(C8R_MIXED, shape.a_tile, M.n_bins).total;
  const bool ex = M.kind == C8R_EXPONENTIAL;
  if (formalism == C8R_ENDPOINT) {
    if (ex) return launch_forward_ops<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>>(a, grid, threads, smem, st);
    return launch_forward_ops<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>>(a, grid, threads, smem, st);
  }
  if (ex) return launch_forward_ops<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL>>(a, grid, threads, smem, st);
  return launch_forward_ops<OpsMixed<C8R_ZHS, C8R_UNIFORM>>(a, grid, threads, smem, st);
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
