// kernels_f64.cu -- instantiation of the FP64 forward, arrival-listing and
// adjoint kernels.  Compiled with --fmad=false: every FP64 operation rounds as
// written, as in a plain FP64 evaluation of the formulas.
#include "pair_f64.cuh"

namespace c8r {

cudaError_t launch_forward_f64(int formalism, bool lin, const void* tiles, int64_t n_tiles, const AntRec* ants,
                               int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                               cudaStream_t st) {
  if (lin) return launch_forward_f64_lin(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
  return forward_f64<false>(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
}

cudaError_t launch_arrivals_f64(int formalism, const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                const MedParams& M, int32_t* branch, int32_t* bin, float* frac, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n * (int64_t)n_ant + 255) / 256);
  if (formalism == C8R_ENDPOINT)
    k_arrivals<OpsF64<C8R_ENDPOINT>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin, frac);
  else
    k_arrivals<OpsF64<C8R_ZHS>><<<blocks, 256, 0, st>>>(tiles, n, ants, n_ant, M, branch, bin, frac);
  return cudaGetLastError();
}

cudaError_t launch_backward_f64(int formalism, bool lin, BwdArgs& a, const FwdShape& shape, int sm_count,
                                cudaStream_t st) {
  if (lin) return launch_backward_f64_lin(formalism, a, shape, sm_count, st);
  return backward_f64<false>(formalism, a, shape, sm_count, st);
}

}  // namespace c8r
