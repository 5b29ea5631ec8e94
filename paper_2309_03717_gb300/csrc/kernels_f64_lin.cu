// kernels_f64_lin.cu -- instantiation of the FP64 forward and adjoint kernels
// with the linear (two-bin) deposit.  Compiled with --fmad=false, as the other
// FP64 unit: every FP64 operation rounds as written.
#include "pair_f64.cuh"

namespace c8r {

cudaError_t launch_forward_f64_lin(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                                   const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                                   cudaStream_t st) {
  return forward_f64<true>(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
}

cudaError_t launch_backward_f64_lin(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count,
                                    cudaStream_t st) {
  return backward_f64<true>(formalism, a, shape, sm_count, st);
}

}  // namespace c8r
