// kernels_mixed_lin.cu -- instantiation of the mixed-precision forward and
// adjoint kernels with the linear (two-bin) deposit, in a translation unit of
// its own so that it compiles in parallel with the one-bin kernels.
#include "pair_mixed.cuh"

namespace c8r {

cudaError_t launch_forward_mixed_lin(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants,
                                     int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count,
                                     int* err, cudaStream_t st) {
  return forward_mixed<true>(formalism, tiles, n_tiles, ants, n_ant, M, acc, shape, sm_count, err, st);
}

cudaError_t launch_backward_mixed_lin(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count,
                                      cudaStream_t st) {
  return backward_mixed<true>(formalism, a, shape, sm_count, st);
}

}  // namespace c8r
