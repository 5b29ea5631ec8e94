// kernels_f64.cu -- instantiation of the FP64 forward, arrival-listing and
// adjoint kernels.  Compiled with --fmad=false: every FP64 operation rounds as
// written, as in a plain FP64 evaluation of the formulas.
#include "pair_f64.cuh"

namespace c8r {

cudaError_t launch_forward_f64(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                               const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                               cudaStream_t st) {
  FwdArgs a{tiles, n_tiles, ants, n_ant, shape.a_tile, acc, err, FwdGrid{}, M};
  if (formalism == C8R_ENDPOINT) {
    using O = OpsF64<C8R_ENDPOINT>;
    const int64_t ctas =
        forward_grid(a, shape, sm_count * forward_blocks_per_sm<O>(shape.a_tile), sizeof(Acc4D) * O::kAccRows);
    return launch_forward_ops<O>(a, ctas, st);
  }
  using O = OpsF64<C8R_ZHS>;
  const int64_t ctas =
      forward_grid(a, shape, sm_count * forward_blocks_per_sm<O>(shape.a_tile), sizeof(Acc4D) * O::kAccRows);
  return launch_forward_ops<O>(a, ctas, st);
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

cudaError_t launch_backward_f64(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count, cudaStream_t st) {
  if (formalism == C8R_ZHS) return launch_backward_ops<OpsF64<C8R_ZHS>>(a, shape, sm_count, st);
  return launch_backward_ops<OpsF64<C8R_ENDPOINT>>(a, shape, sm_count, st);
}

}  // namespace c8r
