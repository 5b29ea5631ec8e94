// c8r_internal.h -- host-side declarations shared by the libc8r translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/c8r.h"
#include "c8r_device.cuh"

namespace c8r {

// launch shape of the forward kernels
struct FwdShape {
  int a_tile;  // antennas per CTA: each thread holds one staged track and loops over them
  int waves;   // target number of waves (all CTAs resident at once) per launch
  int replicas = 1;  // copies of the accumulator (acc_replicas)
};

// SoA track pointers of the caller, already offset to a chunk
struct TrackPtrs {
  int dtype;
  const void* f[12];
};

size_t tile_bytes(int precision);
// bytes of one accumulator element (one bin of one antenna: x, y, z, pad)
inline size_t acc_elem_bytes(int precision) { return precision == C8R_FP64 ? 32 : 16; }
// accumulator rows per antenna: the mixed ZHS path adds a row of box edges
inline int acc_rows(int precision, int formalism) { return precision == C8R_MIXED && formalism == C8R_ZHS ? 2 : 1; }
// copies of the accumulator the forward kernel spreads its reductions over (CTA
// range r adds into copy r % replicas; the fetch sums them).  Most reductions go
// into the few bins per antenna that the pulse arrives in, and with many CTAs
// on one antenna tile at a time those bins' L2 slices become the bottleneck.
// The copies split each hot bin over several addresses.  Measured (pair-kernel
// time): ZHS on a 160-antenna array (5 antenna tiles) 41 -> 34 ms with 2
// copies, no better with 4; Endpoint there unchanged (issue-bound) and 2 %
// slower with the linear deposit; on a 64-antenna array (2 tiles) Endpoint
// 1.18 -> 0.97 ms with 2 (0.95 with 8), ZHS 1.10 -> 0.73 ms with 4, and with
// the linear deposit Endpoint 2.68 -> 1.70 ms with 2.  So the count follows the
// CTAs per antenna tile (resident CTAs / antenna tiles): about one copy per 200
// for Endpoint and per 100 for ZHS, rounded down to a power of two, at most 8,
// and only as many as fit the 48 MB of L2 the forward grid budgets for
// accumulator rows (more would split the antenna tiles into more L2 blocks,
// with more CTAs per tile again).
// the batched launch: its many showers' antenna tiles spread the CTAs, so 2
// copies for ZHS and 1 for Endpoint
inline int acc_replicas(int precision, int formalism) { return acc_rows(precision, formalism) == 2 ? 2 : 1; }
// a context: from its antenna count, bins and antenna tile
inline int acc_replicas(int precision, int formalism, int n_ant, int n_bins, int a_tile, int sm_count) {
  if (precision != C8R_MIXED) return 1;
  const int64_t ant_tiles = (n_ant + a_tile - 1) / a_tile;
  const int64_t resident = (int64_t)sm_count * (formalism == C8R_ZHS ? 7 : 6);
  const int64_t per_tile = resident / (ant_tiles > 0 ? ant_tiles : 1);
  const int64_t per_copy = formalism == C8R_ZHS ? 100 : 200;
  int64_t want = (per_tile + per_copy - 1) / per_copy;
  const size_t one = (size_t)n_ant * n_bins * 16 * acc_rows(precision, formalism);
  const int64_t fit = (int64_t)(((size_t)48 << 20) / (one > 0 ? one : 1));
  if (want > fit) want = fit;
  if (want > 8) want = 8;
  int r = 1;
  while (r * 2 <= want) r *= 2;  // a power of two
  return r;
}
// accumulator [replicas][n_ant][rows][n_bins] -> traces [n_ant][3][n_bins]: the
// copies are summed; with rows == 2 the second row (box edges) is integrated over
// the bins and added; add != 0 adds into out.  FP32 only for add or replicas > 1
cudaError_t launch_acc_to_traces(int precision, const void* acc, int n_ant, int n_bins, int rows, void* out, int add,
                                 cudaStream_t st, int replicas = 1);

// dL/dtraces [n_ant][3][n_bins] -> bin-major [n_ant][n_bins] accumulator elements
cudaError_t launch_traces_to_bin_major(int precision, const void* g, int n_ant, int n_bins, void* out,
                                       cudaStream_t st);

// ingest: filter + derived per-track quantities into tiles; counts kept tracks
// into *kept unless kept is NULL, and (mixed precision, form not NULL) adds the
// kept tracks to form[0] and those whose start point sees the antenna array's
// centroid (M.cen_*) from above within 45 degrees to form[1]
cudaError_t launch_ingest(int precision, const TrackPtrs& t, int64_t n, void* tiles, const MedParams& M,
                          unsigned long long* kept, cudaStream_t st, unsigned long long* form = nullptr);

struct BwdArgs;

// per-precision launchers (kernels_f64.cu / kernels_mixed.cu); `lin` selects
// the linear (two-bin) deposit, whose kernels live in kernels_*_lin.cu
cudaError_t launch_forward_f64(int formalism, bool lin, const void* tiles, int64_t n_tiles, const AntRec* ants,
                               int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                               cudaStream_t st);
cudaError_t launch_forward_mixed(int formalism, bool lin, const void* tiles, int64_t n_tiles, const AntRec* ants,
                                 int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count,
                                 int* err, cudaStream_t st);
cudaError_t launch_forward_f64_lin(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                                   const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                                   cudaStream_t st);
cudaError_t launch_forward_mixed_lin(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants,
                                     int n_ant, const MedParams& M, void* acc, const FwdShape& shape, int sm_count,
                                     int* err, cudaStream_t st);
cudaError_t launch_arrivals_f64(int formalism, const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                const MedParams& M, int32_t* branch, int32_t* bin, float* frac, cudaStream_t st);
cudaError_t launch_arrivals_mixed(int formalism, const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                  const MedParams& M, int32_t* branch, int32_t* bin, float* frac, cudaStream_t st);
cudaError_t launch_backward_f64(int formalism, bool lin, BwdArgs& a, const FwdShape& shape, int sm_count,
                                cudaStream_t st);
cudaError_t launch_backward_mixed(int formalism, bool lin, BwdArgs& a, const FwdShape& shape, int sm_count,
                                  cudaStream_t st);
cudaError_t launch_backward_f64_lin(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count, cudaStream_t st);
cudaError_t launch_backward_mixed_lin(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count,
                                      cudaStream_t st);
// one running sum of the gradient over the bins, (x, y, z) as float-float
// (h + l): formed in FP64, stored as two FP32 parts so that the mixed adjoint
// takes the sum over a run of bins as (h1 - h0) + (l1 - l0) on the FP32 pipe
struct alignas(32) PrefixFF {
  float hx, hy, hz, hpad;
  float lx, ly, lz, lpad;
};
// running sums over the bins of a bin-major FP32 gradient [n_ant][n_bins]
// (mixed path): out [n_ant][n_bins + 1], entry k = the sum over bins < k
cudaError_t launch_bin_running_sums(const void* g, int n_ant, int n_bins, PrefixFF* out, cudaStream_t st);

// process-wide test knobs (c8r_set_wait_limit, c8r_inject_alloc_failures)
uint32_t current_wait_limit();
// cudaMalloc, unless an injected allocation failure is pending (then it
// returns cudaErrorMemoryAllocation without allocating)
cudaError_t dev_malloc(void** p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

// helpers shared by the context and the batch runner
void fill_medium(MedParams& M, int kind, double n_or_N0, double H, int n_bins, double dt_ns, double eps_C,
                 double earth_radius = 0.0);
void fill_antenna(AntRec& r, double x, double y, double z, double t_ref_ns, const MedParams& M);
// the antenna array's centroid (MedParams::cen_*), which the ingest's votes for
// the arrival form of the one-bin Endpoint kernels refer to
void set_form_centroid(MedParams& M, const double* pos_xyz, int n_ant);
// MedParams::flat and its altitude terms: set when the medium is the flat
// exponential atmosphere and every antenna has the same z (exactly)
void set_flat_array(MedParams& M, const double* pos_xyz, int n_ant);

}  // namespace c8r
