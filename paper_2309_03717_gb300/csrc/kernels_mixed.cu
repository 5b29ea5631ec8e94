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
// walks the bins in chunks of kScanT x kScanE, each thread kScanE consecutive
// bins: the thread's total of the edges, an exclusive scan of the totals over
// the CTA, then the running sum over the thread's bins from there, plus the
// carry of the chunks before.  All sums in float-float on the FP32 pipe
// (~2^-44 relative after 2^24 bins, far below the FP32 output); FP64 runs at
// 1/64 of the FP32 rate on this part.
constexpr int kScanT = 256;         // threads of the float-float scans
constexpr int kScanE = 8;           // consecutive bins per thread and chunk

__device__ __forceinline__ ff ff_sum(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  ff r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  e = __fadd_rn(e, a.l);
  ff r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

// exclusive prefix over the CTA (kScanT threads, all of them calling) of each
// thread's three float-float values v[], in excl[], and the CTA total, in
// tot[]: warp shuffles, then the totals of the warps before (warp_tot is
// written and read here; the caller synchronises before reusing it)
__device__ __forceinline__ void cta_exclusive_scan_ff3(const ff v[3], ff excl[3], ff tot[3],
                                                       ff (*warp_tot)[kScanT / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  ff inc[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const ff u{__shfl_up_sync(0xffffffffu, inc[c].h, d), __shfl_up_sync(0xffffffffu, inc[c].l, d)};
      if (lane >= d) inc[c] = ff_sum(inc[c], u);
    }
    if (lane == 31) warp_tot[c][wid] = inc[c];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ff before{0.0f, 0.0f};
    tot[c] = ff{0.0f, 0.0f};
#pragma unroll
    for (int w = 0; w < kScanT / 32; ++w) {
      const ff t = warp_tot[c][w];
      if (w < wid) before = ff_sum(before, t);
      tot[c] = ff_sum(tot[c], t);
    }
    ff lanes{__shfl_up_sync(0xffffffffu, inc[c].h, 1), __shfl_up_sync(0xffffffffu, inc[c].l, 1)};
    if (lane == 0) lanes = ff{0.0f, 0.0f};
    excl[c] = ff_sum(before, lanes);
  }
}

// the edges of bin k summed over the accumulator copies, added to run[]
__device__ __forceinline__ void add_edges(const float4* edge, int64_t k, int replicas, int64_t stride, ff run[3]) {
  for (int r = 0; r < replicas; ++r) {
    const float4 e = edge[k + r * stride];
    run[0] = ff_add_f(run[0], e.x);
    run[1] = ff_add_f(run[1], e.y);
    run[2] = ff_add_f(run[2], e.z);
  }
}

__global__ void __launch_bounds__(kScanT) k_acc_scan_to_traces(const float4* acc, int n_bins, float* out, int add,
                                                               int replicas, int64_t stride) {
  __shared__ ff warp_tot[3][kScanT / 32];
  const int a = blockIdx.x;
  const float4* direct = acc + (size_t)a * 2 * n_bins;
  const float4* edge = direct + n_bins;
  float* o = out + (size_t)a * 3 * n_bins;
  ff carry[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int base = 0; base < n_bins; base += kScanT * kScanE) {
    const int k0 = base + threadIdx.x * kScanE;
    const int k1 = min(k0 + kScanE, n_bins);
    // this thread's total of the edges, and the edges before its bins
    ff v[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int k = k0; k < k1; ++k) add_edges(edge, k, replicas, stride, v);
    ff excl[3], tot[3], run[3];
    cta_exclusive_scan_ff3(v, excl, tot, warp_tot);
#pragma unroll
    for (int c = 0; c < 3; ++c) run[c] = ff_sum(carry[c], excl[c]);
    // the running sum over this thread's bins, plus the direct deposits
    for (int k = k0; k < k1; ++k) {
      add_edges(edge, k, replicas, stride, run);
      ff d[3] = {run[0], run[1], run[2]};
      for (int r = 0; r < replicas; ++r) {
        const float4 u = direct[k + r * stride];
        d[0] = ff_add_f(d[0], u.x);
        d[1] = ff_add_f(d[1], u.y);
        d[2] = ff_add_f(d[2], u.z);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float r = __fadd_rn(d[c].h, d[c].l);
        if (add)
          o[(size_t)c * n_bins + k] += r;
        else
          o[(size_t)c * n_bins + k] = r;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] = ff_sum(carry[c], tot[c]);
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
    k_acc_scan_to_traces<<<(unsigned)n_ant, kScanT, 0, st>>>(static_cast<const float4*>(acc), n_bins,
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

// running sums over the bins of a bin-major gradient, stored as float-float:
// out[a][k] = sum_{j < k} g[a][j], k = 0 .. n_bins (one CTA per antenna), laid
// out like the trace scan (kScanE consecutive bins per thread, a CTA-wide
// exclusive scan of the threads' totals, a carry over chunks), in float-float
// on the FP32 pipe: after k additions a sum is off by at most ~2k u^2 of the
// largest partial sum (u = 2^-24), ~1e-11 of it at 2048 bins, against the
// adjoint's need of ~1e-7 of the sums it forms from two of them
__device__ __forceinline__ PrefixFF prefix_ff(const ff s[3]) {
  PrefixFF p;
  p.hx = s[0].h;
  p.hy = s[1].h;
  p.hz = s[2].h;
  p.lx = s[0].l;
  p.ly = s[1].l;
  p.lz = s[2].l;
  p.hpad = p.lpad = 0.0f;
  return p;
}
__global__ void __launch_bounds__(kScanT) k_bin_running_sums(const float4* g, int n_bins, PrefixFF* out) {
  __shared__ ff warp_tot[3][kScanT / 32];
  const int a = blockIdx.x;
  const float4* row = g + (size_t)a * n_bins;
  PrefixFF* o = out + (size_t)a * (n_bins + 1);
  ff carry[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  if (threadIdx.x == 0) o[0] = prefix_ff(carry);
  for (int base = 0; base < n_bins; base += kScanT * kScanE) {
    const int k0 = base + threadIdx.x * kScanE;
    const int k1 = min(k0 + kScanE, n_bins);
    ff v[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int k = k0; k < k1; ++k) {
      const float4 e = row[k];
      v[0] = ff_add_f(v[0], e.x);
      v[1] = ff_add_f(v[1], e.y);
      v[2] = ff_add_f(v[2], e.z);
    }
    ff excl[3], tot[3], run[3];
    cta_exclusive_scan_ff3(v, excl, tot, warp_tot);
#pragma unroll
    for (int c = 0; c < 3; ++c) run[c] = ff_sum(carry[c], excl[c]);
    for (int k = k0; k < k1; ++k) {
      const float4 e = row[k];
      run[0] = ff_add_f(run[0], e.x);
      run[1] = ff_add_f(run[1], e.y);
      run[2] = ff_add_f(run[2], e.z);
      o[k + 1] = prefix_ff(run);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) carry[c] = ff_sum(carry[c], tot[c]);
    __syncthreads();  // warp_tot is rewritten by the next chunk
  }
}

cudaError_t launch_bin_running_sums(const void* g, int n_ant, int n_bins, PrefixFF* out, cudaStream_t st) {
  if (n_ant <= 0 || n_bins <= 0) return cudaSuccess;
  k_bin_running_sums<<<(unsigned)n_ant, kScanT, 0, st>>>(static_cast<const float4*>(g), n_bins, out);
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
