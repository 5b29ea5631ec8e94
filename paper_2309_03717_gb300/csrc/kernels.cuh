// kernels.cuh -- CTA-level loops shared by the FP64 and the mixed-precision
// translation units.  Each TU supplies an `Ops` class with the per-pair
// arithmetic (load/live/pair_main/pair_deferred, adj) and instantiates the
// kernels below.
//
// Forward (§2 flow: each track goes to every antenna of the collection): a CTA
// owns a tile of antennas and a contiguous range of derived-track tiles.  It
// streams its range through a two-slot ring of shared-memory tiles filled by
// TMA bulk copies (cp.async.bulk + mbarrier, bounded waits).  For every staged
// tile each thread loads one track into registers and evaluates it against
// every antenna of the tile;
// pairs whose arithmetic takes a rare branch (Endpoint near the Cherenkov
// angle) are queued in shared memory and evaluated together after the main
// pass, so that both branches run in full warps.  Each deposit goes into the
// L2-resident accumulator [antenna][bin][x, y, z, 0] with one native vector
// reduction (atomicAdd on float4; three FP64 reductions in the FP64 path); a
// constant run of bins (ZHS) is added as its two edges into a second row that
// the fetch integrates.  The mixed accumulator has 1 to 8 copies (CTA range r
// adds into copy r % copies, acc_replicas) that the fetch sums.  Shared-memory
// float atomics are not used: they stall the issuing warp, while the global
// reductions are fire-and-forget.
#pragma once

#include <type_traits>

#include "c8r_internal.h"

namespace c8r {

constexpr int kMaxATile = 32;
constexpr int kFwdMaxThreads = 512;

// what the main pass of a pair leaves for after it (Ops::pair_main): nothing,
// the whole pair (Endpoint near the Cherenkov angle: Ops::pair_deferred), or
// one or both endpoints whose bin the FP32 arrival left open
// (Ops::end_deferred)
enum : int { kDeferNone = 0, kDeferPair = 1, kDeferEnd0 = 4, kDeferEnd1 = 8 };
// entries of each shared-memory list of the third sweep (second endpoints of
// pairs with both endpoints set aside; near-Cherenkov pairs the FP32 check did
// not settle as zero), forward and adjoint kernels; more such entries in a tile
// are taken from the queue
constexpr int kFwdListCap = 128;
constexpr int kBwdListCap = 64;

// dynamic shared memory of the forward kernels: two staged track tiles, their
// mbarriers, the antenna tile and (defer) the queue of set-aside pairs, one
// 16-bit entry per (track, antenna) pair of a tile (q_cap entries): whole pairs
// fill it from the front, pairs with set-aside endpoints from the back
struct FwdLayout {
  size_t stage_bytes, bar_off, ant_off, q_off, total;
  int q_cap;
};
__host__ __device__ inline FwdLayout fwd_layout(int precision, int a_tile, bool defer) {
  FwdLayout L;
  L.stage_bytes = precision == C8R_FP64 ? kTileBytesF64 : kTileBytesMixed;
  L.bar_off = 2 * L.stage_bytes;
  L.ant_off = L.bar_off + 128;
  L.q_off = L.ant_off + (size_t)a_tile * sizeof(AntRec);
  L.q_cap = defer ? kTileT * a_tile : 0;
  L.total = L.q_off + (size_t)L.q_cap * sizeof(uint16_t);
  return L;
}

// accumulator element: one bin of one antenna, components x, y, z (+ padding)
struct alignas(32) Acc4D {
  double x, y, z, w;
};
template <typename T>
struct AccOf;
template <>
struct AccOf<float> {
  using type = float4;
};
template <>
struct AccOf<double> {
  using type = Acc4D;
};

// CTA -> (antenna tile, track range).  Antenna tiles are grouped into blocks
// whose accumulators fit comfortably in L2; inside a block the antenna tile
// varies fastest, so CTAs resident together read the same track range (L2
// reuse of the track tiles) and add into a bounded set of accumulator rows.
struct FwdGrid {
  int ant_tiles;        // total antenna tiles
  int tiles_per_block;  // antenna tiles per L2 block
  int64_t ranges;       // track ranges
  int64_t tiles_per_range;
  __host__ __device__ inline void decode(int64_t cta, int& ant_tile, int64_t& range) const {
    const int64_t per_block = (int64_t)tiles_per_block * ranges;
    const int64_t b = cta / per_block;
    const int64_t rem = cta - b * per_block;
    const int nb = min(tiles_per_block, ant_tiles - (int)b * tiles_per_block);
    range = rem / nb;
    ant_tile = (int)(b * tiles_per_block + rem % nb);
  }
};

struct FwdArgs {
  const void* tiles;
  int64_t n_tiles;
  const AntRec* ants;
  int n_ant;
  int a_tile;
  void* acc;  // [n_ant][n_bins] accumulator elements
  int* err;
  FwdGrid g;
  MedParams M;
  int replicas = 1;            // accumulator copies; CTA range r adds into copy r % replicas
  int64_t replica_stride = 0;  // accumulator elements per copy
};

struct BwdArgs {
  const void* tiles;
  int64_t n;          // tracks
  int64_t n_tiles;    // derived tiles holding them
  const AntRec* ants;
  int n_ant;
  int a_tile;
  const void* G;      // dL/dtraces, bin-major [n_ant][n_bins] of (x, y, z, 0) accumulator elements
  const PrefixFF* Gp;  // mixed ZHS: running sums of G over the bins, [n_ant][n_bins + 1] (entry k: bins < k)
  c8r_track_grads out;
  double* ant_grad;   // [n_ant][3]
  double* dN0;
  int* err;
  FwdGrid g;          // set by the launcher
  MedParams M;
};

// deposit of a 3-vector into bin k of one antenna's shared trace
template <typename T>
__device__ __forceinline__ void dep3(T* tr, int n_bins, int k, T vx, T vy, T vz) {
  atomicAdd(tr + k, vx);
  atomicAdd(tr + n_bins + k, vy);
  atomicAdd(tr + 2 * n_bins + k, vz);
}

// Sinks: the pair functions report deposits through dep() and their branch and
// arrival positions through rec(); the forward kernel adds deposits into the
// global accumulator, the validation listing records bins.  Both run the same
// arithmetic.
template <typename T>
struct GlobalSink;
template <>
struct GlobalSink<float> {
  // accumulator of one antenna: n bins, followed (formalisms that add boxes) by
  // n bins of box edges, which the fetch integrates over the bins
  float4* row;
  int n;
  __device__ __forceinline__ void dep(int k, float x, float y, float z) {
    atomicAdd(row + k, make_float4(x, y, z, 0.0f));
  }
  // the same (x, y, z) into every bin k0..k1 (0 <= k0 <= k1 < n): +v at the
  // box's first bin and -v after its last in the edge row, so a box of any
  // length costs at most two reductions
  __device__ __forceinline__ void dep_box(int k0, int k1, float x, float y, float z) {
    if (k1 - k0 < 2) {
      dep(k0, x, y, z);
      if (k1 > k0) dep(k1, x, y, z);
      return;
    }
    atomicAdd(row + n + k0, make_float4(x, y, z, 0.0f));
    if (k1 + 1 < n) atomicAdd(row + n + k1 + 1, make_float4(-x, -y, -z, 0.0f));
  }
  __device__ __forceinline__ void rec(int, ff, ff) {}
  __device__ __forceinline__ void rec(int, double, double) {}
};
template <>
struct GlobalSink<double> {
  Acc4D* row;
  int n;
  __device__ __forceinline__ void dep(int k, double x, double y, double z) {
    atomicAdd(&row[k].x, x);
    atomicAdd(&row[k].y, y);
    atomicAdd(&row[k].z, z);
  }
  __device__ __forceinline__ void rec(int, ff, ff) {}
  __device__ __forceinline__ void rec(int, double, double) {}
};

struct ArrivalSink {
  int32_t* branch;
  int32_t* bin;
  float* frac;
  int64_t j;
  int N;
  __device__ __forceinline__ void dep(int, float, float, float) {}
  __device__ __forceinline__ void dep(int, double, double, double) {}
  __device__ __forceinline__ void dep_box(int, int, float, float, float) {}
  __device__ __forceinline__ void rec(int b, ff ua, ff ub) {
    float fa, fb;
    int ka = bin_raw(ua, N, fa), kb = bin_raw(ub, N, fb);
    branch[j] = b;
    bin[2 * j] = ka;
    bin[2 * j + 1] = kb;
    frac[2 * j] = fa;
    frac[2 * j + 1] = fb;
  }
  __device__ __forceinline__ void rec(int b, double ua, double ub) {
    double ka = floor(ua), kb = floor(ub);
    branch[j] = b;
    bin[2 * j] = ka < 0.0 ? -1 : (ka >= (double)N ? N : (int)ka);
    bin[2 * j + 1] = kb < 0.0 ? -1 : (kb >= (double)N ? N : (int)kb);
    frac[2 * j] = (float)(ua - ka);
    frac[2 * j + 1] = (float)(ub - kb);
  }
};

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Stream derived-track tiles [t_begin, t_end) through the two-slot TMA ring and
// evaluate every (track, antenna) pair of the n_here antennas in ant_s, adding
// deposits into the accumulator rows starting at acc_row0 (the row of ant_s[0]).
// `it` counts the tiles this CTA has consumed so far (it sets the slot and the
// mbarrier phase) and is advanced.  Returns false if a bounded wait gave up; the
// CTA then has no copy in flight and must stop.
template <class Ops>
__device__ bool stream_range(unsigned char* smem, const FwdLayout& L, uint64_t* bar, const AntRec* ant_s,
                             typename AccOf<typename Ops::acc_t>::type* acc_row0, int n_here,
                             const unsigned char* src, int64_t t_begin, int64_t t_end, int64_t& it,
                             const MedParams& M) {
  using acc_t = typename Ops::acc_t;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int N = M.n_bins;
  const size_t row_stride = (size_t)N * Ops::kAccRows;
  const uint32_t bytes = (uint32_t)L.stage_bytes;
  // pairs the main pass sets aside (Ops::kDefers): entry = track lane |
  // antenna << 7 | set-aside endpoints << 10 (kDeferEnd0/1 bits); whole pairs
  // from the front (q_cnt), pairs with set-aside endpoints from the back
  // (q_back); one counter each per staging slot.  A pair makes at most one
  // entry, so the two ends never meet.
  uint16_t* queue = reinterpret_cast<uint16_t*>(smem + L.q_off);
  __shared__ int q_cnt[2], q_back[2], q_second, q_exact;
  // two short lists for a third sweep, so that every sweep runs one kind of
  // work per lane: the second endpoints of pairs with both endpoints set aside
  // (list[0, cap)), and the near-Cherenkov pairs that the FP32 check could not
  // settle as zero (list[cap, 2 cap))
  constexpr int kCap = kFwdListCap;
  __shared__ uint16_t list[Ops::kDefers ? 2 * kCap : 1];
  if (tid == 0) {
    q_cnt[0] = q_cnt[1] = 0;
    q_back[0] = q_back[1] = 0;
    q_second = q_exact = 0;
    for (int s = 0; s < 2 && t_begin + s < t_end; ++s) {
      const int st = (int)((it + s) & 1);
      mbar_expect_tx(&bar[st], bytes);
      bulk_g2s(smem + st * L.stage_bytes, src + (t_begin + s) * (int64_t)bytes, bytes, &bar[st]);
    }
  }
  if (Ops::kDefers) __syncthreads();  // counters zeroed before the first entry is added
  for (int64_t t = t_begin; t < t_end; ++t, ++it) {
    const int st = (int)(it & 1);
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const bool ok = mbar_wait_bounded(&bar[st], parity, M.wait_limit);
    if (ok) {
      // one track per thread, held in registers, against every antenna of the tile
      for (int l = tid; l < kTileT; l += nthr) {
        typename Ops::Track tr;
        Ops::load(smem + st * L.stage_bytes, l, M, tr);
        if (!Ops::live(tr)) continue;
#pragma unroll 1
        for (int ant = 0; ant < n_here; ++ant) {
          GlobalSink<acc_t> sink{acc_row0 + (size_t)ant * row_stride, N};
          const int code = Ops::pair_main(tr, Ops::load_ant(ant_s + ant), M, sink);
          if constexpr (Ops::kDefers) {
            if (code == kDeferPair)
              queue[atomicAdd(&q_cnt[st], 1)] = (uint16_t)(l | (ant << 7));
            else if (code != kDeferNone)
              queue[L.q_cap - 1 - atomicAdd(&q_back[st], 1)] = (uint16_t)(l | (ant << 7) | (code << 10));
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        // let the copies already issued land before giving up
        for (int64_t j = it; j < it + 2 && j - it + t < t_end; ++j) mbar_wait_bounded(&bar[j & 1], (uint32_t)((j >> 1) & 1));
      }
      return false;
    }
    if constexpr (Ops::kDefers) {
      // the set-aside work, evaluated together so that each kind runs in full
      // warps (whole pairs first, then set-aside endpoints); the staged tile is
      // still in place
      const int nf = q_cnt[st], nq = nf + q_back[st];
      for (int i = tid; i < nq; i += nthr) {
        const int e = i < nf ? queue[i] : queue[L.q_cap - 1 - (i - nf)];
        const int l = e & (kTileT - 1), ant = (e >> 7) & (kMaxATile - 1);
        GlobalSink<acc_t> sink{acc_row0 + (size_t)ant * row_stride, N};
        const AntRec A = Ops::load_ant(ant_s + ant);
        if (i < nf) {
          if constexpr (Ops::kFastBins) {
            if (!Ops::near_zero_fast(smem + st * L.stage_bytes, l, A, M)) {
              const int k = atomicAdd(&q_exact, 1);
              if (k < kCap) list[kCap + k] = (uint16_t)(e & 0xfff);
            }
          } else {
            typename Ops::Track tr;
            Ops::load(smem + st * L.stage_bytes, l, M, tr);
            Ops::pair_deferred(tr, A, M, sink);
          }
        } else {
          const int ends = (e >> 10) & (kDeferEnd0 | kDeferEnd1);
          if (ends == (kDeferEnd0 | kDeferEnd1)) {
            const int k = atomicAdd(&q_second, 1);
            if (k < kCap) list[k] = (uint16_t)(e & 0xfff);
          }
          Ops::end_deferred(smem + st * L.stage_bytes, l, A, M, sink, (ends & kDeferEnd0) ? kDeferEnd0 : kDeferEnd1);
        }
      }
      __syncthreads();
      // the third sweep: the second endpoints, then the near-Cherenkov pairs for
      // the float-float evaluation; each from its list or, when more than the
      // list holds were set aside (the whole CTA sees the counts alike), from
      // the queue: every pair with both endpoints set aside, every
      // near-Cherenkov pair (those decided zero come out zero again)
      const int ns = q_second, ne = q_exact, nb = nq - nf;
      const bool ov2 = ns > kCap, ovE = ne > kCap;
      const int nA = ov2 ? nb : ns, nB = Ops::kFastBins ? (ovE ? nf : ne) : 0;
      for (int i = tid; i < nA + nB; i += nthr) {
        int e;
        if (i < nA) {
          if (ov2) {
            e = queue[L.q_cap - 1 - i];
            if (((e >> 10) & (kDeferEnd0 | kDeferEnd1)) != (kDeferEnd0 | kDeferEnd1)) continue;
          } else {
            e = list[i];
          }
        } else {
          e = ovE ? queue[i - nA] : list[kCap + (i - nA)];
        }
        const int l = e & (kTileT - 1), ant = (e >> 7) & (kMaxATile - 1);
        GlobalSink<acc_t> sink{acc_row0 + (size_t)ant * row_stride, N};
        const AntRec A = Ops::load_ant(ant_s + ant);
        if (i < nA) {
          Ops::end_deferred(smem + st * L.stage_bytes, l, A, M, sink, kDeferEnd1);
        } else {
          typename Ops::Track tr;
          Ops::load(smem + st * L.stage_bytes, l, M, tr);
          Ops::pair_deferred(tr, A, M, sink);
        }
      }
      // slot st is refilled below (after the third sweep has read it); its
      // counters are next used two tiles on
      if (nA + nB > 0) __syncthreads();
      if (tid == 0) q_cnt[st] = q_back[st] = q_second = q_exact = 0;
    }
    if (tid == 0 && t + 2 < t_end) {
      mbar_expect_tx(&bar[st], bytes);
      bulk_g2s(smem + st * L.stage_bytes, src + (t + 2) * (int64_t)bytes, bytes, &bar[st]);
    }
  }
  return true;
}

template <class Ops>
__global__ void __launch_bounds__(kTileT, Ops::kMinBlocks) k_forward(const FwdArgs a) {
  using acc_t = typename Ops::acc_t;
  using acc4 = typename AccOf<acc_t>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  const FwdLayout L = fwd_layout(Ops::kPrec, a.a_tile, Ops::kDefers);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  AntRec* ant_s = reinterpret_cast<AntRec*>(smem + L.ant_off);
  int ant_tile;
  int64_t range;
  a.g.decode(blockIdx.x, ant_tile, range);
  const int ant0 = ant_tile * a.a_tile;
  const int n_here = min(a.a_tile, a.n_ant - ant0);
  const int64_t t_begin = range * a.g.tiles_per_range;
  const int64_t t_end = min(t_begin + a.g.tiles_per_range, a.n_tiles);
  if (t_begin >= t_end || n_here <= 0) return;  // uniform over the CTA
  const int tid = threadIdx.x;
  for (int i = tid; i < n_here; i += blockDim.x) ant_s[i] = a.ants[ant0 + i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int64_t it = 0;
  acc4* row0 = static_cast<acc4*>(a.acc) + (size_t)ant0 * a.M.n_bins * Ops::kAccRows +
               (size_t)(range % a.replicas) * a.replica_stride;
  if (!stream_range<Ops>(smem, L, bar, ant_s, row0, n_here, static_cast<const unsigned char*>(a.tiles), t_begin,
                         t_end, it, a.M)) {
    if (tid == 0) atomicExch(a.err, kErrWaitTimeout);
  }
}

inline int forward_threads(int a_tile) {
  const int t = kTileT * a_tile;
  return t < kFwdMaxThreads ? t : kFwdMaxThreads;
}

// grid of the forward launch: about `waves` full waves of resident CTAs (a whole
// number of them when the antenna tiles allow, so no wave runs part-empty);
// antenna tiles grouped so that one block's accumulator rows take at most
// l2_budget bytes
inline int64_t forward_grid(FwdArgs& a, const FwdShape& shape, int resident, size_t acc_elem_bytes) {
  FwdGrid& g = a.g;
  g.ant_tiles = (a.n_ant + shape.a_tile - 1) / shape.a_tile;
  const size_t l2_budget = (size_t)48 << 20;
  // an antenna tile's rows in every copy of the accumulator
  const size_t tile_bytes = (size_t)shape.a_tile * a.M.n_bins * acc_elem_bytes * (shape.replicas > 1 ? shape.replicas : 1);
  int tpb = (int)(l2_budget / (tile_bytes > 0 ? tile_bytes : 1));
  g.tiles_per_block = tpb < 1 ? 1 : (tpb > g.ant_tiles ? g.ant_tiles : tpb);
  int64_t target = (int64_t)shape.waves * resident;
  int64_t ranges = (target + g.ant_tiles - 1) / g.ant_tiles;
  {
    // round the CTA count up to a whole number of waves: ranges x ant_tiles = k x resident
    int64_t x = resident, y = g.ant_tiles;
    while (y) {
      const int64_t r = x % y;
      x = y;
      y = r;
    }
    const int64_t step = resident / x;  // ranges must be a multiple of this
    if (step > 0 && step <= 4 * ranges) ranges = (ranges + step - 1) / step * step;
  }
  if (ranges < 1) ranges = 1;
  if (ranges > a.n_tiles) ranges = a.n_tiles;
  g.tiles_per_range = (a.n_tiles + ranges - 1) / ranges;
  g.ranges = (a.n_tiles + g.tiles_per_range - 1) / g.tiles_per_range;
  return (int64_t)g.ant_tiles * g.ranges;
}

template <class Ops>
cudaError_t launch_forward_ops(const FwdArgs& a, int64_t ctas, cudaStream_t st) {
  const size_t smem = fwd_layout(Ops::kPrec, a.a_tile, Ops::kDefers).total;
  auto k = k_forward<Ops>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ctas, kTileT, smem, st>>>(a);
  return cudaGetLastError();
}

// resident CTAs of the forward kernel per SM
template <class Ops>
int forward_blocks_per_sm(int a_tile) {
  int n = 0;
  const size_t smem = fwd_layout(Ops::kPrec, a_tile, Ops::kDefers).total;
  cudaFuncSetAttribute(k_forward<Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward<Ops>, kTileT, smem) != cudaSuccess) n = 1;
  return n < 1 ? 1 : n;
}

// ---------------------------------------------------------------------------
// arrival listing: one thread per (track, antenna)
// ---------------------------------------------------------------------------
template <class Ops>
__global__ void __launch_bounds__(256) k_arrivals(const void* tiles, int64_t n, const AntRec* ants, int n_ant,
                                                  MedParams M, int32_t* branch, int32_t* bin, float* frac) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n * n_ant) return;
  const int64_t i = j / n_ant;
  const int a = (int)(j % n_ant);
  branch[j] = -1;
  bin[2 * j] = bin[2 * j + 1] = -1;
  frac[2 * j] = frac[2 * j + 1] = 0.0f;
  const AntRec A = ants[a];
  ArrivalSink sink{branch, bin, frac, j, M.n_bins};
  const unsigned char* T = static_cast<const unsigned char*>(tiles) + (i / kTileT) * (int64_t)Ops::kTileBytes;
  Ops::fwd(T, (int)(i % kTileT), A, M, sink);
}

// ---------------------------------------------------------------------------
// adjoint (Endpoint): one thread per track, loop over all antennas; track
// gradients stay in registers and are written once; antenna gradients are
// warp-reduced into shared memory and added to global memory once per CTA.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The sums over the 32 lanes of a warp of three values (a, b, c) by a
// reduce-scatter: at offset 16 the lower half keeps (a, b) and the upper half
// (c, 0), each sending the pair it does not keep; at offset 8 each lane keeps
// one of its two partial sums; offsets 4, 2 and 1 finish them.  Six shuffles
// instead of three sums' fifteen.  Lanes 0-7 return the sum of a, lanes 8-15
// that of b, lanes 16-23 that of c (lanes 24-31: 0).  Every lane must call it.
template <typename T>
__device__ __forceinline__ T warp_sum3(T a, T b, T c, int lane) {
  const bool h16 = (lane & 16) != 0;
  T k0 = h16 ? c : a, k1 = h16 ? T(0) : b;
  const T s0 = h16 ? a : c, s1 = h16 ? b : T(0);
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool h8 = (lane & 8) != 0;
  T v = h8 ? k1 : k0;
  v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Refractivity part F = (n_avg - 1) R of the optical path R + F and its
// derivatives (reading M; the ZHS adjoint needs them, the Endpoint deposits do
// not depend on the arrival time).  Exponential medium: F = N0 E_m R rho(x),
// rho(x) = (1 - exp(-x))/x, x = (z_a - z_m)/H, rho' = (exp(-x) - rho)/x; both
// by their series for |x| < 1e-3.  Uniform medium: F = (n - 1) R, and "N0"
// stands for n - 1.
template <typename T>
struct RefrGrad {
  T dF_dR, dF_dzm, dF_dza, dF_dN0, dn_dzm, dn_dN0;
};
template <typename T>
__device__ __forceinline__ RefrGrad<T> refraction_grad(int kind, T R, T x, T E, T N0, T invH, T nm1) {
  RefrGrad<T> g;
  if (kind == C8R_UNIFORM) {
    g.dF_dR = nm1;
    g.dF_dzm = g.dF_dza = T(0);
    g.dF_dN0 = R;
    g.dn_dzm = T(0);
    g.dn_dN0 = T(1);
    return g;
  }
  T rho, drho;
  if (fabs(x) < T(1e-3)) {
    rho = T(1) + x * (T(-0.5) + x * (T(1) / T(6) + x * (T(-1) / T(24))));
    drho = T(-0.5) + x * (T(1) / T(3) + x * (T(-1) / T(8) + x * (T(1) / T(30))));
  } else if constexpr (std::is_same<T, float>::value) {
    // FP32 gradients: the approximate exponential and quotient (a few ulp)
    const float em = __expf(-x);
    const float ix = __frcp_rn(x);
    rho = (1.0f - em) * ix;
    drho = (em - rho) * ix;
  } else {
    const T em = exp(-x);
    rho = (T(1) - em) / x;
    drho = (em - rho) / x;
  }
  g.dF_dR = N0 * E * rho;
  g.dF_dzm = -N0 * R * E * (rho + drho) * invH;
  g.dF_dza = N0 * R * E * drho * invH;
  g.dF_dN0 = E * R * rho;
  g.dn_dzm = -N0 * E * invH;
  g.dn_dN0 = E;
  return g;
}

// Adjoint, laid out like the forward pass: a CTA owns an antenna tile and a
// range of derived-track tiles streamed through the TMA ring; each thread holds
// one track of the staged tile and walks the tile's antennas, keeping the
// track's 11 gradients in registers and adding them to the output with one
// reduction per gradient and antenna tile.  Antenna gradients are warp-reduced
// into shared memory and added to the FP64 output once per CTA.  Pairs set
// aside by Ops::adj_main (Endpoint near the Cherenkov angle) are evaluated
// together after the main pass over each tile, in full warps.
template <typename T>
__device__ __forceinline__ void add_track_grads(const c8r_track_grads& out, int64_t i, const T tg[11]) {
  T* o[11] = {(T*)out.x0, (T*)out.y0, (T*)out.z0, (T*)out.x1, (T*)out.y1, (T*)out.z1,
              (T*)out.t0, (T*)out.t1, (T*)out.bx, (T*)out.by, (T*)out.bz};
#pragma unroll
  for (int k = 0; k < 11; ++k)
    if (tg[k] != T(0)) atomicAdd(o[k] + i, tg[k]);
}

template <class Ops>
__global__ void __launch_bounds__(kTileT, Ops::kBwdMinBlocks) k_backward(const BwdArgs a) {
  using acc_t = typename Ops::acc_t;
  using acc4 = typename AccOf<acc_t>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  const MedParams& M = a.M;
  const FwdLayout L = fwd_layout(Ops::kPrec, a.a_tile, Ops::kDefers);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  AntRec* ant_s = reinterpret_cast<AntRec*>(smem + L.ant_off);
  uint16_t* queue = reinterpret_cast<uint16_t*>(smem + L.q_off);
  __shared__ acc_t sg[3 * kMaxATile + 1];  // antenna gradients of the tile, then dN0
  // set-aside work as in the forward kernel: whole pairs from the front of the
  // queue, pairs with set-aside endpoints from the back, and two short lists for
  // a third sweep (second endpoints; near-Cherenkov pairs not settled as zero)
  __shared__ int q_cnt[2], q_back[2], q_second, q_exact;
  constexpr int kCap = kBwdListCap;
  __shared__ uint16_t list[Ops::kDefers ? 2 * kCap : 1];
  int ant_tile;
  int64_t range;
  a.g.decode(blockIdx.x, ant_tile, range);
  const int ant0 = ant_tile * a.a_tile;
  const int n_here = min(a.a_tile, a.n_ant - ant0);
  const int64_t t_begin = range * a.g.tiles_per_range;
  const int64_t t_end = min(t_begin + a.g.tiles_per_range, a.n_tiles);
  if (t_begin >= t_end || n_here <= 0) return;  // uniform over the CTA
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int N = M.n_bins;
  const acc4* G = static_cast<const acc4*>(a.G) + (size_t)ant0 * N;
  const PrefixFF* Gp = a.Gp ? a.Gp + (size_t)ant0 * (N + 1) : nullptr;
  for (int i = tid; i < n_here; i += nthr) ant_s[i] = a.ants[ant0 + i];
  for (int i = tid; i < 3 * n_here + 1; i += nthr) sg[i] = acc_t(0);
  const uint32_t bytes = (uint32_t)L.stage_bytes;
  const unsigned char* src = static_cast<const unsigned char*>(a.tiles);
  if (tid == 0) {
    q_cnt[0] = q_cnt[1] = 0;
    q_back[0] = q_back[1] = 0;
    q_second = q_exact = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
    for (int s = 0; s < 2 && t_begin + s < t_end; ++s) {
      mbar_expect_tx(&bar[s], bytes);
      bulk_g2s(smem + s * L.stage_bytes, src + (t_begin + s) * (int64_t)bytes, bytes, &bar[s]);
    }
  }
  __syncthreads();
  acc_t dn_acc = 0;
  int64_t it = 0;
  for (int64_t t = t_begin; t < t_end; ++t, ++it) {
    const int st = (int)(it & 1);
    const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((it >> 1) & 1), M.wait_limit);
    const unsigned char* stage = smem + st * L.stage_bytes;
    // every lane walks the antennas (dead slots included) so the warp reductions see all 32
    for (int l = tid; l < kTileT; l += nthr) {
      const int64_t i = t * kTileT + l;
      typename Ops::Track tr;
      Ops::load(stage, l, M, tr);
      const bool live = ok && i < a.n && Ops::live(tr);
      acc_t tg[11];
#pragma unroll
      for (int k = 0; k < 11; ++k) tg[k] = acc_t(0);
#pragma unroll 1
      for (int ant = 0; ant < n_here; ++ant) {
        acc_t ga[3] = {0, 0, 0};
        const PrefixFF* Gp_a = Gp ? Gp + (size_t)ant * (N + 1) : nullptr;
        const int code =
            live ? Ops::adj_main(tr, Ops::load_ant(ant_s + ant), M, G + (size_t)ant * N, Gp_a, tg, ga, dn_acc)
                 : kDeferNone;
        if constexpr (Ops::kDefers) {
          if (code == kDeferPair)
            queue[atomicAdd(&q_cnt[st], 1)] = (uint16_t)(l | (ant << 7));
          else if (code != kDeferNone)
            queue[L.q_cap - 1 - atomicAdd(&q_back[st], 1)] = (uint16_t)(l | (ant << 7) | (code << 10));
        }
        const int lane = tid & 31;
        const acc_t v = warp_sum3(ga[0], ga[1], ga[2], lane);  // x at lane 0, y at 8, z at 16
        if ((lane & 7) == 0 && lane < 24 && v != acc_t(0)) atomicAdd(&sg[3 * ant + (lane >> 3)], v);
      }
      if (live) add_track_grads<acc_t>(a.out, i, tg);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, kErrWaitTimeout);
        for (int64_t j = it; j < it + 2 && j - it + t < t_end; ++j) mbar_wait_bounded(&bar[j & 1], (uint32_t)((j >> 1) & 1));
      }
      return;
    }
    if constexpr (Ops::kDefers) {
      const int nf = q_cnt[st], nq = nf + q_back[st];
      for (int q = tid; q < nq; q += nthr) {
        const int e = q < nf ? queue[q] : queue[L.q_cap - 1 - (q - nf)];
        const int l = e & (kTileT - 1), ant = (e >> 7) & (kMaxATile - 1);
        const AntRec A = Ops::load_ant(ant_s + ant);
        acc_t ga[3] = {0, 0, 0};
        if (q < nf) {
          bool exact = true;
          if constexpr (Ops::kFastBins) {
            // a pair settled as zero has no adjoint either
            exact = false;
            if (!Ops::near_zero_fast(stage, l, A, M)) {
              const int k = atomicAdd(&q_exact, 1);
              if (k < kCap) list[kCap + k] = (uint16_t)(e & 0xfff);
            }
          }
          if (exact) {
            typename Ops::Track tr;
            Ops::load(stage, l, M, tr);
            acc_t tg[11];
#pragma unroll
            for (int k = 0; k < 11; ++k) tg[k] = acc_t(0);
            Ops::adj_deferred(tr, A, M, G + (size_t)ant * N, Gp ? Gp + (size_t)ant * (N + 1) : nullptr, tg, ga,
                              dn_acc);
            add_track_grads<acc_t>(a.out, t * kTileT + l, tg);
          }
        } else {
          const int ends = (e >> 10) & (kDeferEnd0 | kDeferEnd1);
          if (ends == (kDeferEnd0 | kDeferEnd1)) {
            const int k = atomicAdd(&q_second, 1);
            if (k < kCap) list[k] = (uint16_t)(e & 0xfff);
          }
          Ops::adj_end_deferred(stage, l, A, M, G + (size_t)ant * N, a.out, t * kTileT + l, ga, dn_acc,
                                (ends & kDeferEnd0) ? kDeferEnd0 : kDeferEnd1);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (ga[c] != acc_t(0)) atomicAdd(&sg[3 * ant + c], ga[c]);
      }
      __syncthreads();
      // the third sweep, as in the forward kernel: second endpoints, then the
      // near-Cherenkov pairs for the float-float evaluation (from the lists, or
      // from the queue when a list overflowed)
      const int ns = q_second, ne = q_exact, nb = nq - nf;
      const bool ov2 = ns > kCap, ovE = ne > kCap;
      const int nA = ov2 ? nb : ns, nB = Ops::kFastBins ? (ovE ? nf : ne) : 0;
      for (int q = tid; q < nA + nB; q += nthr) {
        int e;
        if (q < nA) {
          if (ov2) {
            e = queue[L.q_cap - 1 - q];
            if (((e >> 10) & (kDeferEnd0 | kDeferEnd1)) != (kDeferEnd0 | kDeferEnd1)) continue;
          } else {
            e = list[q];
          }
        } else {
          e = ovE ? queue[q - nA] : list[kCap + (q - nA)];
        }
        const int l = e & (kTileT - 1), ant = (e >> 7) & (kMaxATile - 1);
        const AntRec A = Ops::load_ant(ant_s + ant);
        acc_t ga[3] = {0, 0, 0};
        if (q < nA) {
          Ops::adj_end_deferred(stage, l, A, M, G + (size_t)ant * N, a.out, t * kTileT + l, ga, dn_acc, kDeferEnd1);
        } else {
          typename Ops::Track tr;
          Ops::load(stage, l, M, tr);
          acc_t tg[11];
#pragma unroll
          for (int k = 0; k < 11; ++k) tg[k] = acc_t(0);
          Ops::adj_deferred(tr, A, M, G + (size_t)ant * N, Gp ? Gp + (size_t)ant * (N + 1) : nullptr, tg, ga, dn_acc);
          add_track_grads<acc_t>(a.out, t * kTileT + l, tg);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (ga[c] != acc_t(0)) atomicAdd(&sg[3 * ant + c], ga[c]);
      }
      // slot st is refilled below (after the third sweep has read it); its
      // counters are next used two tiles on
      if (nA + nB > 0) __syncthreads();
      if (tid == 0) q_cnt[st] = q_back[st] = q_second = q_exact = 0;
    }
    if (tid == 0 && t + 2 < t_end) {
      mbar_expect_tx(&bar[st], bytes);
      bulk_g2s(smem + st * L.stage_bytes, src + (t + 2) * (int64_t)bytes, bytes, &bar[st]);
    }
  }
  const acc_t d = warp_sum(dn_acc);
  if ((tid & 31) == 0 && d != acc_t(0)) atomicAdd(&sg[3 * n_here], d);
  __syncthreads();
  for (int k = tid; k < 3 * n_here; k += nthr)
    if (sg[k] != acc_t(0)) atomicAdd(&a.ant_grad[3 * (size_t)ant0 + k], (double)sg[k]);
  if (tid == 0 && sg[3 * n_here] != acc_t(0)) atomicAdd(a.dN0, (double)sg[3 * n_here]);
}

template <class Ops>
cudaError_t launch_backward_ops(BwdArgs& a, const FwdShape& shape, int sm_count, cudaStream_t st) {
  const size_t smem = fwd_layout(Ops::kPrec, a.a_tile, Ops::kDefers).total;
  auto k = k_backward<Ops>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTileT, smem);
  if (e != cudaSuccess) return e;
  FwdArgs f{a.tiles, a.n_tiles, a.ants, a.n_ant, a.a_tile, nullptr, a.err, FwdGrid{}, a.M};
  FwdShape one = shape;  // the L2 grouping covers one bin-major gradient, not the forward's accumulator copies
  one.replicas = 1;
  const int64_t ctas = forward_grid(f, one, sm_count * (per_sm < 1 ? 1 : per_sm), sizeof(typename AccOf<typename Ops::acc_t>::type));
  a.g = f.g;
  k<<<(unsigned)ctas, kTileT, smem, st>>>(a);
  return cudaGetLastError();
}

// gradient of one deposit l = kappa (g.V)/(D R) with respect to d = x_a - x_e,
// beta and the source index n (with bins held fixed):
//   dl/dd    = kappa/(D R^2) [ -(rhat.g) V + c (g - rhat (rhat.g)) - (g.V)(n V/D + rhat) ]
//   dl/dbeta = kappa/(D R)   [ (rhat.g) rhat - g + (g.V) n rhat / D ]
//   dl/dn    = kappa (g.V) c / (D^2 R)
template <typename T>
__device__ __forceinline__ void deposit_adjoint(const T rh[3], const T V[3], T c, T D, T R, T n, const T g[3],
                                                T kappa, T dd[3], T db[3], T& dnsrc) {
  const T gV = g[0] * V[0] + g[1] * V[1] + g[2] * V[2];
  const T rg = rh[0] * g[0] + rh[1] * g[1] + rh[2] * g[2];
  T invD, f1, f2;
  if constexpr (std::is_same<T, float>::value) {
    // FP32 path: correctly rounded reciprocals instead of three full divisions
    invD = __frcp_rn(D);
    const float invR = __frcp_rn(R);
    f2 = kappa * invD * invR;
    f1 = f2 * invR;
  } else {
    invD = T(1) / D;
    f1 = kappa * invD / (R * R);
    f2 = kappa * invD / R;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dd[k] = f1 * (-rg * V[k] + c * (g[k] - rh[k] * rg) - gV * (n * V[k] * invD + rh[k]));
    db[k] = f2 * (rg * rh[k] - g[k] + gV * n * rh[k] * invD);
  }
  dnsrc = f2 * gV * c * invD;
}

}  // namespace c8r
