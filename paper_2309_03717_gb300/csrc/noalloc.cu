// noalloc.cu -- the mixed-precision forward pass (ingest + pair kernel) for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or allocator callback, code that is only allowed to
// use memory it was handed, or long-running services that must not grow their
// device footprint after start-up.  c8r_traces_noalloc serves them.  Instead of
// a context, its scratch (the derived-track tiles of one chunk, the antenna
// table and a status word) lives in file-scope __device__ arrays of fixed size,
// which every GPU that loads the library holds until the process exits.  The
// caller passes the tracks and the output traces.
//
// In host code the names of those arrays are host-side stand-ins, not device
// addresses, so the device addresses are looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, with that device
// current) and handed to the kernels.
#include <mutex>

#include "ingest.cuh"
#include "pair_mixed.cuh"

namespace c8r {
namespace {

constexpr int kNaChunkTracks = 65536;                   // tracks per internal chunk
constexpr int kNaChunkTiles = kNaChunkTracks / kTileT;  // 512 tiles
constexpr int kNaMaxAnt = 1024;
constexpr int kNaMaxBins = 1 << 24;
constexpr int kNaMaxDevices = 64;

// 512 tiles x 12.8 KB = 6.55 MB of track scratch, 96 KB of antenna table
static __device__ __align__(256) unsigned char g_na_tiles[(size_t)kNaChunkTiles * kTileBytesMixed];
static __device__ __align__(256) AntRec g_na_ants[kNaMaxAnt];
static __device__ __align__(256) int g_na_err[4];

struct NaAddrs {
  void* tiles = nullptr;
  AntRec* ants = nullptr;
  int* err = nullptr;
  cudaError_t status = cudaSuccess;
};
NaAddrs g_na_addrs[kNaMaxDevices];
std::once_flag g_na_once[kNaMaxDevices];

// deposits straight into the caller's traces [n_ant][3][n_bins]
struct TraceSink {
  float* tr;  // traces of one antenna
  int N;
  __device__ __forceinline__ void dep(int k, float x, float y, float z) {
    atomicAdd(tr + k, x);
    atomicAdd(tr + N + k, y);
    atomicAdd(tr + 2 * N + k, z);
  }
  __device__ __forceinline__ void dep_box(int k0, int k1, float x, float y, float z) {
    for (int k = k0; k <= k1; ++k) dep(k, x, y, z);
  }
  __device__ __forceinline__ void rec(int, ff, ff) {}
  __device__ __forceinline__ void rec(int, double, double) {}
};

struct NaArgs {
  const unsigned char* tiles;
  int64_t n_tiles;
  int64_t tiles_per_range;
  const AntRec* ants;
  int n_ant;
  int a_tile;
  float* out;
  int* err;
  MedParams M;
};

// grid.x = antenna tile, grid.y = track range; same streaming scheme as the
// context path (two-slot TMA ring, bounded mbarrier waits)
template <class Ops>
__global__ void __launch_bounds__(kFwdMaxThreads, 1) k_forward_noalloc(const NaArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FwdLayout L = fwd_layout(C8R_MIXED, a.a_tile, false);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  AntRec* ant_s = reinterpret_cast<AntRec*>(smem + L.ant_off);
  const int N = a.M.n_bins;
  const int ant0 = blockIdx.x * a.a_tile;
  const int n_here = min(a.a_tile, a.n_ant - ant0);
  const int64_t t_begin = (int64_t)blockIdx.y * a.tiles_per_range;
  const int64_t t_end = min(t_begin + a.tiles_per_range, a.n_tiles);
  if (t_begin >= t_end || n_here <= 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < n_here; i += nthr) ant_s[i] = a.ants[ant0 + i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const uint32_t bytes = (uint32_t)L.stage_bytes;
  if (tid == 0)
    for (int s = 0; s < 2 && t_begin + s < t_end; ++s) {
      mbar_expect_tx(&bar[s], bytes);
      bulk_g2s(smem + s * L.stage_bytes, a.tiles + (t_begin + s) * (int64_t)bytes, bytes, &bar[s]);
    }
  const int n_pairs = kTileT * n_here;
  int64_t it = 0;
  for (int64_t t = t_begin; t < t_end; ++t, ++it) {
    const int st = (int)(it & 1);
    const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((it >> 1) & 1), a.M.wait_limit);
    if (ok) {
      for (int p = tid; p < n_pairs; p += nthr) {
        const int ant = p / kTileT;
        TraceSink sink{a.out + (size_t)(ant0 + ant) * 3 * N, N};
        Ops::fwd(smem + st * L.stage_bytes, p % kTileT, ant_s[ant], a.M, sink);
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, kErrWaitTimeout);
        for (int64_t j = it; j < it + 2 && j - it + t < t_end; ++j)
          mbar_wait_bounded(&bar[j & 1], (uint32_t)((j >> 1) & 1));
      }
      return;
    }
    if (tid == 0 && t + 2 < t_end) {
      mbar_expect_tx(&bar[st], bytes);
      bulk_g2s(smem + st * L.stage_bytes, a.tiles + (t + 2) * (int64_t)bytes, bytes, &bar[st]);
    }
  }
}

template <class Ops>
cudaError_t launch_na(const NaArgs& a, dim3 grid, cudaStream_t st) {
  const size_t smem = fwd_layout(C8R_MIXED, a.a_tile, false).total;
  auto k = k_forward_noalloc<Ops>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, forward_threads(a.a_tile), smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace c8r

using namespace c8r;

extern "C" int c8r_traces_noalloc(const c8r_tracks* tracks, int64_t n, int32_t n_ant, const double* pos_xyz,
                                  const double* t_start_ns, int32_t n_bins, double dt_ns, int formalism,
                                  int medium_kind, double n_or_N0, double scale_height_m, float* out_traces,
                                  void* cuda_stream) {
  if (!tracks || !pos_xyz || !t_start_ns || !out_traces) return C8R_EINVAL;
  if (n < 0 || n_ant < 1 || n_bins < 1 || !(dt_ns > 0.0) || !std::isfinite(dt_ns)) return C8R_EINVAL;
  if (n_ant > kNaMaxAnt || n_bins > kNaMaxBins) return C8R_ETOOBIG;
  if (formalism != C8R_ENDPOINT && formalism != C8R_ZHS) return C8R_EINVAL;
  if (tracks->dtype != C8R_F32 && tracks->dtype != C8R_F64) return C8R_EINVAL;
  if (medium_kind == C8R_UNIFORM) {
    if (!std::isfinite(n_or_N0) || !(n_or_N0 > 0.0)) return C8R_EINVAL;
  } else if (medium_kind == C8R_EXPONENTIAL) {
    if (!std::isfinite(n_or_N0) || n_or_N0 < 0.0 || !std::isfinite(scale_height_m) || !(scale_height_m > 0.0))
      return C8R_EINVAL;
  } else {
    return C8R_EINVAL;
  }
  const void* f[12] = {tracks->x0, tracks->y0, tracks->z0, tracks->x1, tracks->y1, tracks->z1,
                       tracks->t0, tracks->t1, tracks->bx, tracks->by, tracks->bz, tracks->q};
  if (n > 0)
    for (int k = 0; k < 12; ++k)
      if (!f[k]) return C8R_EINVAL;
  for (int a = 0; a < n_ant; ++a)
    if (!std::isfinite(pos_xyz[3 * a]) || !std::isfinite(pos_xyz[3 * a + 1]) || !std::isfinite(pos_xyz[3 * a + 2]) ||
        !std::isfinite(t_start_ns[a]))
      return C8R_EINVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return C8R_ECUDA;
  // once per device, with that device current: device addresses of the scratch
  std::call_once(g_na_once[dev], [dev] {
    NaAddrs& s = g_na_addrs[dev];
    s.status = cudaGetSymbolAddress(&s.tiles, g_na_tiles);
    if (s.status == cudaSuccess) s.status = cudaGetSymbolAddress((void**)&s.ants, g_na_ants);
    if (s.status == cudaSuccess) s.status = cudaGetSymbolAddress((void**)&s.err, g_na_err);
  });
  const NaAddrs& na = g_na_addrs[dev];
  if (na.status != cudaSuccess || !na.tiles || !na.ants || !na.err) return C8R_ECUDA;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  MedParams M;
  fill_medium(M, medium_kind, n_or_N0, scale_height_m, n_bins, dt_ns, 1e-3);
  M.wait_limit = current_wait_limit();
  // antenna table, built on the host stack in blocks and copied into the scratch
  constexpr int kBlock = 64;
  AntRec block[kBlock];
  for (int a0 = 0; a0 < n_ant; a0 += kBlock) {
    const int m = (n_ant - a0) < kBlock ? (n_ant - a0) : kBlock;
    for (int i = 0; i < m; ++i) {
      const double* p = pos_xyz + 3 * (size_t)(a0 + i);
      fill_antenna(block[i], p[0], p[1], p[2], t_start_ns[a0 + i], M);
    }
    // from pageable memory: returns once the source has been consumed
    if (cudaMemcpyAsync(na.ants + a0, block, sizeof(AntRec) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return C8R_ECUDA;
  }
  if (cudaMemsetAsync(na.err, 0, sizeof(int) * 4, st) != cudaSuccess) return C8R_ECUDA;
  if (n == 0) return C8R_OK;

  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int a_tile = n_ant < 8 ? n_ant : 8;
  const int ant_tiles = (n_ant + a_tile - 1) / a_tile;
  const size_t es = tracks->dtype == C8R_F64 ? 8 : 4;
  const bool ex = medium_kind == C8R_EXPONENTIAL;
  for (int64_t off = 0; off < n; off += kNaChunkTracks) {
    const int64_t m = (n - off) < kNaChunkTracks ? (n - off) : kNaChunkTracks;
    TrackPtrs tp;
    tp.dtype = tracks->dtype;
    for (int k = 0; k < 12; ++k) tp.f[k] = static_cast<const char*>(f[k]) + off * es;
    const int64_t n_tiles = (m + kTileT - 1) / kTileT;
    cudaError_t e = launch_ingest_map(C8R_MIXED, tp, ingest_detail::IdentityMap{m}, n_tiles * kTileT, na.tiles, M,
                                      nullptr, st);
    if (e != cudaSuccess) return C8R_ECUDA;
    NaArgs a;
    a.tiles = static_cast<const unsigned char*>(na.tiles);
    a.n_tiles = n_tiles;
    int64_t ranges = (4LL * sms + ant_tiles - 1) / ant_tiles;
    if (ranges > n_tiles) ranges = n_tiles;
    a.tiles_per_range = (n_tiles + ranges - 1) / ranges;
    ranges = (n_tiles + a.tiles_per_range - 1) / a.tiles_per_range;
    a.ants = na.ants;
    a.n_ant = n_ant;
    a.a_tile = a_tile;
    a.out = out_traces;
    a.err = na.err;
    a.M = M;
    const dim3 grid((unsigned)ant_tiles, (unsigned)ranges);
    if (formalism == C8R_ENDPOINT)
      e = ex ? launch_na<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>>(a, grid, st)
             : launch_na<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>>(a, grid, st);
    else
      e = ex ? launch_na<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL>>(a, grid, st)
             : launch_na<OpsMixed<C8R_ZHS, C8R_UNIFORM>>(a, grid, st);
    if (e != cudaSuccess) return C8R_ECUDA;
  }
  // the status word: a kernel that gave up a bounded wait returned early, so
  // the traces are incomplete (read into host memory; the copy and the
  // synchronisation allocate nothing)
  int status = kErrNone;
  if (cudaMemcpyAsync(&status, na.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return C8R_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return C8R_ECUDA;
  return status == kErrNone ? C8R_OK : C8R_ECANCELLED;
}
