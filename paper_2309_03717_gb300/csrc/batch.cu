// batch.cu -- many independent showers of uneven size in one persistent launch
// (not in the paper, whose radio process handles one shower; this is the
// batching the GPU needs to stay busy on small showers).
//
// The host cuts every shower into work items (antenna tile x range of derived
// track tiles) and uploads the list, largest shower first and, inside a shower,
// antenna tiles fastest (so the items in flight share track tiles in L2 and add
// into one shower's accumulator rows); for the one-bin Endpoint evaluation the
// showers are grouped by the form of their FP32 arrival (a vote per shower),
// and each group gets a launch of its own.  A persistent grid of every CTA the
// device holds pops items from a global atomic counter; for each item a CTA streams the item's
// track tiles through the same TMA ring as the single-shower kernel and adds the
// deposits into the batch accumulator.  The CTA polls a cancel word between
// items.  Zeroing the accumulator, the ingest of all showers, the counter reset,
// the persistent kernel and the conversion into the caller's trace layout are
// captured once into a CUDA graph and replayed.  The tile shape (antennas per
// CTA, track tiles per item) is picked by a small autotuner that times the
// candidates on a subsample of the real work list and caches the choice.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "ingest.cuh"
#include "pair_mixed.cuh"

namespace c8r {

struct WorkItem {
  int32_t ant0;     // first antenna (index into the concatenated table)
  int32_t n_here;   // antennas in this item
  int64_t t_begin;  // first derived-track tile
  int64_t t_end;
};

struct BatchArgs {
  const void* tiles;
  const WorkItem* items;
  int n_items;
  const AntRec* ants;
  float4* acc;           // [replicas][sum n_ant][rows][n_bins] accumulator
  int* counter;
  const int* cancel;
  int* err;
  int a_tile;
  MedParams M;
  int replicas;            // accumulator copies: work item i adds into copy i % replicas
  int64_t replica_stride;  // elements per copy
};

// slot -> caller track index for the concatenated showers: shower s owns tiles
// [tile_off[s], tile_off[s+1]) and tracks [track_off[s], track_off[s]+n_tracks[s])
struct BatchMap {
  const int64_t* tile_off;  // [n_showers + 1]
  const int64_t* track_off;
  const int64_t* n_tracks;
  int n_showers;
  __device__ __forceinline__ int64_t operator()(int64_t g) const {
    const int64_t tile = g / kTileT;
    int lo = 0, hi = n_showers - 1;
    while (lo < hi) {  // last s with tile_off[s] <= tile
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= tile) lo = mid;
      else hi = mid - 1;
    }
    const int64_t l = g - tile_off[lo] * kTileT;
    return l < n_tracks[lo] ? track_off[lo] + l : -1;
  }
};

// the arrival-form vote of each shower (Endpoint): of the kept tracks in up
// to kVoteTiles of its derived-track tiles, those whose start point sees the
// shower's antenna centroid from above within 45 degrees (the test of the
// single-shower ingest).  One CTA per shower of a chunk of up to kVoteChunk.
constexpr int kVoteTiles = 64;
constexpr int kVoteChunk = 64;
struct VoteShower {
  int64_t t_begin, t_end;  // derived-track tiles
  float cx, cy, cz;        // antenna centroid
};
struct VoteArgs {
  VoteShower s[kVoteChunk];
};
__global__ void __launch_bounds__(256) k_batch_votes(const float* tiles, const VoteArgs a, unsigned* out) {
  const VoteShower v = a.s[blockIdx.x];
  const int64_t t_end = min(v.t_end, v.t_begin + (int64_t)kVoteTiles);
  unsigned kept = 0, above = 0;
  for (int64_t i = v.t_begin * kTileT + threadIdx.x; i < t_end * kTileT; i += blockDim.x) {
    const float* T = tiles + (i / kTileT) * (int64_t)(fm::NFIELDS * kTileT);
    const int l = (int)(i % kTileT);
    if (T[fm::AMPE * kTileT + l] == 0.0f) continue;  // filtered track or padding
    ++kept;
    const float sx = v.cx - T[fm::X0 * kTileT + l], sy = v.cy - T[fm::Y0 * kTileT + l];
    const float sz = v.cz - T[fm::Z0 * kTileT + l];
    above += (sz < 0.0f && sx * sx + sy * sy < sz * sz) ? 1u : 0u;
  }
  __shared__ unsigned sk, sa;
  if (threadIdx.x == 0) sk = sa = 0;
  __syncthreads();
  if (kept) atomicAdd(&sk, kept);
  if (above) atomicAdd(&sa, above);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sk;
    out[2 * blockIdx.x + 1] = sa;
  }
}

template <class Ops>
__global__ void __launch_bounds__(kTileT, Ops::kMinBlocks) k_batch(const BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const MedParams& M = a.M;
  const FwdLayout L = fwd_layout(Ops::kPrec, a.a_tile, Ops::kDefers);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  AntRec* ant_s = reinterpret_cast<AntRec*>(smem + L.ant_off);
  __shared__ int s_item;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  int64_t it = 0;
  for (;;) {
    if (tid == 0) {
      const int cancelled = *(volatile const int*)a.cancel;
      s_item = cancelled ? -1 : atomicAdd(a.counter, 1);
      if (cancelled) atomicExch(a.err, kErrCancelled);
    }
    __syncthreads();
    const int idx = s_item;
    if (idx < 0 || idx >= a.n_items) break;
    const WorkItem w = a.items[idx];
    for (int i = tid; i < w.n_here; i += nthr) ant_s[i] = a.ants[w.ant0 + i];
    __syncthreads();
    float4* acc = a.acc + (size_t)(idx % a.replicas) * a.replica_stride + (size_t)w.ant0 * M.n_bins * Ops::kAccRows;
    if (!stream_range<Ops>(smem, L, bar, ant_s, acc, w.n_here,
                           static_cast<const unsigned char*>(a.tiles), w.t_begin, w.t_end, it, M)) {
      if (tid == 0) atomicExch(a.err, kErrWaitTimeout);
      return;
    }
    __syncthreads();
  }
}

// resident CTAs per SM of the batch kernel for antenna tiles of a_tile
template <class Ops>
int batch_blocks_per_sm(int a_tile) {
  const size_t smem = fwd_layout(C8R_MIXED, a_tile, Ops::kDefers).total;
  auto k = k_batch<Ops>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTileT, smem) != cudaSuccess) return 1;
  return per_sm < 1 ? 1 : per_sm;
}

// persistent grid: every CTA that fits on the device at once
template <class Ops>
cudaError_t launch_batch_ops(const BatchArgs& a, int sm_count, cudaStream_t st) {
  const size_t smem = fwd_layout(C8R_MIXED, a.a_tile, Ops::kDefers).total;
  auto k = k_batch<Ops>;
  const int per_sm = batch_blocks_per_sm<Ops>(a.a_tile);
  k<<<sm_count * per_sm, kTileT, smem, st>>>(a);
  return cudaGetLastError();
}

template <class F>
auto with_batch_ops(int formalism, int kind, bool split, bool flat, F f) {
  const bool ex = kind == C8R_EXPONENTIAL;
  // the arrival form of the one-bin Endpoint kernel (OpsMixed::kSplit) and, for
  // the direct form, the flat-array kernel of the exponential medium
  // (OpsMixed::kFlat)
  if (formalism == C8R_ENDPOINT) {
    if (!ex)
      return split ? f(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, false, true>{}) : f(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM>{});
    if (split) return f(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, true>{});
    return flat ? f(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, false, true>{})
                : f(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL>{});
  }
  return ex ? f(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL>{}) : f(OpsMixed<C8R_ZHS, C8R_UNIFORM>{});
}

cudaError_t launch_batch(const BatchArgs& a, int formalism, int sm_count, cudaStream_t st) {
  return with_batch_ops(formalism, a.M.kind, a.M.split != 0, a.M.flat != 0,
                        [&](auto ops) { return launch_batch_ops<decltype(ops)>(a, sm_count, st); });
}

int batch_resident(int formalism, int kind, int a_tile, int sm_count) {
  return sm_count * with_batch_ops(formalism, kind, false, false,
                                   [&](auto ops) { return batch_blocks_per_sm<decltype(ops)>(a_tile); });
}

// ---------------------------------------------------------------------------
// autotuner: candidates are timed on the device; choices are cached in a text
// file (C8R_TUNE_CACHE, default $HOME/.cache/c8r_tune.txt) keyed by a string
// ---------------------------------------------------------------------------
struct TuneChoice {
  int a_tile;
  int64_t tiles_per_item;
};

static std::string tune_cache_path() {
  if (const char* p = std::getenv("C8R_TUNE_CACHE")) return p;
  if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/c8r_tune.txt";
  return "";
}

static bool tune_lookup(const std::string& key, TuneChoice& c) {
  const std::string path = tune_cache_path();
  if (path.empty()) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream ss(line);
    std::string k;
    TuneChoice t{};
    if (ss >> k >> t.a_tile >> t.tiles_per_item && k == key && t.a_tile > 0 && t.tiles_per_item > 0) {
      c = t;
      return true;
    }
  }
  return false;
}

static void tune_store(const std::string& key, const TuneChoice& c) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // one level, best effort
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << c.a_tile << " " << c.tiles_per_item << "\n";
}

}  // namespace c8r

using namespace c8r;

struct c8r_batch {
  int device = 0;
  int sm_count = 0;
  std::string err;
  int n_showers = 0;
  int formalism = C8R_ENDPOINT;
  MedParams M{};
  std::vector<int64_t> n_tracks, track_off, tile_off;
  std::vector<int32_t> n_ant, ant_off;
  int64_t total_tracks = 0, total_tiles = 0, total_pairs = 0;
  int total_ant = 0;
  AntRec* d_ants = nullptr;
  void* d_tiles = nullptr;
  int64_t* d_tile_off = nullptr;
  int64_t* d_track_off = nullptr;
  int64_t* d_n_tracks = nullptr;
  WorkItem* d_items = nullptr;
  int n_items = 0;
  int* d_counter = nullptr;
  int* d_cancel = nullptr;
  int* d_err = nullptr;
  // the arrival form of each shower (Endpoint, one-bin: MedParams::split);
  // the work list holds the split-form showers' items first, n_items_split of
  // them, then the direct-form showers', each group run by its own launch
  std::vector<char> shower_split;
  int n_items_split = 0;
  std::vector<float> cen;  // per shower: antenna centroid (x, y, z)
  float4* d_acc = nullptr;  // [replicas][total_ant][rows][n_bins] accumulator
  size_t acc_bytes = 0;
  int replicas = 1;
  cudaStream_t cap_stream = nullptr;  // graph capture (the caller's stream may be the legacy default stream)
  cudaStream_t aux_stream = nullptr;  // non-blocking: cancel word updates while a batch runs
  bool tuned = false;
  TuneChoice choice{4, 64};
  // graph bound to (tracks, out) of its capture
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_src = nullptr;
  const void* g_tracks[12] = {};
  void* g_out = nullptr;
};

namespace {

int bfail(c8r_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}

// the work list: the split-form showers first, then the direct-form ones (their
// count of items in *n_split), each group largest shower first
std::vector<WorkItem> make_items(const c8r_batch* b, int a_tile, int64_t tpi, int* n_split = nullptr) {
  std::vector<int> order(b->n_showers);
  for (int s = 0; s < b->n_showers; ++s) order[s] = s;
  auto split_of = [&](int s) { return b->shower_split.empty() || b->shower_split[s]; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (split_of(x) != split_of(y)) return split_of(x);
    return b->n_tracks[x] * (int64_t)b->n_ant[x] > b->n_tracks[y] * (int64_t)b->n_ant[y];
  });
  std::vector<WorkItem> v;
  if (n_split) *n_split = 0;
  for (int s : order) {
    const int64_t nt = b->tile_off[s + 1] - b->tile_off[s];
    if (nt == 0) continue;
    for (int64_t r = 0; r < nt; r += tpi) {
      for (int a0 = 0; a0 < b->n_ant[s]; a0 += a_tile) {
        WorkItem w;
        w.ant0 = b->ant_off[s] + a0;
        w.n_here = std::min(a_tile, b->n_ant[s] - a0);
        w.t_begin = b->tile_off[s] + r;
        w.t_end = b->tile_off[s] + std::min(nt, r + tpi);
        v.push_back(w);
      }
    }
    if (n_split && split_of(s)) *n_split = (int)v.size();
  }
  return v;
}

int upload_items(c8r_batch* b, const std::vector<WorkItem>& v) {
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  b->n_items = (int)v.size();
  if (v.empty()) return C8R_OK;
  cudaError_t e = dev_malloc(&b->d_items, sizeof(WorkItem) * v.size());
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, v.data(), sizeof(WorkItem) * v.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(b, C8R_ENOMEM, std::string("work list upload: ") + cudaGetErrorString(e));
  return C8R_OK;
}

// tiles per item giving about `waves` items per resident CTA for tile width a_tile
int64_t tpi_for(const c8r_batch* b, int a_tile, int waves) {
  const double pair_units = (double)b->total_pairs / (kTileT * (double)a_tile);
  const int resident = batch_resident(b->formalism, b->M.kind, a_tile, b->sm_count);
  int64_t t = (int64_t)(pair_units / ((double)waves * resident));
  return std::max<int64_t>(t, 8);
}

// zero the accumulator and ingest the tracks
int enqueue_ingest(c8r_batch* b, const TrackPtrs& tp, cudaStream_t st) {
  BatchMap map{b->d_tile_off, b->d_track_off, b->d_n_tracks, b->n_showers};
  cudaError_t e = cudaMemsetAsync(b->d_acc, 0, b->acc_bytes, st);
  if (e == cudaSuccess)
    e = launch_ingest_map(C8R_MIXED, tp, map, b->total_tiles * kTileT, b->d_tiles, b->M, nullptr, st);
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("batch ingest: ") + cudaGetErrorString(e));
  return C8R_OK;
}

// run the persistent kernel over the first n_items_limit items of the work list
// (the split-form group, then the direct-form group, one launch each, each
// with its own item counter: d_counter[0] and d_counter[3])
int enqueue_kernel(c8r_batch* b, int n_items_limit, cudaStream_t st) {
  const int rows = acc_rows(C8R_MIXED, b->formalism);
  const int n = std::min(b->n_items, n_items_limit);
  const int ns = std::min(b->n_items_split, n);
  const int first[2] = {0, ns}, count[2] = {ns, n - ns};
  for (int g = 0; g < 2; ++g) {
    if (count[g] <= 0) continue;
    int* counter = b->d_counter + (g == 0 ? 0 : 3);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("batch counter: ") + cudaGetErrorString(e));
    BatchArgs a{b->d_tiles, b->d_items + first[g], count[g], b->d_ants, b->d_acc, counter,
                b->d_cancel, b->d_err, b->choice.a_tile, b->M, b->replicas,
                (int64_t)b->total_ant * b->M.n_bins * rows};
    a.M.wait_limit = current_wait_limit();
    a.M.split = g == 0 ? 1 : 0;
    e = launch_batch(a, b->formalism, b->sm_count, st);
    if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  }
  return C8R_OK;
}

// zero the accumulator, ingest, run the persistent kernel over the first
// n_items_limit items, and (out != NULL) add the accumulator into out
int enqueue(c8r_batch* b, const TrackPtrs& tp, float* out, int n_items_limit, cudaStream_t st) {
  int r = enqueue_ingest(b, tp, st);
  if (r == C8R_OK) r = enqueue_kernel(b, n_items_limit, st);
  if (r != C8R_OK) return r;
  if (out) {
    cudaError_t e = launch_acc_to_traces(C8R_MIXED, b->d_acc, b->total_ant, b->M.n_bins,
                                         acc_rows(C8R_MIXED, b->formalism), out, 1, st, b->replicas);
    if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("batch fetch: ") + cudaGetErrorString(e));
  }
  return C8R_OK;
}

// the arrival form of each shower's one-bin Endpoint evaluation
// (MedParams::split) from its votes (k_batch_votes on the ingested tiles): the
// split form when at least half of the tracks counted see the shower's antenna
// centroid from above within 45 degrees.  Once per batch, before the first
// run: one ingest, the vote kernel (its counts written into the accumulator,
// which every run zeroes first), a synchronous read.
int choose_forms(c8r_batch* b, const TrackPtrs& tp, cudaStream_t st) {
  b->shower_split.assign(b->n_showers, 1);
  BatchMap map{b->d_tile_off, b->d_track_off, b->d_n_tracks, b->n_showers};
  cudaError_t e =
      launch_ingest_map(C8R_MIXED, tp, map, b->total_tiles * kTileT, b->d_tiles, b->M, nullptr, st);
  unsigned* counts = reinterpret_cast<unsigned*>(b->d_acc);  // 2 x n_showers <= accumulator elements x 4
  std::vector<unsigned> h(2 * (size_t)b->n_showers, 0u);
  for (int s0 = 0; e == cudaSuccess && s0 < b->n_showers; s0 += kVoteChunk) {
    const int m = std::min(kVoteChunk, b->n_showers - s0);
    VoteArgs va;
    for (int i = 0; i < m; ++i) {
      const int s = s0 + i;
      va.s[i] = VoteShower{b->tile_off[s], b->tile_off[s + 1], b->cen[3 * s], b->cen[3 * s + 1], b->cen[3 * s + 2]};
    }
    k_batch_votes<<<(unsigned)m, 256, 0, st>>>(static_cast<const float*>(b->d_tiles), va, counts + 2 * s0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), counts, sizeof(unsigned) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("batch form votes: ") + cudaGetErrorString(e));
  for (int s = 0; s < b->n_showers; ++s)
    if (h[2 * s] > 0) b->shower_split[s] = 2 * (size_t)h[2 * s + 1] >= h[2 * s] ? 1 : 0;
  return C8R_OK;
}

int autotune(c8r_batch* b, const TrackPtrs& tp, cudaStream_t st) {
  if (b->formalism == C8R_ENDPOINT && (b->M.kind == C8R_UNIFORM || b->M.kind == C8R_EXPONENTIAL)) {
    const int r = choose_forms(b, tp, st);
    if (r != C8R_OK) return r;
  }
  char keybuf[160];
  std::snprintf(keybuf, sizeof keybuf, "batch3:N%d:f%d:m%d:sm%d:P%lld", b->M.n_bins, b->formalism, b->M.kind,
                b->sm_count, (long long)(b->total_pairs >> 26));
  const std::string key = keybuf;
  TuneChoice best{};
  if (tune_lookup(key, best) && best.a_tile <= kMaxATile) {
    b->choice = best;
    b->tuned = true;
    return upload_items(b, make_items(b, best.a_tile, best.tiles_per_item, &b->n_items_split));
  }
  std::vector<TuneChoice> cands;
  for (int at : {8, 16, 32})
    for (int waves : {4, 8, 16, 32}) cands.push_back({at, tpi_for(b, at, waves)});
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_rate = -1.0;
  // the tracks are ingested once; each candidate's kernel is timed alone on the
  // leading items of its work list (largest showers first) that carry a quarter
  // of the pairs, but at least four items per resident CTA
  int r = enqueue_ingest(b, tp, st);
  if (r != C8R_OK) return r;
  for (const TuneChoice& c : cands) {
    b->choice = c;
    std::vector<WorkItem> v = make_items(b, c.a_tile, c.tiles_per_item, &b->n_items_split);
    const int min_items = 4 * batch_resident(b->formalism, b->M.kind, c.a_tile, b->sm_count);
    int lim = 0;
    double pairs = 0;
    while (lim < (int)v.size() && (pairs < 0.25 * (double)b->total_pairs || lim < min_items)) {
      pairs += (double)(v[lim].t_end - v[lim].t_begin) * kTileT * v[lim].n_here;
      ++lim;
    }
    r = upload_items(b, v);
    if (r != C8R_OK) return r;
    cudaEventRecord(e0, st);
    r = enqueue_kernel(b, lim, st);
    if (r != C8R_OK) return r;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return bfail(b, C8R_ECUDA, "autotuner timing failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double rate = ms > 0 ? pairs / ms : 0.0;
    if (rate > best_rate) {
      best_rate = rate;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->choice = best;
  b->tuned = true;
  // timings of kernels that gave up a bounded wait mean nothing: keep the
  // choice for this batch only (its status word stays set for c8r_batch_sync)
  int status = kErrNone;
  if (cudaMemcpy(&status, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && status == kErrNone)
    tune_store(key, best);
  return upload_items(b, make_items(b, best.a_tile, best.tiles_per_item, &b->n_items_split));
}

}  // namespace

extern "C" {

int c8r_batch_create(c8r_batch** out, int device, const c8r_batch_desc* d, int kind, double n_or_N0, double H) {
  if (!out || !d) return C8R_EINVAL;
  *out = nullptr;
  c8r_batch* b = new (std::nothrow) c8r_batch();
  if (!b) return C8R_ENOMEM;
  auto bad = [&](int code, const char* m) {
    b->err = m;
    *out = b;  // hand the object back so the caller can read the message
    return code;
  };
  if (d->n_showers < 1 || !d->n_tracks || !d->track_offset || !d->n_ant || !d->ant_offset || !d->pos_xyz ||
      !d->t_start_ns)
    return bad(C8R_EINVAL, "batch descriptor incomplete");
  if (d->n_bins < 1 || !(d->dt_ns > 0.0)) return bad(C8R_EINVAL, "n_bins / dt_ns");
  if (d->formalism != C8R_ENDPOINT && d->formalism != C8R_ZHS) return bad(C8R_EINVAL, "formalism");
  if (kind != C8R_UNIFORM && kind != C8R_EXPONENTIAL) return bad(C8R_EINVAL, "medium kind (uniform or exponential)");
  if (kind == C8R_UNIFORM ? !(n_or_N0 > 0.0) : !(n_or_N0 >= 0.0 && H > 0.0)) return bad(C8R_EINVAL, "medium");
  if (d->n_bins > (1 << 24)) return bad(C8R_ETOOBIG, "n_bins exceeds 2^24");
  if (cudaSetDevice(device) != cudaSuccess) return bad(C8R_EINVAL, "device");
  b->device = device;
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device);
  b->n_showers = d->n_showers;
  b->formalism = d->formalism;
  fill_medium(b->M, kind, n_or_N0, H, d->n_bins, d->dt_ns, 1e-3);
  b->n_tracks.assign(d->n_tracks, d->n_tracks + d->n_showers);
  b->track_off.assign(d->track_offset, d->track_offset + d->n_showers);
  b->n_ant.assign(d->n_ant, d->n_ant + d->n_showers);
  b->ant_off.assign(d->ant_offset, d->ant_offset + d->n_showers);
  b->tile_off.assign(d->n_showers + 1, 0);
  for (int s = 0; s < d->n_showers; ++s) {
    if (b->n_tracks[s] < 0 || b->n_ant[s] < 1 || b->track_off[s] < 0 || b->ant_off[s] < 0)
      return bad(C8R_EINVAL, "negative count/offset or shower without antennas");
    b->tile_off[s + 1] = b->tile_off[s] + (b->n_tracks[s] + kTileT - 1) / kTileT;
    b->total_tracks = std::max<int64_t>(b->total_tracks, b->track_off[s] + b->n_tracks[s]);
    b->total_ant = std::max<int>(b->total_ant, b->ant_off[s] + b->n_ant[s]);
    b->total_pairs += b->n_tracks[s] * (int64_t)b->n_ant[s];
  }
  b->total_tiles = b->tile_off[d->n_showers];
  set_flat_array(b->M, d->pos_xyz, b->total_ant);
  b->M.split = 1;
  b->cen.assign(3 * (size_t)b->n_showers, 0.0f);
  for (int s = 0; s < b->n_showers; ++s) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < b->n_ant[s]; ++a)
      for (int k = 0; k < 3; ++k) c[k] += d->pos_xyz[3 * (size_t)(b->ant_off[s] + a) + k];
    for (int k = 0; k < 3; ++k) b->cen[3 * (size_t)s + k] = (float)(c[k] / b->n_ant[s]);
  }
  std::vector<AntRec> recs(b->total_ant);
  for (int a = 0; a < b->total_ant; ++a) {
    const double* p = d->pos_xyz + 3 * (size_t)a;
    if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2]) || !std::isfinite(d->t_start_ns[a]))
      return bad(C8R_EINVAL, "antenna values must be finite");
    fill_antenna(recs[a], p[0], p[1], p[2], d->t_start_ns[a], b->M);
  }
  cudaError_t e = dev_malloc(&b->d_ants, sizeof(AntRec) * recs.size());
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ants, recs.data(), sizeof(AntRec) * recs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->total_tiles > 0) e = dev_malloc(&b->d_tiles, (size_t)b->total_tiles * kTileBytesMixed);
  const size_t sb = sizeof(int64_t) * (b->n_showers + 1);
  if (e == cudaSuccess) e = dev_malloc(&b->d_tile_off, sb);
  if (e == cudaSuccess) e = dev_malloc(&b->d_track_off, sb);
  if (e == cudaSuccess) e = dev_malloc(&b->d_n_tracks, sb);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tile_off, b->tile_off.data(), sb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_track_off, b->track_off.data(), sizeof(int64_t) * b->n_showers, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_n_tracks, b->n_tracks.data(), sizeof(int64_t) * b->n_showers, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dev_malloc(&b->d_counter, sizeof(int) * 8);
  if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, sizeof(int) * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->err = std::string("batch allocation: ") + cudaGetErrorString(e);
    *out = b;
    return C8R_ENOMEM;
  }
  b->d_cancel = b->d_counter + 1;
  b->d_err = b->d_counter + 2;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->aux_stream, cudaStreamNonBlocking) != cudaSuccess) {
    b->err = "stream creation failed";
    *out = b;
    return C8R_ECUDA;
  }
  b->replicas = acc_replicas(C8R_MIXED, b->formalism);
  b->acc_bytes = (size_t)b->total_ant * b->M.n_bins * sizeof(float4) * acc_rows(C8R_MIXED, b->formalism) *
                 b->replicas;
  if (dev_malloc(&b->d_acc, b->acc_bytes) != cudaSuccess) {
    cudaGetLastError();
    b->d_acc = nullptr;
    b->err = "batch accumulator allocation failed";
    *out = b;
    return C8R_ENOMEM;
  }
  b->choice = {8, tpi_for(b, 8, 8)};
  *out = b;
  return upload_items(b, make_items(b, b->choice.a_tile, b->choice.tiles_per_item, &b->n_items_split));
}

void c8r_batch_destroy(c8r_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->graph_src) cudaGraphDestroy(b->graph_src);
  cudaFree(b->d_ants);
  cudaFree(b->d_tiles);
  cudaFree(b->d_tile_off);
  cudaFree(b->d_track_off);
  cudaFree(b->d_n_tracks);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_acc);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->aux_stream) cudaStreamDestroy(b->aux_stream);
  delete b;
}

const char* c8r_batch_last_error(const c8r_batch* b) { return b ? b->err.c_str() : "batch is NULL"; }

int c8r_batch_run(c8r_batch* b, const c8r_tracks* t, float* out, int use_graph, void* stream) {
  if (!b || !t || !out) return bfail(b, C8R_EINVAL, "NULL argument");
  if (t->dtype != C8R_F32 && t->dtype != C8R_F64) return bfail(b, C8R_EINVAL, "tracks.dtype");
  const void* f[12] = {t->x0, t->y0, t->z0, t->x1, t->y1, t->z1, t->t0, t->t1, t->bx, t->by, t->bz, t->q};
  for (int k = 0; k < 12; ++k)
    if (!f[k]) return bfail(b, C8R_EINVAL, "a track array pointer is NULL");
  cudaSetDevice(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TrackPtrs tp;
  tp.dtype = t->dtype;
  for (int k = 0; k < 12; ++k) tp.f[k] = f[k];
  if (b->total_tiles == 0) return C8R_OK;
  if (!b->tuned) {
    int r = autotune(b, tp, st);
    if (r != C8R_OK) return r;
  }
  if (!use_graph) return enqueue(b, tp, out, b->n_items, st);
  bool same = b->graph && b->g_out == out;
  for (int k = 0; k < 12 && same; ++k) same = b->g_tracks[k] == f[k];
  if (!same) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_src) cudaGraphDestroy(b->graph_src);
    b->graph = nullptr;
    b->graph_src = nullptr;
    cudaStream_t cs = b->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    int r = enqueue(b, tp, out, b->n_items, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (r != C8R_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return bfail(b, C8R_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    b->graph_src = g;
    b->g_out = out;
    for (int k = 0; k < 12; ++k) b->g_tracks[k] = f[k];
  }
  cudaError_t e = cudaGraphLaunch(b->graph, st);
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return C8R_OK;
}

int c8r_batch_set_cancel(c8r_batch* b, int value) {
  if (!b) return C8R_EINVAL;
  cudaSetDevice(b->device);
  int v = value ? 1 : 0;
  cudaError_t e = cudaMemcpyAsync(b->d_cancel, &v, sizeof(int), cudaMemcpyHostToDevice, b->aux_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->aux_stream);
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("cancel word: ") + cudaGetErrorString(e));
  return C8R_OK;
}

int c8r_batch_sync(c8r_batch* b, void* stream) {
  if (!b) return C8R_EINVAL;
  cudaSetDevice(b->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("synchronise: ") + cudaGetErrorString(e));
  int err = 0;
  e = cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(b, C8R_ECUDA, std::string("read status: ") + cudaGetErrorString(e));
  if (err != kErrNone) {
    cudaMemset(b->d_err, 0, sizeof(int));
    return bfail(b, C8R_ECANCELLED,
                 err == kErrCancelled ? "batch cancelled: work items were skipped"
                                      : "a kernel gave up a bounded wait; results are incomplete");
  }
  return C8R_OK;
}

}  // extern "C"
