// api.cu -- the C ABI of libc8r: context, configuration, validation and the
// launch sequence of the hot path (ingest -> forward) per chunk of tracks.
//
// Mapping to the paper (§4 listing): c8r_set_medium plays the role of
// make_simple_radio_propagator(environment), c8r_set_antennas that of
// make_radio_process_CoREAS/ZHS(detector, propagator, nthreads) (the thread
// count has no meaning here: the grid covers every track x antenna pair), and
// c8r_push_tracks that of the radio process receiving tracks (§2 flow).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace c8r {

static thread_local std::string g_create_error;

// polls of a bounded wait (c8r_set_wait_limit; < 0: kWaitLimit) and the
// injected allocation failures (c8r_inject_alloc_failures): allocations to let
// through first, then allocations to fail
static std::atomic<int64_t> g_wait_polls{-1};
static std::mutex g_alloc_mutex;
static int32_t g_alloc_skip = 0, g_alloc_fail = 0;

uint32_t current_wait_limit() {
  const int64_t v = g_wait_polls.load();
  return v < 0 ? kWaitLimit : (uint32_t)(v > (int64_t)kWaitLimit ? kWaitLimit : v);
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (g_alloc_fail > 0) {
      if (g_alloc_skip > 0) {
        --g_alloc_skip;
      } else {
        --g_alloc_fail;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
    }
  }
  return cudaMalloc(p, bytes);
}

void fill_medium(MedParams& M, int kind, double n_or_N0, double H, int n_bins, double dt_ns, double eps_C,
                 double earth_radius) {
  std::memset(&M, 0, sizeof(M));
  auto split = [](double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
  };
  M.kind = kind;
  M.n_bins = n_bins;
  M.wait_limit = kWaitLimit;
  M.dt_ns = dt_ns;
  M.inv_c_ns = 1.0 / kCns;
  M.eps_Cd = eps_C;
  M.eps_C = (float)eps_C;
  const double kc = 1.0 / (kCns * dt_ns);
  split(kc, M.kc_h, M.kc_l);
  split(1.0 / dt_ns, M.idt_h, M.idt_l);
  M.ampE = (float)(kKendpoint / (dt_ns * 1e-9));
  M.kzhs = (float)kKzhs;
  if (kind == C8R_UNIFORM) {
    M.n = n_or_N0;
    M.N0 = 0.0;
    M.H = 1.0;
    M.invH = 0.0;
    split(n_or_N0 * kc, M.s_h, M.s_l);
    M.nf = (float)n_or_N0;
    M.nm1f = (float)(n_or_N0 - 1.0);
  } else {
    M.n = 1.0;
    M.N0 = n_or_N0;
    M.H = H;
    M.invH = 1.0 / H;
    split(n_or_N0 * H * kc, M.cN_h, M.cN_l);
    split(1.0 / H, M.invH_h, M.invH_l);
    M.N0f = (float)n_or_N0;
    M.nf = 1.0f;
    M.R_E = earth_radius;
    M.RE_f = (float)earth_radius;
  }
}

void fill_antenna(AntRec& r, double x, double y, double z, double t_ref_ns, const MedParams& M) {
  std::memset(&r, 0, sizeof(r));
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  r.x = x;
  r.y = y;
  r.z = z;
  r.t_ref = t_ref_ns;
  r.Ea = (M.kind != C8R_UNIFORM) ? std::exp(-z / M.H) : 1.0;  // flat: the sphere's part comes per pair
  split(x, r.xh, r.xl);
  split(y, r.yh, r.yl);
  split(z, r.zh, r.zl);
  split(t_ref_ns / M.dt_ns, r.tauh, r.taul);
  split(r.Ea, r.Eah, r.Eal);
  // the antenna's shifted time of the FP32 arrival (arrival_fast): t_ref/dt +
  // k z with the same float-float k the kernels use (n/(c dt) in the uniform
  // medium, 1/(c dt) in the exponential one), at the exact altitude
  const double kff = M.kind == C8R_UNIFORM ? (double)M.s_h + (double)M.s_l : (double)M.kc_h + (double)M.kc_l;
  const double Ta = t_ref_ns / M.dt_ns + kff * z;
  split(Ta, r.Tah, r.Tal);
  // error-bound constants of the FP32 arrival (arrival_bin_fast): twice the
  // bins per metre (n/(c dt), or (1 + N0)/(c dt) as an upper bound for the
  // exponential medium) times the neglected low part of the position, 16 u^2
  // |T_a| (u = 2^-24) for the float-float shifted times, and a floor of 1e-6
  // bin; and the relative error of the refractivity term from the low part of
  // the altitude where the quotient is taken (|dz| > 1e-3 H)
  const double kc = 1.0 / (kCns * M.dt_ns);
  const double nmax = M.kind == C8R_UNIFORM ? M.n : 1.0 + M.N0;
  const double al = std::sqrt((double)r.xl * r.xl + (double)r.yl * r.yl + (double)r.zl * r.zl);
  const double u = 1.0 / 16777216.0;
  r.fb_abs = (float)(2.02 * nmax * kc * al + 16.0 * u * u * std::fabs(Ta) + 1e-6);
  r.fb_rel_v = M.kind == C8R_UNIFORM ? 0.0f : (float)(1.01 * std::fabs((double)r.zl) / (0.999e-3 * M.H));
}

void set_flat_array(MedParams& M, const double* pos_xyz, int n_ant) {
  M.flat = 0;
  if (M.kind != C8R_EXPONENTIAL || n_ant <= 0) return;
  const double z = pos_xyz[2];
  for (int a = 1; a < n_ant; ++a)
    if (pos_xyz[3 * (size_t)a + 2] != z) return;
  // split as fill_antenna splits the antennas' z and exp(-z/H)
  M.flat = 1;
  M.flat_zh = (float)z;
  M.flat_zl = (float)(z - (double)M.flat_zh);
  const double E = std::exp(-z / M.H);
  M.flat_Eh = (float)E;
  M.flat_El = (float)(E - (double)M.flat_Eh);
}

void set_form_centroid(MedParams& M, const double* pos_xyz, int n_ant) {
  double c[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < n_ant; ++a)
    for (int k = 0; k < 3; ++k) c[k] += pos_xyz[3 * (size_t)a + k];
  const double inv = n_ant > 0 ? 1.0 / n_ant : 0.0;
  M.cen_x = (float)(c[0] * inv);
  M.cen_y = (float)(c[1] * inv);
  M.cen_z = (float)(c[2] * inv);
}

// the default launch shape: 32 antennas per CTA, 32 waves (a sweep over
// 16-32 antennas and 8-32 waves on the 2e7-track, 160-antenna shower put it ~1.5 %
// ahead of 16 antennas and 8 waves for both formalisms)
constexpr int kDefaultATile = 32;
constexpr int kDefaultWaves = 32;
constexpr int kMaxBins = 1 << 24;

}  // namespace c8r

using namespace c8r;

struct c8r_ctx {
  int device = 0;
  int sm_count = 0;
  std::string err;
  // medium
  bool medium_set = false;
  int med_kind = C8R_UNIFORM;
  double med_a = 1.0, med_H = 1.0, med_RE = 0.0;
  double eps_C = 1e-3;
  int deposit = C8R_DEPOSIT_BIN;
  // antennas
  bool ants_set = false;
  int n_ant = 0, n_bins = 0, formalism = C8R_ENDPOINT, precision = C8R_MIXED;
  double dt_ns = 0.0;
  std::vector<double> pos, t_start;
  AntRec* d_ants = nullptr;
  void* d_acc = nullptr;     // accumulator [n_ant][n_bins][x, y, z, pad]
  size_t acc_bytes = 0;
  void* d_stage = nullptr;   // [n_ant][3][n_bins] staging for copies to host
  void* d_gbm = nullptr;     // backward: dL/dtraces, bin-major [n_ant][n_bins] accumulator elements
  PrefixFF* d_gpre = nullptr;  // backward (mixed ZHS): running sums of d_gbm over the bins, [n_ant][n_bins + 1]
  size_t trace_bytes = 0;
  // scratch: derived-track tiles for one chunk
  void* d_tiles = nullptr;
  int64_t tiles_cap = 0;      // tiles allocated
  int64_t chunk_tracks = (int64_t)1 << 25;
  // counters (device): kept tracks, then the two arrival-form votes of the
  // ingest (kept tracks, tracks seeing the array from above); error word
  unsigned long long* d_kept = nullptr;
  int* d_err = nullptr;
  // the arrival form of the one-bin Endpoint kernels (MedParams::split) and
  // the asynchronous read-back of the votes it is chosen from
  bool split = true;
  int form_mode = C8R_FORM_AUTO;         // c8r_set_arrival_form
  unsigned long long* h_form = nullptr;  // pinned: [kept tracks, seen from above]
  cudaEvent_t ev_form = nullptr;
  bool form_pending = false;
  int64_t pushed = 0;
  cudaStream_t last_stream = nullptr;
  FwdShape shape{1, 8};
  int user_a_tile = 0, user_waves = 0;
  // kernel timing (c8r_profile): event pairs of pair-kernel and ingest launches
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pair, ev_ingest;
  std::vector<cudaEvent_t> ev_pool;
  MedParams M{};
};

namespace {

int fail(c8r_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
int cuda_fail(c8r_ctx* c, cudaError_t e, const char* where) {
  return fail(c, C8R_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// the arrival form of the one-bin Endpoint kernels (MedParams::split), from the
// ingest's votes of earlier pushes: the split form when at least half of the
// tracks counted see the antenna array's centroid from above within 45
// degrees.  The votes are copied to pinned memory after a push and read once
// the copy has landed, so no launch waits for them; both forms give the same
// bins, the choice only sets the speed.
void form_poll(c8r_ctx* c) {
  if (c->form_mode != C8R_FORM_AUTO) {
    c->split = c->form_mode == C8R_FORM_SPLIT;
    c->M.split = c->split ? 1 : 0;
    return;
  }
  if (!c->form_pending) return;
  const cudaError_t q = cudaEventQuery(c->ev_form);
  if (q == cudaErrorNotReady) {
    if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
    return;
  }
  c->form_pending = false;
  if (q != cudaSuccess || c->h_form[0] == 0) return;
  c->split = 2 * c->h_form[1] >= c->h_form[0];
  c->M.split = c->split ? 1 : 0;
}

void form_fetch(c8r_ctx* c, cudaStream_t st) {
  if (c->form_mode != C8R_FORM_AUTO || c->form_pending || !c->h_form || !c->ev_form || c->precision != C8R_MIXED)
    return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  if (cudaMemcpyAsync(c->h_form, c->d_kept + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaEventRecord(c->ev_form, st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c->form_pending = true;
}

// a new antenna layout or medium: earlier votes no longer apply
void form_reset(c8r_ctx* c) {
  if (c->form_pending) cudaEventSynchronize(c->ev_form);
  c->form_pending = false;
  cudaMemset(c->d_kept + 1, 0, 2 * sizeof(unsigned long long));
  c->split = c->form_mode != C8R_FORM_DIRECT;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

int rebuild_tables(c8r_ctx* c) {
  if (!c->ants_set) return C8R_OK;
  fill_medium(c->M, c->med_kind, c->med_a, c->med_H, c->n_bins, c->dt_ns, c->eps_C, c->med_RE);
  set_form_centroid(c->M, c->pos.data(), c->n_ant);
  set_flat_array(c->M, c->pos.data(), c->n_ant);
  c->M.split = c->split ? 1 : 0;
  std::vector<AntRec> recs(c->n_ant);
  for (int a = 0; a < c->n_ant; ++a)
    fill_antenna(recs[a], c->pos[3 * a], c->pos[3 * a + 1], c->pos[3 * a + 2], c->t_start[a], c->M);
  cudaError_t e = cudaMemcpy(c->d_ants, recs.data(), sizeof(AntRec) * c->n_ant, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "upload antenna table");
  return C8R_OK;
}

void free_antenna_state(c8r_ctx* c) {
  if (c->d_ants) cudaFree(c->d_ants);
  if (c->d_acc) cudaFree(c->d_acc);
  if (c->d_stage) cudaFree(c->d_stage);
  if (c->d_gbm) cudaFree(c->d_gbm);
  c->d_gbm = nullptr;
  if (c->d_gpre) cudaFree(c->d_gpre);
  c->d_gpre = nullptr;
  c->d_ants = nullptr;
  c->d_acc = nullptr;
  c->d_stage = nullptr;
  c->ants_set = false;
}

int ensure_tiles(c8r_ctx* c, int64_t n_tracks) {
  int64_t need = (n_tracks + kTileT - 1) / kTileT;
  if (need <= c->tiles_cap) return C8R_OK;
  if (c->d_tiles) cudaFree(c->d_tiles);
  c->d_tiles = nullptr;
  c->tiles_cap = 0;
  size_t bytes = (size_t)need * tile_bytes(c->precision);
  cudaError_t e = dev_malloc(&c->d_tiles, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, C8R_ENOMEM, "cudaMalloc of the derived-track scratch (" + std::to_string(bytes) + " bytes) failed");
  }
  c->tiles_cap = need;
  return C8R_OK;
}

int check_tracks(c8r_ctx* c, const c8r_tracks* t, int64_t n) {
  if (!t) return fail(c, C8R_EINVAL, "tracks is NULL");
  if (n < 0) return fail(c, C8R_EINVAL, "negative track count");
  if (t->dtype != C8R_F32 && t->dtype != C8R_F64) return fail(c, C8R_EINVAL, "tracks.dtype must be C8R_F32 or C8R_F64");
  if (n == 0) return C8R_OK;
  const void* f[12] = {t->x0, t->y0, t->z0, t->x1, t->y1, t->z1, t->t0, t->t1, t->bx, t->by, t->bz, t->q};
  for (int k = 0; k < 12; ++k)
    if (!f[k]) return fail(c, C8R_EINVAL, "a track array pointer is NULL");
  return C8R_OK;
}

TrackPtrs offset_tracks(const c8r_tracks* t, int64_t off) {
  TrackPtrs p;
  p.dtype = t->dtype;
  const size_t es = t->dtype == C8R_F64 ? 8 : 4;
  const void* f[12] = {t->x0, t->y0, t->z0, t->x1, t->y1, t->z1, t->t0, t->t1, t->bx, t->by, t->bz, t->q};
  for (int k = 0; k < 12; ++k) p.f[k] = static_cast<const char*>(f[k]) + off * es;
  return p;
}

cudaEvent_t take_event(c8r_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int ready(c8r_ctx* c) {
  if (!c) return C8R_EINVAL;
  if (!c->ants_set) return fail(c, C8R_ESTATE, "c8r_set_antennas has not been called");
  if (!c->medium_set) return fail(c, C8R_ESTATE, "c8r_set_medium has not been called");
  return C8R_OK;
}

}  // namespace

extern "C" {

int c8r_create(c8r_ctx** out, int device) {
  if (!out) {
    g_create_error = "out is NULL";
    return C8R_EINVAL;
  }
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    g_create_error = std::string("no CUDA device ") + std::to_string(device) + " (" +
                     (e == cudaSuccess ? "out of range" : cudaGetErrorString(e)) + ")";
    return C8R_EINVAL;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return C8R_ECUDA;
  }
  c8r_ctx* c = new (std::nothrow) c8r_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return C8R_ENOMEM;
  }
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  e = dev_malloc(&c->d_kept, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = dev_malloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_kept, 0, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    g_create_error = std::string("context allocation: ") + cudaGetErrorString(e);
    c8r_destroy(c);
    return C8R_ENOMEM;
  }
  // the read-back of the arrival-form votes is an optimisation: without its
  // pinned buffer or event the split form stays chosen
  if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_form), 2 * sizeof(unsigned long long), cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_form, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (c->h_form) cudaFreeHost(c->h_form);
    c->h_form = nullptr;
    c->ev_form = nullptr;
  }
  *out = c;
  return C8R_OK;
}

void c8r_destroy(c8r_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (auto& pr : c->ev_ingest) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto& pr : c->ev_pair) cudaEventDestroy(pr.second);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  free_antenna_state(c);
  if (c->d_tiles) cudaFree(c->d_tiles);
  if (c->d_kept) cudaFree(c->d_kept);
  if (c->d_err) cudaFree(c->d_err);
  if (c->form_pending) cudaEventSynchronize(c->ev_form);  // the votes' copy lands before its buffer goes
  if (c->ev_form) cudaEventDestroy(c->ev_form);
  if (c->h_form) cudaFreeHost(c->h_form);
  delete c;
}

const char* c8r_last_error(const c8r_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int c8r_set_medium(c8r_ctx* c, int kind, double n_or_N0, double H) {
  if (!c) return C8R_EINVAL;
  if (kind == C8R_UNIFORM) {
    if (!std::isfinite(n_or_N0) || !(n_or_N0 > 0.0)) return fail(c, C8R_EINVAL, "uniform medium needs finite n > 0");
  } else if (kind == C8R_EXPONENTIAL || kind == C8R_EXPONENTIAL_RAY) {
    if (!std::isfinite(n_or_N0) || n_or_N0 < 0.0) return fail(c, C8R_EINVAL, "exponential medium needs finite N0 >= 0");
    if (!std::isfinite(H) || !(H > 0.0)) return fail(c, C8R_EINVAL, "exponential medium needs finite H > 0");
  } else if (kind == C8R_EXPONENTIAL_SPHERICAL) {
    return fail(c, C8R_EINVAL, "the spherical-Earth medium is set with c8r_set_medium_spherical");
  } else {
    return fail(c, C8R_EINVAL, "unknown medium kind");
  }
  cudaSetDevice(c->device);
  c->med_kind = kind;
  c->med_a = n_or_N0;
  c->med_H = H;
  c->med_RE = 0.0;
  c->medium_set = true;
  return rebuild_tables(c);
}

int c8r_set_medium_spherical(c8r_ctx* c, double N0, double H, double RE) {
  if (!c) return C8R_EINVAL;
  if (!std::isfinite(N0) || N0 < 0.0) return fail(c, C8R_EINVAL, "spherical medium needs finite N0 >= 0");
  if (!std::isfinite(H) || !(H > 0.0)) return fail(c, C8R_EINVAL, "spherical medium needs finite H > 0");
  if (!std::isfinite(RE) || !(RE > 0.0)) return fail(c, C8R_EINVAL, "spherical medium needs a finite Earth radius > 0");
  cudaSetDevice(c->device);
  c->med_kind = C8R_EXPONENTIAL_SPHERICAL;
  c->med_a = N0;
  c->med_H = H;
  c->med_RE = RE;
  c->medium_set = true;
  return rebuild_tables(c);
}

int c8r_set_cherenkov_threshold(c8r_ctx* c, double eps) {
  if (!c) return C8R_EINVAL;
  if (!std::isfinite(eps) || !(eps > 0.0 && eps < 1.0)) return fail(c, C8R_EINVAL, "eps_C must be in (0, 1)");
  c->eps_C = eps;
  cudaSetDevice(c->device);
  return rebuild_tables(c);
}

int c8r_set_deposit(c8r_ctx* c, int deposit) {
  if (!c) return C8R_EINVAL;
  if (deposit != C8R_DEPOSIT_BIN && deposit != C8R_DEPOSIT_LINEAR)
    return fail(c, C8R_EINVAL, "deposit must be C8R_DEPOSIT_BIN or C8R_DEPOSIT_LINEAR");
  c->deposit = deposit;
  return C8R_OK;
}

int c8r_set_antennas(c8r_ctx* c, int32_t n_ant, const double* pos, const double* t_start, int32_t n_bins,
                     double dt_ns, int formalism, int precision) {
  if (!c) return C8R_EINVAL;
  if (n_ant < 1) return fail(c, C8R_EINVAL, "n_ant must be >= 1");
  if (n_bins < 1) return fail(c, C8R_EINVAL, "n_bins must be >= 1");
  if (!pos || !t_start) return fail(c, C8R_EINVAL, "antenna arrays are NULL");
  if (!std::isfinite(dt_ns) || !(dt_ns > 0.0)) return fail(c, C8R_EINVAL, "dt_ns must be finite and > 0");
  if (formalism != C8R_ENDPOINT && formalism != C8R_ZHS) return fail(c, C8R_EINVAL, "unknown formalism");
  if (precision != C8R_FP64 && precision != C8R_MIXED) return fail(c, C8R_EINVAL, "unknown precision");
  if (!finite_all(pos, 3 * (size_t)n_ant) || !finite_all(t_start, n_ant))
    return fail(c, C8R_EINVAL, "antenna positions / start times must be finite");
  if (n_bins > kMaxBins) return fail(c, C8R_ETOOBIG, "n_bins = " + std::to_string(n_bins) + " exceeds 2^24");
  cudaSetDevice(c->device);
  if (c->ants_set && n_ant == c->n_ant && n_bins == c->n_bins && formalism == c->formalism &&
      precision == c->precision && dt_ns == c->dt_ns) {
    // the same layout (an antenna array being moved, e.g. by an optimiser):
    // keep the device memory, replace the table and discard the traces
    c->pos.assign(pos, pos + 3 * (size_t)n_ant);
    c->t_start.assign(t_start, t_start + n_ant);
    cudaError_t e = cudaMemset(c->d_acc, 0, c->acc_bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "trace reset");
    c->pushed = 0;
    cudaMemset(c->d_kept, 0, sizeof(unsigned long long));
    return rebuild_tables(c);
  }
  free_antenna_state(c);
  if (c->precision != precision && c->d_tiles) {
    cudaFree(c->d_tiles);
    c->d_tiles = nullptr;
    c->tiles_cap = 0;
  }
  c->n_ant = n_ant;
  c->n_bins = n_bins;
  c->dt_ns = dt_ns;
  c->formalism = formalism;
  c->precision = precision;
  c->pos.assign(pos, pos + 3 * (size_t)n_ant);
  c->t_start.assign(t_start, t_start + n_ant);
  const int want = c->user_a_tile > 0 ? c->user_a_tile : kDefaultATile;
  c->shape.a_tile = want < n_ant ? want : n_ant;
  c->shape.waves = c->user_waves > 0 ? c->user_waves : kDefaultWaves;
  c->trace_bytes = (size_t)n_ant * 3 * n_bins * (precision == C8R_FP64 ? 8 : 4);
  c->acc_bytes = (size_t)n_ant * n_bins * acc_elem_bytes(precision) * acc_rows(precision, formalism);
  c->shape.replicas = acc_replicas(precision, formalism, n_ant, n_bins, c->shape.a_tile, c->sm_count);
  c->acc_bytes *= c->shape.replicas;
  cudaError_t e = dev_malloc(&c->d_ants, sizeof(AntRec) * n_ant);
  if (e == cudaSuccess) e = dev_malloc(&c->d_acc, c->acc_bytes);
  if (e == cudaSuccess) e = cudaMemset(c->d_acc, 0, c->acc_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_antenna_state(c);
    return fail(c, C8R_ENOMEM, std::string("antenna state allocation: ") + cudaGetErrorString(e));
  }
  c->ants_set = true;
  c->pushed = 0;
  cudaMemset(c->d_kept, 0, sizeof(unsigned long long));
  form_reset(c);
  return rebuild_tables(c);
}

int c8r_set_launch_shape(c8r_ctx* c, int a_tile, int waves, int64_t chunk_tracks) {
  if (!c) return C8R_EINVAL;
  if (a_tile < 0 || a_tile > kMaxATile || waves < 0 || waves > 1024 || chunk_tracks < 0)
    return fail(c, C8R_EINVAL, "launch shape out of range");
  c->user_a_tile = a_tile;
  c->user_waves = waves;
  c->chunk_tracks = chunk_tracks > 0 ? chunk_tracks : (int64_t)1 << 25;
  if (c->ants_set) {
    const int want = a_tile > 0 ? a_tile : kDefaultATile;
    c->shape.a_tile = want < c->n_ant ? want : c->n_ant;
    c->shape.waves = waves > 0 ? waves : kDefaultWaves;
  }
  return C8R_OK;
}

int c8r_set_arrival_form(c8r_ctx* c, int form) {
  if (!c) return C8R_EINVAL;
  if (form != C8R_FORM_AUTO && form != C8R_FORM_SPLIT && form != C8R_FORM_DIRECT)
    return fail(c, C8R_EINVAL, "unknown arrival form");
  c->form_mode = form;
  if (form != C8R_FORM_AUTO) {
    c->split = form == C8R_FORM_SPLIT;
    c->M.split = c->split ? 1 : 0;
  }
  return C8R_OK;
}

int c8r_push_tracks(c8r_ctx* c, const c8r_tracks* t, int64_t n, void* stream) {
  int r = ready(c);
  if (r != C8R_OK) return r;
  if ((r = check_tracks(c, t, n)) != C8R_OK) return r;
  if (n == 0) return C8R_OK;
  cudaSetDevice(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->last_stream = st;
  const int64_t chunk = n < c->chunk_tracks ? n : c->chunk_tracks;
  if ((r = ensure_tiles(c, chunk)) != C8R_OK) return r;
  const bool lin = c->deposit == C8R_DEPOSIT_LINEAR;
  form_poll(c);
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t m = (n - off) < chunk ? (n - off) : chunk;
    TrackPtrs p = offset_tracks(t, off);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (c->profiling) {
      e0 = take_event(c);
      e1 = take_event(c);
      e2 = take_event(c);
      cudaEventRecord(e0, st);
    }
    cudaError_t e = launch_ingest(c->precision, p, m, c->d_tiles, c->M, c->d_kept, st, c->d_kept + 1);
    if (e != cudaSuccess) return cuda_fail(c, e, "ingest launch");
    if (c->profiling) cudaEventRecord(e1, st);
    const int64_t n_tiles = (m + kTileT - 1) / kTileT;
    MedParams M = c->M;
    M.wait_limit = current_wait_limit();
    e = (c->precision == C8R_FP64)
            ? launch_forward_f64(c->formalism, lin, c->d_tiles, n_tiles, c->d_ants, c->n_ant, M, c->d_acc,
                                 c->shape, c->sm_count, c->d_err, st)
            : launch_forward_mixed(c->formalism, lin, c->d_tiles, n_tiles, c->d_ants, c->n_ant, M, c->d_acc,
                                   c->shape, c->sm_count, c->d_err, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "forward launch");
    if (c->profiling) {
      cudaEventRecord(e2, st);
      c->ev_ingest.push_back({e0, e1});
      c->ev_pair.push_back({e1, e2});
    }
  }
  form_fetch(c, st);
  c->pushed += n;
  return C8R_OK;
}

static cudaError_t fetch_acc(c8r_ctx* c, void* dst, cudaStream_t st) {
  return launch_acc_to_traces(c->precision, c->d_acc, c->n_ant, c->n_bins, acc_rows(c->precision, c->formalism), dst,
                              0, st, c->shape.replicas);
}

int c8r_fetch_traces(c8r_ctx* c, void* dst, int dst_is_device, int reset, void* stream) {
  if (!c) return C8R_EINVAL;
  if (!c->ants_set) return fail(c, C8R_ESTATE, "c8r_set_antennas has not been called");
  if (!dst) return fail(c, C8R_EINVAL, "dst is NULL");
  cudaSetDevice(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dst_is_device) {
    e = fetch_acc(c, dst, st);
  } else {
    if (!c->d_stage) {
      e = dev_malloc(&c->d_stage, c->trace_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        c->d_stage = nullptr;
        return fail(c, C8R_ENOMEM, "staging buffer for the host copy");
      }
    }
    e = fetch_acc(c, c->d_stage, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, c->d_stage, c->trace_bytes, cudaMemcpyDeviceToHost, st);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "trace copy");
  if (reset) {
    e = cudaMemsetAsync(c->d_acc, 0, c->acc_bytes, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "trace reset");
  }
  if (!dst_is_device) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  }
  return C8R_OK;
}

int c8r_reset(c8r_ctx* c, void* stream) {
  if (!c) return C8R_EINVAL;
  if (!c->ants_set) return fail(c, C8R_ESTATE, "c8r_set_antennas has not been called");
  cudaSetDevice(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(c->d_acc, 0, c->acc_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_kept, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset");
  c->pushed = 0;
  return C8R_OK;
}

int c8r_profile(c8r_ctx* c, int enable) {
  if (!c) return C8R_EINVAL;
  c->profiling = enable != 0;
  return C8R_OK;
}

int c8r_profile_read(c8r_ctx* c, double* pair_ms, int64_t* pair_launches, double* ingest_ms,
                     int64_t* ingest_launches) {
  if (!c || !pair_ms || !pair_launches || !ingest_ms || !ingest_launches) return fail(c, C8R_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  double pm = 0.0, im = 0.0;
  cudaError_t err = cudaSuccess;
  for (auto& pr : c->ev_pair) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) err = e;
    pm += ms;
  }
  for (auto& pr : c->ev_ingest) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess) err = e;
    im += ms;
  }
  *pair_ms = pm;
  *ingest_ms = im;
  *pair_launches = (int64_t)c->ev_pair.size();
  *ingest_launches = (int64_t)c->ev_ingest.size();
  // return the events to the pool: ingest pairs own (e0, e1), pair launches own e2
  for (auto& pr : c->ev_ingest) {
    c->ev_pool.push_back(pr.first);
    c->ev_pool.push_back(pr.second);
  }
  for (auto& pr : c->ev_pair) c->ev_pool.push_back(pr.second);
  c->ev_pair.clear();
  c->ev_ingest.clear();
  if (err != cudaSuccess) return cuda_fail(c, err, "profile events");
  return C8R_OK;
}

int c8r_stats(c8r_ctx* c, c8r_stats_t* out) {
  if (!c || !out) return fail(c, C8R_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  unsigned long long kept = 0;
  int err = 0;
  e = cudaMemcpy(&kept, c->d_kept, sizeof(kept), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&err, c->d_err, sizeof(err), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read counters");
  out->tracks_pushed = c->pushed;
  out->tracks_kept = (int64_t)kept;
  out->pairs = (int64_t)kept * c->n_ant;
  // the stream has drained: the votes' copy, if one was made, has landed
  if (c->form_pending) cudaEventSynchronize(c->ev_form);
  form_poll(c);
  out->arrival_form = c->split ? C8R_FORM_SPLIT : C8R_FORM_DIRECT;
  if (err != kErrNone) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return fail(c, C8R_ECANCELLED, "a kernel gave up a bounded wait on its track pipeline; results are incomplete");
  }
  return C8R_OK;
}

int c8r_arrivals(c8r_ctx* c, const c8r_tracks* t, int64_t n, int32_t* branch, int32_t* bin, float* frac,
                 void* stream) {
  int r = ready(c);
  if (r != C8R_OK) return r;
  if ((r = check_tracks(c, t, n)) != C8R_OK) return r;
  if (n == 0) return C8R_OK;
  if (!branch || !bin || !frac) return fail(c, C8R_EINVAL, "output arrays are NULL");
  cudaSetDevice(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->last_stream = st;
  const int64_t chunk = n < c->chunk_tracks ? n : c->chunk_tracks;
  if ((r = ensure_tiles(c, chunk)) != C8R_OK) return r;
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t m = (n - off) < chunk ? (n - off) : chunk;
    const int64_t j0 = off * c->n_ant;
    cudaError_t e = launch_ingest(c->precision, offset_tracks(t, off), m, c->d_tiles, c->M, nullptr, st);
    if (e == cudaSuccess)
      e = (c->precision == C8R_FP64)
              ? launch_arrivals_f64(c->formalism, c->d_tiles, m, c->d_ants, c->n_ant, c->M, branch + j0,
                                    bin + 2 * j0, frac + 2 * j0, st)
              : launch_arrivals_mixed(c->formalism, c->d_tiles, m, c->d_ants, c->n_ant, c->M, branch + j0,
                                      bin + 2 * j0, frac + 2 * j0, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "arrivals launch");
  }
  return C8R_OK;
}

int c8r_backward(c8r_ctx* c, const c8r_tracks* t, int64_t n, const void* grad_traces, const c8r_track_grads* out,
                 double* ant_grad, double* dN0, void* stream) {
  int r = ready(c);
  if (r != C8R_OK) return r;
  if ((r = check_tracks(c, t, n)) != C8R_OK) return r;
  if (c->med_kind == C8R_EXPONENTIAL_SPHERICAL || c->med_kind == C8R_EXPONENTIAL_RAY)
    return fail(c, C8R_EINVAL, "c8r_backward does not take the spherical-Earth medium or curved rays");
  if (!grad_traces || !out || !ant_grad || !dN0) return fail(c, C8R_EINVAL, "NULL gradient pointer");
  const int want = c->precision == C8R_FP64 ? C8R_F64 : C8R_F32;
  if (out->dtype != want) return fail(c, C8R_EINVAL, "out_tracks.dtype must match the context precision");
  if (n == 0) return C8R_OK;
  const bool lin = c->deposit == C8R_DEPOSIT_LINEAR;
  void* g[11] = {out->x0, out->y0, out->z0, out->x1, out->y1, out->z1, out->t0, out->t1, out->bx, out->by, out->bz};
  for (int k = 0; k < 11; ++k)
    if (!g[k]) return fail(c, C8R_EINVAL, "a gradient array pointer is NULL");
  cudaSetDevice(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->last_stream = st;
  const int64_t chunk = n < c->chunk_tracks ? n : c->chunk_tracks;
  if ((r = ensure_tiles(c, chunk)) != C8R_OK) return r;
  const size_t es = want == C8R_F64 ? 8 : 4;
  if (!c->d_gbm) {
    cudaError_t e = dev_malloc(&c->d_gbm, (size_t)c->n_ant * c->n_bins * acc_elem_bytes(c->precision));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->d_gbm = nullptr;
      return fail(c, C8R_ENOMEM, "backward gradient buffer");
    }
  }
  const bool prefix = c->formalism == C8R_ZHS && c->precision == C8R_MIXED;  // the FP64 adjoint sums bin by bin
  if (prefix && !c->d_gpre) {
    cudaError_t e = dev_malloc(&c->d_gpre, (size_t)c->n_ant * (c->n_bins + 1) * sizeof(PrefixFF));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->d_gpre = nullptr;
      return fail(c, C8R_ENOMEM, "backward running-sum buffer");
    }
  }
  {
    cudaError_t e = launch_traces_to_bin_major(c->precision, grad_traces, c->n_ant, c->n_bins, c->d_gbm, st);
    if (e == cudaSuccess && prefix) e = launch_bin_running_sums(c->d_gbm, c->n_ant, c->n_bins, c->d_gpre, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient layout");
  }
  form_poll(c);
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t m = (n - off) < chunk ? (n - off) : chunk;
    cudaError_t e = launch_ingest(c->precision, offset_tracks(t, off), m, c->d_tiles, c->M, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "ingest launch");
    c8r_track_grads o = *out;
    void** og[11] = {&o.x0, &o.y0, &o.z0, &o.x1, &o.y1, &o.z1, &o.t0, &o.t1, &o.bx, &o.by, &o.bz};
    for (int k = 0; k < 11; ++k) *og[k] = static_cast<char*>(*og[k]) + off * es;
    BwdArgs ba{c->d_tiles, m, (m + kTileT - 1) / kTileT, c->d_ants, c->n_ant, c->shape.a_tile, c->d_gbm,
               prefix ? c->d_gpre : nullptr, o, ant_grad, dN0, c->d_err, FwdGrid{}, c->M};
    ba.M.wait_limit = current_wait_limit();
    e = (c->precision == C8R_FP64) ? launch_backward_f64(c->formalism, lin, ba, c->shape, c->sm_count, st)
                                   : launch_backward_mixed(c->formalism, lin, ba, c->shape, c->sm_count, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "backward launch");
  }
  return C8R_OK;
}

int c8r_set_wait_limit(int64_t polls) {
  g_wait_polls.store(polls < 0 ? -1 : polls);
  return C8R_OK;
}

int c8r_inject_alloc_failures(int32_t skip, int32_t n) {
  if (skip < 0 || n < 0) return C8R_EINVAL;
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  g_alloc_skip = skip;
  g_alloc_fail = n;
  return C8R_OK;
}

}  // extern "C"
