/*
 * c8r.h -- C ABI of the GB300 radio-emission library (libc8r).
 *
 * The library runs the step that the CORSIKA 8 radio module repeats for every
 * particle track and every antenna (paper §2: a track passes the track filter,
 * goes to the formalism, is looped over all antennas of the antenna collection,
 * fed to the propagator, and the result is stored in the antenna).  The two
 * formalisms are the ones the paper names in §1: "Endpoint" (CoREAS) and "ZHS".
 * The user-facing factories of §4 map onto it as follows:
 *
 *   make_simple_radio_propagator(environment)      -> c8r_set_medium
 *   make_radio_process_CoREAS/ZHS(detector, ...)   -> c8r_set_antennas
 *   RadioProcess receiving a track                 -> c8r_push_tracks
 *   reading the antenna instances                  -> c8r_fetch_traces
 *
 * Conventions for every call:
 *   - Return value: C8R_OK (0) or a negative C8R_E* code; c8r_last_error()
 *     then holds a one-line message.  No call aborts the process.
 *   - Units: metres and nanoseconds at the interface.  Traces hold the electric
 *     field in V/m (Endpoint) or the vector potential in V s/m (ZHS).
 *   - Ownership: the caller owns every pointer it passes; the library copies
 *     what it keeps (antenna table) and owns only its context's device memory
 *     (the trace accumulator and the derived-track scratch).
 *   - Asynchrony: calls that take a stream enqueue work on it and return; the
 *     caller's device buffers must stay valid until that work has run.  Copies
 *     into host memory synchronise the stream before returning.
 *   - Threads: a context is used by one host thread at a time.
 */
#ifndef C8R_H
#define C8R_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define C8R_OK 0
#define C8R_EINVAL (-1)     /* bad argument (size, pointer, non-finite value, call order) */
#define C8R_ENOMEM (-2)     /* device or host allocation failed                         */
#define C8R_ECUDA (-3)      /* a CUDA runtime call or kernel reported an error          */
#define C8R_ECANCELLED (-4) /* a kernel gave up a bounded wait and returned early       */
#define C8R_ETOOBIG (-5)    /* a size beyond the library's limits (n_bins > 2^24)       */
#define C8R_ESTATE (-6)     /* call made before the context was configured for it      */

/* medium kinds (straight-line propagator, §4 listing) */
#define C8R_UNIFORM 0      /* n constant                                              */
#define C8R_EXPONENTIAL 1  /* n(z) = 1 + N0 exp(-z / H), z = altitude in metres         */
#define C8R_EXPONENTIAL_SPHERICAL 2 /* the same over a spherical Earth (c8r_set_medium_spherical) */
#define C8R_EXPONENTIAL_RAY 3 /* flat exponential atmosphere with curved (refracted) rays        */

/* formalisms (§1) */
#define C8R_ENDPOINT 0
#define C8R_ZHS 1

/* arithmetic precision of a context */
#define C8R_FP64 0   /* all arithmetic in FP64; traces FP64                            */
#define C8R_MIXED 1  /* FP32 field arithmetic, compensated (float-float) arrival time,
                        bin index and interval ends; traces FP32                       */

/* element type of caller arrays */
#define C8R_F32 0
#define C8R_F64 1

/* deposit shapes (c8r_set_deposit) */
#define C8R_DEPOSIT_BIN 0     /* each deposit in the bin of its arrival time (default)    */
#define C8R_DEPOSIT_LINEAR 1  /* spread over one bin width centred on the arrival time    */

/* form of the FP32 arrival of the mixed one-bin Endpoint kernels (c8r_set_arrival_form) */
#define C8R_FORM_AUTO 0    /* chosen per push from earlier pushes' tracks (default)      */
#define C8R_FORM_SPLIT 1   /* lines of sight near the vertical                           */
#define C8R_FORM_DIRECT 2  /* inclined lines of sight                                    */

typedef struct c8r_ctx c8r_ctx;

/* Particle tracks in structure-of-arrays form: twelve DEVICE arrays of one
 * element type (dtype = C8R_F32 or C8R_F64), each of the length passed with them.
 * Track i runs in a straight line from (x0,y0,z0)[i] at time t0[i] to
 * (x1,y1,z1)[i] at t1[i] (m, ns) with velocity (bx,by,bz)[i] in units of c and
 * charge q[i] in units of e.  A C8R_MIXED context rounds FP64 input to FP32, so
 * times are best given as offsets from an epoch near the shower and positions
 * from a nearby origin: FP32 keeps ~7 digits (a time of 1e4 ns to ~1e-3 ns).
 * The mixed path carries each arrival in float-float (~48 bits): its bin
 * position is good to ~T x 2^-47 bins, T the largest of |t|/dt, |t_start|/dt
 * and the travel time in bins, so T up to ~1e8 keeps it below 1e-6 bin (the
 * edge band inside which either neighbouring bin is correct). */
typedef struct {
  int32_t dtype;
  const void *x0, *y0, *z0;
  const void *x1, *y1, *z1;
  const void *t0, *t1;
  const void *bx, *by, *bz;
  const void *q;
} c8r_tracks;

/* Gradients of a scalar loss with respect to each track's inputs: eleven DEVICE
 * arrays of one element type (C8R_F32 for a C8R_MIXED context, C8R_F64 for
 * C8R_FP64), each as long as the track arrays.  Units: per metre for positions,
 * per nanosecond for times, per unit of beta for the velocity. */
typedef struct {
  int32_t dtype;
  void *x0, *y0, *z0;
  void *x1, *y1, *z1;
  void *t0, *t1;
  void *bx, *by, *bz;
} c8r_track_grads;

typedef struct {
  int64_t tracks_pushed; /* tracks passed to c8r_push_tracks since creation/reset    */
  int64_t tracks_kept;   /* of those, tracks the track filter let through           */
  int64_t pairs;         /* kept tracks x antennas evaluated                         */
  int64_t arrival_form;  /* C8R_FORM_SPLIT or C8R_FORM_DIRECT: the FP32 arrival form the
                            next mixed one-bin Endpoint launch takes (c8r_set_arrival_form) */
} c8r_stats_t;

/* Writable DEVICE arrays for c8r_generate_tracks, one per track field. */
typedef struct {
  int32_t dtype; /* must be C8R_F32 */
  void *x0, *y0, *z0;
  void *x1, *y1, *z1;
  void *t0, *t1;
  void *bx, *by, *bz;
  void *q;
} c8r_tracks_out;

/* ---- lifecycle ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  *out is NULL on failure.
 * The context owns no trace memory until c8r_set_antennas. */
int c8r_create(c8r_ctx** out, int device);

/* Release a context and its device memory.  NULL is accepted.  The caller must
 * not destroy a context while work it enqueued may still be running. */
void c8r_destroy(c8r_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The pointer
 * stays valid until the next call on the context.  ctx == NULL gives the message
 * of the last failed c8r_create in this thread. */
const char* c8r_last_error(const c8r_ctx* ctx);

/* ---- configuration (the §4 factories) -------------------------------------- */

/* Medium of the straight-line propagator (§2 "propagator", §4
 * make_simple_radio_propagator).  kind = C8R_UNIFORM: n_or_N0 is the refractive
 * index n > 0, scale_height_m is ignored.  kind = C8R_EXPONENTIAL: n_or_N0 is the
 * refractivity N0 >= 0 at altitude 0 and scale_height_m is H > 0.
 * Along a straight path the propagator uses the path-averaged index for the
 * travel time and the index at the emission point in the Doppler factor.
 * kind = C8R_EXPONENTIAL_RAY (not in the paper; its "heavier" propagator): the
 * same atmosphere, with the signal following the refracted ray instead of the
 * straight line: the ray in the vertical plane through the emission point and
 * the antenna that keeps n(z) sin(theta) constant (Snell's law for horizontal
 * layers).  Its travel time and its direction at the emission point (for the
 * field vector and the Doppler factor) replace the straight line's; the
 * amplitude keeps the straight distance R.  Paths within 1e-3 of the horizontal
 * keep the straight line.  The adjoint, the batch runner and
 * c8r_traces_noalloc do not take this medium.
 * May be called before or after c8r_set_antennas; traces already accumulated
 * are kept.  EINVAL on non-finite or out-of-range values. */
int c8r_set_medium(c8r_ctx* ctx, int kind, double n_or_N0, double scale_height_m);

/* The exponential medium over a spherical Earth (an Earth-curvature option of the
 * straight-line propagator; the paper notes that the propagator's complexity sets
 * the cost of the step, §2): the Earth's centre is at (0, 0, -earth_radius_m),
 * the altitude of a point x is h(x) = |x - centre| - earth_radius_m and
 * n(x) = 1 + N0 exp(-h(x) / H).  The path stays straight; the travel time uses
 * the integral of n along it (the flat-atmosphere closed form plus an 8-point
 * Gauss-Legendre quadrature of the curvature correction), the Doppler factor
 * n at the emission point.  The adjoint (c8r_backward), the batched launch and
 * c8r_traces_noalloc do not take this medium (EINVAL).  EINVAL unless N0 >= 0,
 * H > 0 and earth_radius_m > 0 are finite.  Sets kind C8R_EXPONENTIAL_SPHERICAL. */
int c8r_set_medium_spherical(c8r_ctx* ctx, double N0, double scale_height_m, double earth_radius_m);

/* Antenna collection ("detector", §2, §4 make_radio_process_*).  pos_xyz: HOST
 * array [n_ant][3] of antenna positions (m); t_start_ns: HOST array [n_ant] of the
 * time of each trace's first bin edge (ns).  Every antenna records n_bins bins of
 * dt_ns, three components each; bin k of antenna a covers
 * [t_start_ns[a] + k dt_ns, t_start_ns[a] + (k + 1) dt_ns).  formalism selects
 * Endpoint or ZHS; precision selects C8R_FP64 or C8R_MIXED.  Allocates (and
 * zeroes) the context's trace accumulator, one (x, y, z) element per antenna and
 * bin, FP64 (C8R_FP64) or FP32 (C8R_MIXED), 32 or 16 bytes per element.  Mixed
 * ZHS keeps a second row per antenna (box edges), and the mixed path keeps 1 to
 * 8 copies of the whole accumulator, more for fewer antennas (up to 48 MB in
 * all), which the fetch sums.  Replaces
 * any previous antenna set and discards its traces (a call with the same
 * n_ant, n_bins, dt_ns, formalism and precision keeps the device memory and
 * only replaces the table, so moving an array between steps is cheap).  EINVAL on n_ant < 1,
 * n_bins < 1, dt_ns <= 0 or non-finite values; ETOOBIG if n_bins > 2^24; ENOMEM. */
int c8r_set_antennas(c8r_ctx* ctx, int32_t n_ant, const double* pos_xyz, const double* t_start_ns,
                     int32_t n_bins, double dt_ns, int formalism, int precision);

/* Threshold eps_C of the near-Cherenkov Endpoint treatment (default 1e-3): when
 * min(|D_start|, |D_end|) < eps_C, D = 1 - n beta.rhat, the pair is evaluated at
 * the track midpoint with linearised arrival times.  EINVAL unless 0 < eps < 1. */
int c8r_set_cherenkov_threshold(c8r_ctx* ctx, double eps_C);

/* Shape of every deposit (not in the paper; it leaves the binning open).
 * C8R_DEPOSIT_BIN (default): a deposit lands in the bin of its arrival time.
 * C8R_DEPOSIT_LINEAR: a deposit arriving at u bins from the window start is
 * spread evenly over [u - 1/2, u + 1/2], i.e. bins floor(u - 1/2) and the next
 * receive 1 - f and f of it, f = u - 1/2 - floor(u - 1/2).  ZHS intervals are
 * spread the same way (the weights are averaged over the interval); an Endpoint
 * pair near the Cherenkov angle whose two linearised arrivals lie between the
 * same two bin centres J - 1/2 and J + 1/2 deposits the exact limit
 * K (t1 - t0) V/(R dt^2) into bin J - 1 and its negative into bin J.  The traces
 * are then continuous in the arrival times, so c8r_backward gives the times
 * informative gradients.  Applies to the tracks pushed (and the adjoints run)
 * after the call; the batch runner and c8r_traces_noalloc use the one-bin
 * deposit.  EINVAL for another value. */
int c8r_set_deposit(c8r_ctx* ctx, int deposit);

/* Launch shape of the forward kernels: antennas per CTA (1..32; each thread
 * holds one track of a staged tile and evaluates it against all of them) and
 * the target number of waves per launch, a wave being every CTA the device
 * holds at once; it sets how many track ranges each antenna tile is cut into.
 * 0 keeps the automatic choice (32 antennas, 32 waves).  The result does not
 * depend on the shape beyond the order of floating-point additions (§5:
 * identical pulses for any number of threads).  Also sets the tracks per
 * internal chunk (0 = 2^25): longer pushes are processed chunk by chunk
 * through the same scratch.  EINVAL outside a_tile 0..32, waves 0..1024,
 * chunk_tracks >= 0. */
int c8r_set_launch_shape(c8r_ctx* ctx, int a_tile, int waves, int64_t chunk_tracks);

/* Form of the FP32 arrival with which the mixed-precision Endpoint kernels of
 * the one-bin deposit (uniform and exponential media) take each bin: the
 * arrival t_e/dt - t_a/dt + n R/(c dt) is evaluated as (T_e - T_a) + k x,
 * T = t/dt + k z formed once per track endpoint and per antenna, x = R - (z_e -
 * z_a), either as rho^2 / (R + z_e - z_a) (C8R_FORM_SPLIT: small errors for
 * emission points seen from the antenna near the vertical) or as R - (z_e -
 * z_a) (C8R_FORM_DIRECT: inclined lines of sight).  A bin is taken from the FP32
 * arrival only where its error bound leaves no bin edge in reach, otherwise
 * from the float-float arrival, so both forms give the same bins; the form only
 * sets how many arrivals need the float-float evaluation, i.e. the speed.
 * C8R_FORM_AUTO (default): the ingest of every push counts the tracks whose
 * start point sees the antenna array's centroid from above within 45 degrees,
 * the counts are copied back asynchronously, and later pushes and adjoints use
 * the split form when at least half of the tracks counted do (the split form
 * until a count has arrived; c8r_set_antennas with a new layout starts over).
 * Other precisions, media and deposits ignore the setting.  EINVAL for another
 * value. */
int c8r_set_arrival_form(c8r_ctx* ctx, int form);

/* ---- the hot path ----------------------------------------------------------- */

/* RadioProcess receiving tracks (§2 flow): for the n tracks, apply the track
 * filter (keep iff q != 0, all fields finite, t1 > t0, |x1 - x0| > 0 and
 * 0 < |beta| < 1), then for every kept track and every antenna run the
 * straight-line propagator, evaluate the formalism and add the result into the
 * antenna's trace.  ACCUMULATES into the context's traces.  Enqueued on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream).  The track arrays
 * must stay valid until the work has run.  n == 0 is a no-op.
 * EINVAL on NULL arrays or n < 0; ESTATE before c8r_set_antennas/c8r_set_medium. */
int c8r_push_tracks(c8r_ctx* ctx, const c8r_tracks* tracks, int64_t n, void* cuda_stream);

/* Copy the accumulated traces, layout [n_ant][3][n_bins] row-major, element type
 * FP64 (C8R_FP64 context) or FP32 (C8R_MIXED), into dst: a device pointer if
 * dst_is_device != 0, else host memory (the call then synchronises the stream).
 * reset != 0 zeroes the accumulator after the copy.  ESTATE before
 * c8r_set_antennas. */
int c8r_fetch_traces(c8r_ctx* ctx, void* dst, int dst_is_device, int reset, void* cuda_stream);

/* Zero the accumulated traces and the statistics. */
int c8r_reset(c8r_ctx* ctx, void* cuda_stream);

/* Adjoint of c8r_push_tracks (not in the paper; a hand-written reverse pass),
 * for both formalisms.  Given the same tracks and grad_traces = dL/dtraces
 * (DEVICE, layout and element type of c8r_fetch_traces), ACCUMULATES dL/d(track
 * inputs) into out_tracks (times per ns), dL/d(antenna positions) into
 * out_ant_grad (DEVICE FP64 [n_ant][3]) and dL/dN0 into *out_dN0 (DEVICE FP64
 * scalar; for a uniform medium the derivative with respect to n - 1).  Bin
 * indices and the near-Cherenkov branch are held fixed: with the one-bin
 * deposit the Endpoint deposits then do not depend on the times (zero time
 * gradients), while the ZHS deposits do, through the fractions of the arrival
 * interval in its first and last bin; with the linear deposit
 * (c8r_set_deposit) every deposit slides between its two bins with its arrival
 * time, so both formalisms give the times informative gradients.
 * The per-pair geometry is recomputed, not stored.  The first call allocates a
 * bin-major copy of grad_traces (and, for ZHS, its running sums over the bins)
 * inside the context (ENOMEM if that fails).  EINVAL for mismatched dtypes. */
int c8r_backward(c8r_ctx* ctx, const c8r_tracks* tracks, int64_t n, const void* grad_traces,
                 const c8r_track_grads* out_tracks, double* out_ant_grad, double* out_dN0, void* cuda_stream);

/* Kernel timing.  While enabled, every ingest and pair-kernel launch of
 * c8r_push_tracks is bracketed by CUDA events recorded on the launching stream.
 * c8r_profile_read synchronises and returns the summed device time (ms) and the
 * launch counts since profiling was enabled, then clears them. */
int c8r_profile(c8r_ctx* ctx, int enable);
int c8r_profile_read(c8r_ctx* ctx, double* pair_ms, int64_t* pair_launches, double* ingest_ms,
                     int64_t* ingest_launches);

/* Statistics since creation or the last reset.  Synchronises the context's last
 * stream.  Also reports (as ECANCELLED) a kernel that gave up a bounded wait. */
int c8r_stats(c8r_ctx* ctx, c8r_stats_t* out);

/* Per (track, antenna) arrival positions exactly as the kernels compute them,
 * for validation: branch[i*n_ant + a] = -1 (track filtered out), 0 (Endpoint,
 * two endpoints), 1 (Endpoint, near-Cherenkov midpoint), 2 (ZHS, one bin) or
 * 3 (ZHS, several bins); bin[2*(i*n_ant+a) + j] and frac[...] give the bin index
 * and the fractional position in the bin of the two arrival times (start/end,
 * the two linearised midpoint arrivals, or the ZHS interval ends).  All DEVICE
 * arrays.  Does not touch the traces. */
int c8r_arrivals(c8r_ctx* ctx, const c8r_tracks* tracks, int64_t n, int32_t* branch, int32_t* bin, float* frac,
                 void* cuda_stream);

/* ---- batched showers (not in the paper) -------------------------------------- */

/* Many independent showers of uneven size in persistent launches (one, or for
 * the Endpoint formalism one per form of the FP32 arrival its showers take,
 * see c8r_set_arrival_form; the form is chosen per shower).  Shower s
 * has n_tracks[s] tracks stored at offset track_offset[s] of the concatenated
 * track arrays, n_ant[s] antennas at offset ant_offset[s] of the concatenated
 * antenna arrays, and its traces at offset ant_offset[s]*3*n_bins of the
 * concatenated FP32 trace buffer.  All showers share the medium, n_bins, dt_ns
 * and formalism; precision is C8R_MIXED.  Host arrays are read during the call. */
typedef struct {
  int32_t n_showers;
  const int64_t* n_tracks;      /* HOST [n_showers]                            */
  const int64_t* track_offset;  /* HOST [n_showers]                            */
  const int32_t* n_ant;         /* HOST [n_showers]                            */
  const int32_t* ant_offset;    /* HOST [n_showers]                            */
  const double* pos_xyz;        /* HOST [sum n_ant][3], m                      */
  const double* t_start_ns;     /* HOST [sum n_ant], ns                        */
  int32_t n_bins;
  double dt_ns;
  int32_t formalism;
} c8r_batch_desc;

typedef struct c8r_batch c8r_batch;

/* Prepare a batch on `device` for the given layout and medium (kind, n_or_N0,
 * scale height as in c8r_set_medium): uploads the antenna tables, sizes the
 * scratch, builds the work list and picks the tile shape with the autotuner. */
int c8r_batch_create(c8r_batch** out, int device, const c8r_batch_desc* desc, int medium_kind, double n_or_N0,
                     double scale_height_m);
void c8r_batch_destroy(c8r_batch* b);
const char* c8r_batch_last_error(const c8r_batch* b);

/* Run the batch: tracks = concatenated DEVICE track arrays (FP32), traces_out =
 * DEVICE FP32 [sum n_ant][3][n_bins], ACCUMULATED.  use_graph != 0 replays a CUDA
 * graph captured on the first call (the capture happens on cuda_stream); the
 * graph is bound to the track and trace pointers of that first call and is
 * recaptured when they change. */
int c8r_batch_run(c8r_batch* b, const c8r_tracks* tracks, float* traces_out, int use_graph, void* cuda_stream);

/* Set (value != 0) or clear the batch's cancel word.  Persistent CTAs read it
 * before taking each work item and stop when it is set; c8r_batch_sync then
 * reports ECANCELLED.  Uses an internal non-blocking stream, so it can be called
 * while a batch runs.  The word stays set until cleared. */
int c8r_batch_set_cancel(c8r_batch* b, int value);

/* Synchronise cuda_stream and report the batch's status: ECANCELLED if the last
 * run was cancelled or a kernel gave up a bounded wait (the status is cleared). */
int c8r_batch_sync(c8r_batch* b, void* cuda_stream);

/* ---- forward pass without device allocation ------------------------------------ */

/* The paper has no counterpart to this entry point.  It is the mixed-precision
 * forward pass (c8r_push_tracks of a C8R_MIXED context) for callers that cannot
 * allocate device memory: code running inside another framework's allocator or
 * memory pool, code that may only touch memory it was handed, or services that
 * must not grow their device footprint after start-up.  It allocates nothing:
 * its scratch (the derived-track tiles of one chunk of 65536 tracks, 6.6 MB; an
 * antenna table of at most 1024 antennas, 96 KB; a status word) is a set of
 * fixed-size __device__ arrays that every GPU which loads the library holds until
 * the process exits.  Tracks are processed in chunks of 65536 through that
 * scratch, so n is not limited.
 *
 * Arguments as c8r_set_medium / c8r_set_antennas / c8r_push_tracks: tracks are
 * DEVICE arrays, pos_xyz [n_ant][3] (m) and t_start_ns [n_ant] are HOST arrays,
 * out_traces is a DEVICE FP32 array [n_ant][3][n_bins] that the call ACCUMULATES
 * into (zero it first for a fresh result).  The work runs on cuda_stream on the
 * current device, and the call synchronises that stream before it returns (it
 * reads the status word back).  Returns C8R_ETOOBIG if n_ant > 1024 or
 * n_bins > 2^24, C8R_EINVAL for other invalid arguments, C8R_ECUDA if a CUDA
 * call fails, and C8R_ECANCELLED if a kernel gave up a bounded wait on its
 * track pipeline and returned early (the traces are then incomplete).
 *
 * The first call on a device looks up the device addresses of the scratch
 * arrays (once per device, with that device current).  Every call on a device
 * shares the same scratch,
 * which keeps the last call's contents (the status word is cleared at the start
 * of each call): calls whose work overlaps on the GPU race, so issue them on one
 * stream or synchronise between them.  The antenna table is copied from pageable
 * host memory, which synchronises the stream before the copy. */
int c8r_traces_noalloc(const c8r_tracks* tracks, int64_t n, int32_t n_ant, const double* pos_xyz,
                       const double* t_start_ns, int32_t n_bins, double dt_ns, int formalism, int medium_kind,
                       double n_or_N0, double scale_height_m, float* out_traces, void* cuda_stream);

/* ---- test and diagnostic knobs (not in the paper) ------------------------------ */

/* Polls that each bounded wait of a forward, adjoint, batched or
 * allocation-free kernel makes on its staged track tile before it gives up
 * (the kernel then drains the copies it has in flight with the full limit,
 * sets its status word and returns, and the call reports C8R_ECANCELLED).
 * polls < 0 restores the default (2^22 polls); 0 makes every such wait give up
 * at once, which lets a test run the give-up path without a fault or a hang.
 * Process-wide; applies to kernels launched, and batch graphs captured, after
 * the call. */
int c8r_set_wait_limit(int64_t polls);

/* Fault injection on the host: of the library's next device allocations
 * (contexts, antenna state, derived-track scratch, adjoint and staging buffers,
 * batches), let `skip` through and make the following n fail as if the device
 * were out of memory, without calling the allocator.  The calls that make them
 * return C8R_ENOMEM, free what they had allocated and leave the context as it
 * was before the call (or unconfigured, for c8r_set_antennas).  n = 0 clears
 * it.  Process-wide.  EINVAL for a negative argument. */
int c8r_inject_alloc_failures(int32_t skip, int32_t n);

/* ---- synthetic showers generated on the device --------------------------------- */

/* Writes tracks first .. first+n-1 of the counter-based synthetic shower `seed`
 * into out (DEVICE FP32 arrays of length n), enqueued on cuda_stream.  The
 * shower is the one the tests and the benchmark use: start height
 * N(4 km, 1.5 km) truncated to [0.5, 10] km, lateral offset Exp(30 m) at a
 * uniform azimuth, direction -z tilted by N(0, 5 deg) about x and y, length
 * U[0.5, 5] m, gamma log-uniform in [10, 1e4], charge -1 (55 %) or +1, start
 * time (10 km - h)/c; the whole shower is rotated about y by zenith_deg.  Track g
 * is drawn from its own Philox4x32-10 blocks, counter (g, block, tag) and key
 * seed, so chunks of a shower can be generated independently (a stream of tracks
 * without a host-to-device copy; the paper's workload is a full shower, §5).
 * Not in the paper.  EINVAL on NULL arrays, n < 0, first < 0, a non-finite
 * zenith or dtype other than C8R_F32; ECUDA if the launch fails. */
int c8r_generate_tracks(uint64_t seed, int64_t first, int64_t n, double zenith_deg, const c8r_tracks_out* out,
                        void* cuda_stream);

/* ---- device peaks microbenchmark ----------------------------------------------- */

/* Measured issue rates on `device`, in operations per second: FP32 FMA, FP64 FMA,
 * MUFU reciprocal square root, FP32 shared-memory atomic add (scattered bins),
 * FP64 shared-memory atomic add (scattered bins), and global float4 vector
 * reductions (atomicAdd on float4) to scattered elements of a 32 MB
 * L2-resident buffer.  out_rates[6].  Runs for a few milliseconds; allocates
 * and frees its own device memory. */
int c8r_measure_peaks(int device, double* out_rates);

#ifdef __cplusplus
}
#endif

#endif /* C8R_H */
