// pair_mixed.cuh -- per (track, antenna) arithmetic of the mixed-precision path.
//
// FP32 field arithmetic; the arrival time, the bin index and the ends of the
// arrival interval are float-float (about 48 significant bits), which keeps the
// bin of every deposit identical to an FP64 evaluation except within ~1e-7 bin
// of an edge.  The Doppler factor D = 1 - n beta.rhat is formed without the
// cancellation of the direct form (see field_mixed), from 1 - |beta| computed
// per track in FP64 by the ingest kernel.
//
// A thread loads one track of a staged tile into registers (TrackM) once and
// then evaluates it against every antenna of the CTA's antenna tile.
#pragma once

#include "kernels.cuh"

namespace c8r {

// track fields of lane l in a field-major tile
#define TF(f) T[(f) * kTileT + l]

// one track, held in registers while it is evaluated against the antennas
struct TrackM {
  float x0, y0, z0, x1, y1, z1;  // FP32-exact endpoints
  float bx, by, bz, bmag;
  float amp;                     // q K/dt (Endpoint) or q K_A (t1-t0)/dt (ZHS); 0 = dropped
  float tau0h, tau0l, tau1h, tau1l, dtauh, dtaul;
  float T0h, T0l, T1h, T1l;      // Endpoint, plain media: tau + k z at start and end (arrival_fast)
  // a flat antenna array (MedParams::flat, exponential medium): the quotient of
  // the refractivity term, the same for every antenna, per track: FP32 at start
  // and end (Endpoint, arrival_fast), float-float at the midpoint (ZHS)
  float q0v, q1v, qmh, qml;
  ZPart zm;                      // ZHS, flat array: the z part of the midpoint's d
  float E0h, E0l, E1h, E1l, Emh, Eml;
  float nm1_0, nm1_1, nm1_m;     // n - 1 at start, end, midpoint
  float om0, om1, om_m;          // 1 - n|beta| at start, end, midpoint
  // midpoint position and time, float-float
  float mx, mxl, my, myl, mz, mzl, tmh, tml;
};

template <int FORM, int KIND, bool FLAT = false>
__device__ __forceinline__ void load_track_mixed(const float* T, int l, const MedParams& M, TrackM& t) {
  t.amp = FORM == C8R_ENDPOINT ? TF(fm::AMPE) : (TF(fm::AMPE) == 0.0f ? 0.0f : TF(fm::AMPZ));
  if (t.amp == 0.0f) return;  // filtered track or padding
  t.x0 = TF(fm::X0); t.y0 = TF(fm::Y0); t.z0 = TF(fm::Z0);
  t.x1 = TF(fm::X1); t.y1 = TF(fm::Y1); t.z1 = TF(fm::Z1);
  t.bx = TF(fm::BX); t.by = TF(fm::BY); t.bz = TF(fm::BZ);
  t.bmag = TF(fm::BMAG);
  const float omb = TF(fm::OMB);
  t.tau0h = TF(fm::TAU0H); t.tau0l = TF(fm::TAU0L);
  t.tau1h = TF(fm::TAU1H); t.tau1l = TF(fm::TAU1L);
  t.dtauh = TF(fm::DTAUH); t.dtaul = TF(fm::DTAUL);
  if (FORM == C8R_ENDPOINT && (KIND == C8R_UNIFORM || KIND == C8R_EXPONENTIAL)) {
    // the shifted times of the FP32 arrival, once per track (k = n/(c dt) or 1/(c dt))
    const float kh = KIND == C8R_UNIFORM ? M.s_h : M.kc_h, kl = KIND == C8R_UNIFORM ? M.s_l : M.kc_l;
    shifted_time(t.tau0h, t.tau0l, t.z0, 0.0f, kh, kl, t.T0h, t.T0l);
    shifted_time(t.tau1h, t.tau1l, t.z1, 0.0f, kh, kl, t.T1h, t.T1l);
  }
  // n - 1 is formed directly (N0 E, or the uniform n - 1 rounded from FP64): as
  // (1 + x) - 1 in FP32 it would lose ~6e-8, comparable to D near Cherenkov
  t.E0h = t.E1h = t.Emh = 1.0f;
  t.E0l = t.E1l = t.Eml = 0.0f;
  t.nm1_0 = t.nm1_1 = t.nm1_m = M.nm1f;
  if (KIND != C8R_UNIFORM) {
    t.E0h = TF(fm::E0H); t.E0l = TF(fm::E0L);
    t.E1h = TF(fm::E1H); t.E1l = TF(fm::E1L);
    t.Emh = TF(fm::EMH); t.Eml = TF(fm::EML);
    t.nm1_0 = __fmul_rn(M.N0f, t.E0h);
    t.nm1_1 = __fmul_rn(M.N0f, t.E1h);
    t.nm1_m = __fmul_rn(M.N0f, t.Emh);
  }
  if (KIND == C8R_EXPONENTIAL_SPHERICAL) {
    // n - 1 at the points over the sphere: the flat N0 exp(-z/H) times exp(-delta/H)
    t.nm1_0 = __fmul_rn(t.nm1_0, expf(-sphere_excess(t.x0, t.y0, t.z0, M.RE_f) * M.invH_h));
    t.nm1_1 = __fmul_rn(t.nm1_1, expf(-sphere_excess(t.x1, t.y1, t.z1, M.RE_f) * M.invH_h));
    t.nm1_m = __fmul_rn(t.nm1_m, expf(-sphere_excess(0.5f * (t.x0 + t.x1), 0.5f * (t.y0 + t.y1),
                                                     0.5f * (t.z0 + t.z1), M.RE_f) * M.invH_h));
  }
  // 1 - n|beta| = (1 - |beta|) - (n - 1)|beta|
  t.om0 = __fsub_rn(omb, __fmul_rn(t.nm1_0, t.bmag));
  t.om1 = __fsub_rn(omb, __fmul_rn(t.nm1_1, t.bmag));
  t.om_m = __fsub_rn(omb, __fmul_rn(t.nm1_m, t.bmag));
  // midpoint time (t0 + t1)/(2 dt), float-float
  two_sum(t.tau0h, t.tau1h, t.tmh, t.tml);
  t.tml = __fadd_rn(t.tml, __fadd_rn(t.tau0l, t.tau1l));
  t.tmh *= 0.5f;
  t.tml *= 0.5f;
  if (FORM == C8R_ZHS) {
    // midpoint position (x0 + x1)/2, exact in float-float
    two_sum(t.x0, t.x1, t.mx, t.mxl);
    two_sum(t.y0, t.y1, t.my, t.myl);
    two_sum(t.z0, t.z1, t.mz, t.mzl);
    t.mx *= 0.5f; t.mxl *= 0.5f; t.my *= 0.5f; t.myl *= 0.5f; t.mz *= 0.5f; t.mzl *= 0.5f;
  }
  if constexpr (FLAT && KIND == C8R_EXPONENTIAL) {
    // the refractivity quotient against the array's altitude, formed as the
    // per-pair arithmetic forms it (the altitude difference as geo_fast and
    // geo_lite form it), so the values are the same
    if constexpr (FORM == C8R_ENDPOINT) {
      t.q0v = fast_quotient(M, M.flat_Eh, M.flat_El, __fadd_rn(M.flat_zh, -t.z0), t.E0h, t.E0l);
      t.q1v = fast_quotient(M, M.flat_Eh, M.flat_El, __fadd_rn(M.flat_zh, -t.z1), t.E1h, t.E1l);
    } else {
      float dzh, dzl;
      two_sum(M.flat_zh, -t.mz, dzh, dzl);
      dzl = __fadd_rn(dzl, __fsub_rn(M.flat_zl, t.mzl));
      refr_quotient(M, M.flat_Eh, M.flat_El, dzh, dzl, t.Emh, t.Eml, t.qmh, t.qml);
      t.zm = z_part(dzh, dzl, t.bz);
    }
  }
}

// geometry shared by the forward and the adjoint Endpoint evaluation
struct EndpointEvalM {
  GeoM g0, g1, gm;
  FieldM f0, f1, fm;
  int branch;     // 0 two endpoints, 1 midpoint
  ff ua, ub;      // arrivals (start/end, or the two linearised midpoint arrivals)
  bool valid;
  float dop0, dop1;  // curved rays: optical-path change of the start and end paths (m)
};

// curved rays (C8R_EXPONENTIAL_RAY): turn the direction of g (a copy used for
// the field arithmetic; the straight geometry stays with the arrival time and
// the amplitude's R) and return the ray's optical-path change and the change of
// D = 1 - n beta.rhat that the turn makes
__device__ __forceinline__ void ray_turn_mixed(GeoM& g, float nu_e, float bx, float by, float bz, const MedParams& M,
                                               float& dop, float& dD) {
  const float dx = g.s[0], dy = g.s[1], dz = g.s[2], R = g.R0;
  const RayFix<float> r = ray_fix<float, 1>(dx * dx + dy * dy, dz, R, nu_e, M.invH_h);
  float t[3];
  ray_turn_vector<float>(dx, dy, dz, R, r.Q, t);
  g.s[0] = __fadd_rn(g.s[0], t[0]);
  g.s[1] = __fadd_rn(g.s[1], t[1]);
  g.s[2] = __fadd_rn(g.s[2], t[2]);
  dop = r.dop;
  dD = -(1.0f + nu_e) * (bx * t[0] + by * t[1] + bz * t[2]) * g.y;
}

// D in float-float plus a small FP32 change, renormalised
__device__ __forceinline__ ff ff_add_small(ff D, float d) {
  float h, l;
  two_sum(D.h, d, h, l);
  l = __fadd_rn(l, D.l);
  ff r;
  r.h = __fadd_rn(h, l);
  r.l = __fsub_rn(l, __fsub_rn(r.h, h));
  return r;
}

// Endpoint evaluation in three steps, shared by the forward pass (which runs
// the near-Cherenkov pairs apart from the others) and the adjoint.
// (1) propagator and field at both endpoints; false when an emission point
// sits on the antenna (outside the domain of the formula)
template <int KIND>
__device__ __forceinline__ bool endpoint_fields(const TrackM& t, const AntRec& A, const MedParams& M,
                                                EndpointEvalM& e) {
  geo_lite(A, t.x0, t.y0, t.z0, e.g0);
  geo_lite(A, t.x1, t.y1, t.z1, e.g1);
  if (e.g0.R0 == 0.0f || e.g1.R0 == 0.0f) return false;
  if constexpr (KIND == C8R_EXPONENTIAL_RAY) {
    // the field along the ray's direction at each endpoint
    GeoM r0 = e.g0, r1 = e.g1;
    float dD;
    ray_turn_mixed(r0, t.nm1_0, t.bx, t.by, t.bz, M, e.dop0, dD);
    ray_turn_mixed(r1, t.nm1_1, t.bx, t.by, t.bz, M, e.dop1, dD);
    field_mixed(r0, t.bx, t.by, t.bz, t.bmag, t.om0, __fadd_rn(1.0f, t.nm1_0), e.f0);
    field_mixed(r1, t.bx, t.by, t.bz, t.bmag, t.om1, __fadd_rn(1.0f, t.nm1_1), e.f1);
  } else {
    e.dop0 = e.dop1 = 0.0f;
    field_mixed(e.g0, t.bx, t.by, t.bz, t.bmag, t.om0, __fadd_rn(1.0f, t.nm1_0), e.f0);
    field_mixed(e.g1, t.bx, t.by, t.bz, t.bmag, t.om1, __fadd_rn(1.0f, t.nm1_1), e.f1);
  }
  return true;
}

// the near-Cherenkov test: min(|D_start|, |D_end|) < eps_C
__device__ __forceinline__ bool endpoint_near_cherenkov(const EndpointEvalM& e, const MedParams& M) {
  return !(fminf(fabsf(e.f0.D), fabsf(e.f1.D)) >= M.eps_C);
}

// (2a) arrival positions of the two endpoints
template <int KIND>
__device__ __forceinline__ void endpoint_arrivals(const TrackM& t, const AntRec& A, const MedParams& M,
                                                  EndpointEvalM& e) {
  GeoM g0 = e.g0, g1 = e.g1;
  geo_refine(g0);
  geo_refine(g1);
  e.ua = arrival_mixed<KIND>(M, A, g0, t.tau0h, t.tau0l, t.E0h, t.E0l, e.dop0);
  e.ub = arrival_mixed<KIND>(M, A, g1, t.tau1h, t.tau1l, t.E1h, t.E1l, e.dop1);
  e.branch = 0;
}

// (2b) near-Cherenkov: midpoint geometry and the linearised arrivals
// t_m -/+ D_m (t1 - t0)/2; false when the midpoint sits on the antenna
template <int KIND>
__device__ __forceinline__ bool endpoint_midpoint(const TrackM& t, const AntRec& A, const MedParams& M,
                                                  EndpointEvalM& e) {
  float dopm = 0.0f, dDm = 0.0f;
  if constexpr (KIND == C8R_EXPONENTIAL_RAY) {
    // the midpoint's own ray (its direction is not the mean of the endpoints')
    float mx, mxl, my, myl, mz, mzl;
    two_sum(t.x0, t.x1, mx, mxl);
    two_sum(t.y0, t.y1, my, myl);
    two_sum(t.z0, t.z1, mz, mzl);
    geo_lite(A, 0.5f * mx, 0.5f * my, 0.5f * mz, 0.5f * mxl, 0.5f * myl, 0.5f * mzl, e.gm);
    if (e.gm.R0 == 0.0f) return false;
    GeoM r = e.gm;
    ray_turn_mixed(r, t.nm1_m, t.bx, t.by, t.bz, M, dopm, dDm);
    field_mixed(r, t.bx, t.by, t.bz, t.bmag, t.om_m, __fadd_rn(1.0f, t.nm1_m), e.fm);
  } else {
    midpoint_from_endpoints(e.g0, e.g1, e.f0, e.f1, t.bmag, t.om_m, __fadd_rn(1.0f, t.nm1_m), e.gm, e.fm);
    if (e.gm.R0 == 0.0f) return false;
  }
  GeoM g = e.gm;
  geo_refine(g);
  const ff u0 = arrival_mixed<KIND>(M, A, g, t.tmh, t.tml, t.Emh, t.Eml, dopm);
  ff Dm = doppler_ff(g, t.bx, t.by, t.bz, t.nm1_m);
  if constexpr (KIND == C8R_EXPONENTIAL_RAY) Dm = ff_add_small(Dm, dDm);
  // the amplitude's 1/D_m, too, from the float-float D: here |D_m| can be far
  // below the FP32 form's absolute accuracy
  e.fm.D = __fadd_rn(Dm.h, Dm.l);
  float hh, hl;  // D_m (t1 - t0)/(2 dt), float-float
  two_prod(Dm.h, t.dtauh, hh, hl);
  hl = __fmaf_rn(Dm.h, t.dtaul, __fmaf_rn(Dm.l, t.dtauh, hl));
  hh *= 0.5f;
  hl *= 0.5f;
  two_sum(u0.h, -hh, e.ua.h, e.ua.l);
  e.ua.l = __fadd_rn(e.ua.l, __fsub_rn(u0.l, hl));
  two_sum(u0.h, hh, e.ub.h, e.ub.l);
  e.ub.l = __fadd_rn(e.ub.l, __fadd_rn(u0.l, hl));
  e.branch = 1;
  return true;
}

template <int KIND>
__device__ __forceinline__ void endpoint_eval_mixed(const TrackM& t, const AntRec& A, const MedParams& M,
                                                    EndpointEvalM& e) {
  e.valid = false;
  if (!endpoint_fields<KIND>(t, A, M, e)) return;
  if (endpoint_near_cherenkov(e, M)) {
    if (!endpoint_midpoint<KIND>(t, A, M, e)) return;
  } else {
    endpoint_arrivals<KIND>(t, A, M, e);
  }
  e.valid = true;
}

// Linear (two-bin) deposit (reading LD): a deposit arriving at u is spread over
// [u - 1/2, u + 1/2].  With J = floor(u + 1/2) (the "cell" between the bin
// centres J - 1/2 and J + 1/2) and s = u + 1/2 - J, bins J - 1 and J receive
// 1 - s and s of it.  Cells outside [0, N] touch no bin of the window; bin_raw
// clamps them to -1 or N + 1.
__device__ __forceinline__ int lin_cell(ff u, int N, float& s) {
  ff v;
  two_sum(u.h, 0.5f, v.h, v.l);
  v.l = __fadd_rn(v.l, u.l);
  return bin_raw(v, N + 1, s);
}

// ZHS with the linear deposit, an interval [u_lo, u_hi] over more than one cell:
// the tent weights averaged over it, for the bins around its two ends (per unit
// of the whole interval's deposit); every bin strictly between them receives
// 1/W.  First cell: bins J_lo - 1 and J_lo get (1 - s_lo)^2/2 and
// (1 - s_lo^2)/2; last cell: J_hi - 1 and J_hi get s_hi (1 - s_hi/2) and
// s_hi^2/2; every whole cell in between gives 1/2 to each of its two bins.
struct LinEnds {
  int k[4];
  float w[4];
  int n;
};
__device__ __forceinline__ LinEnds lin_ends(int Jlo, float slo, int Jhi, float shi, float invW) {
  const float a = 1.0f - slo;
  const float lo0 = 0.5f * a * a, lo1 = 0.5f * (1.0f - slo * slo);
  const float hi0 = shi * (1.0f - 0.5f * shi), hi1 = 0.5f * shi * shi;
  LinEnds z;
  z.k[0] = Jlo - 1;
  z.w[0] = lo0 * invW;
  z.k[1] = Jlo;
  if (Jhi == Jlo + 1) {
    z.w[1] = (lo1 + hi0) * invW;
    z.k[2] = Jhi;
    z.w[2] = hi1 * invW;
    z.k[3] = -1;
    z.w[3] = 0.0f;
    z.n = 3;
  } else {
    z.w[1] = (lo1 + 0.5f) * invW;
    z.k[2] = Jhi - 1;
    z.w[2] = (hi0 + 0.5f) * invW;
    z.k[3] = Jhi;
    z.w[3] = hi1 * invW;
    z.n = 4;
  }
  return z;
}

template <int FORM, int KIND, bool LIN = false, bool SPLIT = false, bool FLAT = false>
struct OpsMixed {
  using acc_t = float;
  using Track = TrackM;
  static constexpr int kPrec = C8R_MIXED;
  static constexpr int kTileBytes = kTileBytesMixed;
  // CTAs of 128 threads per SM the register budget is set for (curved rays
  // carry the ray solve as well, and the spherical Endpoint kernel its
  // curvature quadrature: fewer CTAs, more registers each; the spherical one at
  // 5 CTAs has no spills and is 1.6 % faster than at 6)
  static constexpr int kMinBlocks =
      FORM == C8R_ENDPOINT ? (KIND == C8R_EXPONENTIAL_RAY ? 4 : (KIND == C8R_EXPONENTIAL_SPHERICAL ? 5 : 6))
                           : (KIND == C8R_EXPONENTIAL_RAY ? 6 : 8);
  // Endpoint: the near-Cherenkov pairs (a minority, spread over most warps)
  // are set aside by the main pass and evaluated together afterwards
  static constexpr bool kDefers = FORM == C8R_ENDPOINT;
  // Endpoint with the one-bin deposit in the plain straight-line media: the
  // main pass takes each bin from the FP32 arrival with its error bound
  // (arrival_bin_fast) and sets aside only the endpoints it cannot decide,
  // for the float-float arrival after the main pass
  static constexpr bool kFastBins =
      FORM == C8R_ENDPOINT && !LIN && (KIND == C8R_UNIFORM || KIND == C8R_EXPONENTIAL);
  // the form of x = R - w in the FP32 arrival (arrival_fast): the split one
  // for lines of sight near the vertical, the direct one otherwise.  Either is
  // exact to its own bound; the host picks the kernel per launch from the
  // share of tracks that see the antenna array from above within 45 degrees
  // (counted by the ingest of earlier launches)
  static constexpr bool kSplit = SPLIT && kFastBins;
  // a flat antenna array: the refractivity quotient per track, in the main pass
  // of the Endpoint forward kernel of the direct arrival form and in the ZHS
  // forward and adjoint kernels, which also take the z part of the midpoint's
  // d once per track (ZPart; the host picks the kernel, MedParams::flat).
  // Measured: 47.96 -> 44.01 ms on 4e6 tracks of the 60-degree array
  // (Endpoint); ZHS 31.96 -> 29.56 ms with the quotient and -> 28.50 ms with
  // the z part as well, on the 2e7-track vertical shower in a step that runs
  // the Endpoint and then the ZHS process on the same tracks.  The split-form
  // Endpoint kernel keeps the quotient per pair (within 0.3 % either way)
  static constexpr bool kFlat =
      FLAT && KIND == C8R_EXPONENTIAL && ((kFastBins && !SPLIT) || FORM == C8R_ZHS);
  // adjoint CTAs (128 threads) per SM the registers are set for (the linear
  // Endpoint adjoint carries the slide of each deposit as well)
  static constexpr int kBwdMinBlocks = (LIN && FORM == C8R_ENDPOINT) ? 4 : 6;
  // ZHS: a second accumulator row holds the edges of box deposits
  static constexpr int kAccRows = FORM == C8R_ZHS ? 2 : 1;

  // the float-float part of an antenna record, as three 16-byte shared-memory
  // loads and one 8-byte load (the shifted time; loads whose fields a pass
  // does not use are dropped by the compiler)
  static __device__ __forceinline__ AntRec load_ant(const AntRec* p) {
    const float4* f = reinterpret_cast<const float4*>(&p->xh);
    const float4 a = f[0], b = f[1], c = f[2];
    const float2 T = *reinterpret_cast<const float2*>(&p->Tah);
    AntRec r;
    r.xh = a.x; r.yh = a.y; r.zh = a.z; r.xl = a.w;
    r.yl = b.x; r.zl = b.y; r.tauh = b.z; r.taul = b.w;
    r.Eah = c.x; r.Eal = c.y; r.fb_abs = c.z; r.fb_rel_v = c.w;
    r.Tah = T.x; r.Tal = T.y;
    return r;
  }

  static __device__ __forceinline__ void load(const void* Tv, int l, const MedParams& M, TrackM& t) {
    load_track_mixed<FORM, KIND, kFlat>(static_cast<const float*>(Tv), l, M, t);
  }
  static __device__ __forceinline__ bool live(const TrackM& t) { return t.amp != 0.0f; }

  // -------------------------------------------------------------------------
  // Endpoint (§1; James et al.): +amp V/(D R) at the start's arrival bin and
  // -amp V/(D R) at the end's, amp = q K / dt; midpoint form near Cherenkov.
  // -------------------------------------------------------------------------
  // The deposits of an evaluated pair; the evaluation is split between
  // pair_main and pair_deferred below.
  // a deposit (x, y, z) arriving in cell J at s, spread over bins J - 1 and J
  template <class Sink>
  static __device__ __forceinline__ void dep_lin(Sink& out, int N, int J, float s, float x, float y, float z) {
    const float r = 1.0f - s;
    if (J >= 1 && J - 1 < N) out.dep(J - 1, x * r, y * r, z * r);
    if (J >= 0 && J < N) out.dep(J, x * s, y * s, z * s);
  }

  // Endpoint deposits spread over two bins each (reading LD).  Near Cherenkov,
  // when both linearised arrivals lie in one cell J, the two spread deposits
  // +/- amp V/(D R) combine to the exact amp (dt_e/dt) V/R into bin J - 1 and
  // its negative into bin J, with no division by D.
  template <class Sink>
  static __device__ __forceinline__ void endpoint_deposit_lin(const TrackM& t, const EndpointEvalM& e,
                                                              const MedParams& M, Sink& out) {
    const int N = M.n_bins;
    out.rec(e.branch, e.ua, e.ub);
    float sa, sb;
    const int Ja = lin_cell(e.ua, N, sa);
    const int Jb = lin_cell(e.ub, N, sb);
    const float amp = t.amp;
    if (e.branch == 0) {
      const float c0 = __fdividef(amp, e.f0.D * e.g0.R0) * (e.f0.invR * e.f0.invR);
      const float c1 = __fdividef(-amp, e.f1.D * e.g1.R0) * (e.f1.invR * e.f1.invR);
      if (Ja == Jb) {
        // both in one cell: add them in registers, two reductions
        const float a0 = c0 * (1.0f - sa), b0 = c1 * (1.0f - sb), a1 = c0 * sa, b1 = c1 * sb;
        if (Ja >= 1 && Ja - 1 < N)
          out.dep(Ja - 1, a0 * e.f0.V[0] + b0 * e.f1.V[0], a0 * e.f0.V[1] + b0 * e.f1.V[1],
                  a0 * e.f0.V[2] + b0 * e.f1.V[2]);
        if (Ja >= 0 && Ja < N)
          out.dep(Ja, a1 * e.f0.V[0] + b1 * e.f1.V[0], a1 * e.f0.V[1] + b1 * e.f1.V[1],
                  a1 * e.f0.V[2] + b1 * e.f1.V[2]);
      } else {
        dep_lin(out, N, Ja, sa, c0 * e.f0.V[0], c0 * e.f0.V[1], c0 * e.f0.V[2]);
        dep_lin(out, N, Jb, sb, c1 * e.f1.V[0], c1 * e.f1.V[1], c1 * e.f1.V[2]);
      }
      return;
    }
    const float i2 = e.fm.invR * e.fm.invR;
    if (Ja == Jb) {
      const float c = amp * t.dtauh * (i2 * e.fm.invR);
      if (Ja >= 1 && Ja - 1 < N) out.dep(Ja - 1, c * e.fm.V[0], c * e.fm.V[1], c * e.fm.V[2]);
      if (Ja >= 0 && Ja < N) out.dep(Ja, -c * e.fm.V[0], -c * e.fm.V[1], -c * e.fm.V[2]);
      return;
    }
    const float c = __fdividef(amp, e.fm.D * e.gm.R0) * i2;
    dep_lin(out, N, Ja, sa, c * e.fm.V[0], c * e.fm.V[1], c * e.fm.V[2]);
    dep_lin(out, N, Jb, sb, -c * e.fm.V[0], -c * e.fm.V[1], -c * e.fm.V[2]);
  }

  template <class Sink>
  static __device__ __forceinline__ void endpoint_deposit(const TrackM& t, const EndpointEvalM& e,
                                                          const MedParams& M, Sink& out) {
    if constexpr (LIN) {
      endpoint_deposit_lin(t, e, M, out);
      return;
    }
    const int N = M.n_bins;
    out.rec(e.branch, e.ua, e.ub);
    float fa, fb;
    const int ka = bin_raw(e.ua, N, fa);
    const int kb = bin_raw(e.ub, N, fb);
    const bool ina = ka >= 0 && ka < N, inb = kb >= 0 && kb < N;
    const float amp = t.amp;
    if (e.branch == 0) {
      const float c0 = __fdividef(amp, e.f0.D * e.g0.R0) * (e.f0.invR * e.f0.invR);
      const float c1 = __fdividef(-amp, e.f1.D * e.g1.R0) * (e.f1.invR * e.f1.invR);
      if (ina && inb && ka == kb) {
        // both deposits in one bin: add them in registers, one reduction
        out.dep(ka, c0 * e.f0.V[0] + c1 * e.f1.V[0], c0 * e.f0.V[1] + c1 * e.f1.V[1],
                c0 * e.f0.V[2] + c1 * e.f1.V[2]);
      } else {
        if (ina) out.dep(ka, c0 * e.f0.V[0], c0 * e.f0.V[1], c0 * e.f0.V[2]);
        if (inb) out.dep(kb, c1 * e.f1.V[0], c1 * e.f1.V[1], c1 * e.f1.V[2]);
      }
      return;
    }
    if (ka == kb) return;  // one bin (or both outside on one side): the bin average of E vanishes
    const float c = __fdividef(amp, e.fm.D * e.gm.R0) * (e.fm.invR * e.fm.invR);
    if (ina) out.dep(ka, c * e.fm.V[0], c * e.fm.V[1], c * e.fm.V[2]);
    if (inb) out.dep(kb, -c * e.fm.V[0], -c * e.fm.V[1], -c * e.fm.V[2]);
  }

  // -------------------------------------------------------------------------
  // ZHS (§1; Zas, Halzen & Stanev): bin averages of the midpoint step
  // potential K_A beta_perp/(R |D|) over [t_m - |D| dt_e/2, t_m + |D| dt_e/2];
  // written as (K_A beta_perp dt_e/(R dt)) x (fraction of the interval in the
  // bin), which needs no division by D and is exact for a one-bin interval.
  // -------------------------------------------------------------------------
  template <class Sink>
  static __device__ __forceinline__ void zhs(const TrackM& t, const AntRec& A, const MedParams& M, Sink& out) {
    const int N = M.n_bins;
    GeoM gm;
    if constexpr (kFlat)
      geo_lite(A, t.mx, t.my, t.mxl, t.myl, t.zm, gm);
    else
      geo_lite(A, t.mx, t.my, t.mz, t.mxl, t.myl, t.mzl, gm);
    if (gm.R0 == 0.0f) return;
    FieldM f;
    float dop = 0.0f, dD = 0.0f;
    if constexpr (KIND == C8R_EXPONENTIAL_RAY) {
      GeoM r = gm;
      ray_turn_mixed(r, t.nm1_m, t.bx, t.by, t.bz, M, dop, dD);
      field_mixed(r, t.bx, t.by, t.bz, t.bmag, t.om_m, __fadd_rn(1.0f, t.nm1_m), f);
    } else {
      field_mixed(gm, t.bx, t.by, t.bz, t.bmag, t.om_m, __fadd_rn(1.0f, t.nm1_m), f);
    }
    ff um, aD;
    if constexpr (kFlat) {
      geo_refine(gm, t.zm);
      um = arrival_mixed_q<KIND>(M, A, gm, t.tmh, t.tml, t.qmh, t.qml, dop);
      aD = doppler_ff(gm, t.bx, t.by, t.zm, t.nm1_m);
    } else {
      geo_refine(gm);
      um = arrival_mixed<KIND>(M, A, gm, t.tmh, t.tml, t.Emh, t.Eml, dop);
      aD = doppler_ff(gm, t.bx, t.by, t.bz, t.nm1_m);
    }
    if constexpr (KIND == C8R_EXPONENTIAL_RAY) aD = ff_add_small(aD, dD);
    if (aD.h < 0.0f) {
      aD.h = -aD.h;
      aD.l = -aD.l;
    }
    float hh, hl;  // |D| (t1 - t0)/(2 dt), float-float
    two_prod(aD.h, t.dtauh, hh, hl);
    hl = __fmaf_rn(aD.h, t.dtaul, __fmaf_rn(aD.l, t.dtauh, hl));
    hh *= 0.5f;
    hl *= 0.5f;
    ff ulo, uhi;
    two_sum(um.h, -hh, ulo.h, ulo.l);
    ulo.l = __fadd_rn(ulo.l, __fsub_rn(um.l, hl));
    two_sum(um.h, hh, uhi.h, uhi.l);
    uhi.l = __fadd_rn(uhi.l, __fadd_rn(um.l, hl));
    const float s = -t.amp * (f.invR * f.invR) * f.invR;  // beta_perp = -V
    const float Mx = s * f.V[0], My = s * f.V[1], Mz = s * f.V[2];
    float flo, fhi;
    const int klo = bin_raw(ulo, N, flo);
    const int khi = bin_raw(uhi, N, fhi);
    out.rec(klo == khi ? 2 : 3, ulo, uhi);
    if constexpr (LIN) {
      // reading LD: the tent weights averaged over the interval
      float slo, shi;
      const int Jlo = lin_cell(ulo, N, slo);
      const int Jhi = lin_cell(uhi, N, shi);
      if (Jlo == Jhi) {
        // inside one cell the tents are linear: the tent at the middle
        dep_lin(out, N, Jlo, 0.5f * (slo + shi), Mx, My, Mz);
        return;
      }
      const float invW = __fdividef(1.0f, 2.0f * hh);
      const LinEnds z = lin_ends(Jlo, slo, Jhi, shi, invW);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < z.n && z.k[i] >= 0 && z.k[i] < N) out.dep(z.k[i], Mx * z.w[i], My * z.w[i], Mz * z.w[i]);
      const int kb = Jlo + 1 < 0 ? 0 : Jlo + 1;
      const int ke = Jhi - 2 > N - 1 ? N - 1 : Jhi - 2;
      if (kb <= ke) out.dep_box(kb, ke, Mx * invW, My * invW, Mz * invW);
      return;
    }
    // the interval's first bin takes the whole deposit (an interval inside one
    // bin: weight 1, M x 1 = M exactly) or the share it covers, in one
    // reduction either way, so that lanes of both kinds take one path
    const bool one = klo == khi;
    const float invW = __fdividef(1.0f, 2.0f * hh);  // 1 / interval length in bins (unused when one)
    const float wlo = one ? 1.0f : gap_to_next_edge(ulo, klo) * invW;
    if (klo >= 0 && klo < N && wlo > 0.0f) out.dep(klo, Mx * wlo, My * wlo, Mz * wlo);
    if (one) return;
    // the partly covered last bin
    if (khi >= 0 && khi < N) {
      const float w = fhi * invW;
      if (w > 0.0f) out.dep(khi, Mx * w, My * w, Mz * w);
    }
    // the whole bins in between (inside the window) all receive M / W
    const int kb = klo + 1 < 0 ? 0 : klo + 1;
    const int ke = khi - 1 > N - 1 ? N - 1 : khi - 1;
    if (kb <= ke) out.dep_box(kb, ke, Mx * invW, My * invW, Mz * invW);
  }

  // the bins of both endpoints from the FP32 arrival (kFastBins) in the form
  // of x = R - w this kernel is compiled for
  static __device__ __forceinline__ void fast_bins(const TrackM& t, const AntRec& A, const MedParams& M,
                                                   const GeoM& g0, const GeoM& g1, float S0, float S1, float P0,
                                                   float P1, int& ka, int& kb) {
    float qa = 0.0f, qb = 0.0f;
    if constexpr (kFlat) {
      qa = t.q0v;
      qb = t.q1v;
    } else if constexpr (KIND == C8R_EXPONENTIAL) {
      qa = fast_quotient(M, A.Eah, A.Eal, g0.s[2], t.E0h, t.E0l);
      qb = fast_quotient(M, A.Eah, A.Eal, g1.s[2], t.E1h, t.E1l);
    }
    ka = arrival_bin_fast<KIND, kSplit>(M, A, g0, S0, P0, t.T0h, t.T0l, qa);
    kb = arrival_bin_fast<KIND, kSplit>(M, A, g1, S1, P1, t.T1h, t.T1l, qb);
  }

  // main pass: every pair except (Endpoint) the near-Cherenkov ones, for which
  // it deposits nothing and returns kDeferPair, and (kFastBins) the endpoints
  // whose bin the FP32 arrival leaves open, returned as kDeferEnd0/kDeferEnd1
  // bits after the other endpoint's deposit
  template <class Sink>
  static __device__ __forceinline__ int pair_main(const TrackM& t, const AntRec& A, const MedParams& M, Sink& out) {
    if constexpr (kFastBins) {
      GeoM g0, g1;
      float S0, S1, P0, P1;
      geo_fast(A, t.x0, t.y0, t.z0, g0, S0, P0);
      geo_fast(A, t.x1, t.y1, t.z1, g1, S1, P1);
      if (g0.R0 == 0.0f || g1.R0 == 0.0f) return kDeferNone;  // an emission point on the antenna
      int ka, kb;
      fast_bins(t, A, M, g0, g1, S0, S1, P0, P1, ka, kb);
      FieldM f0, f1;
      field_mixed(g0, t.bx, t.by, t.bz, t.bmag, t.om0, __fadd_rn(1.0f, t.nm1_0), f0);
      field_mixed(g1, t.bx, t.by, t.bz, t.bmag, t.om1, __fadd_rn(1.0f, t.nm1_1), f1);
      if (!(fminf(fabsf(f0.D), fabsf(f1.D)) >= M.eps_C)) return kDeferPair;
      const bool ina = ka >= 0, inb = kb >= 0;  // decided and inside the window
      const float amp = t.amp;
      const float c0 = __fdividef(amp, f0.D * g0.R0) * (f0.invR * f0.invR);
      const float c1 = __fdividef(-amp, f1.D * g1.R0) * (f1.invR * f1.invR);
      // both deposits in one bin add in registers (one reduction); otherwise
      // one each.  One code path for both kinds of lane: the start's deposit
      // carries the end's when they share the bin (the end's weight 0 else)
      const bool same = ina && inb && ka == kb;
      const float c1s = same ? c1 : 0.0f;
      if (ina)
        out.dep(ka, __fmaf_rn(c1s, f1.V[0], c0 * f0.V[0]), __fmaf_rn(c1s, f1.V[1], c0 * f0.V[1]),
                __fmaf_rn(c1s, f1.V[2], c0 * f0.V[2]));
      if (inb && !same) out.dep(kb, c1 * f1.V[0], c1 * f1.V[1], c1 * f1.V[2]);
      return (ka == kFastUndecided ? kDeferEnd0 : 0) | (kb == kFastUndecided ? kDeferEnd1 : 0);
    } else if constexpr (FORM == C8R_ENDPOINT) {
      EndpointEvalM e;
      if (!endpoint_fields<KIND>(t, A, M, e)) return kDeferNone;
      if (endpoint_near_cherenkov(e, M)) return kDeferPair;
      endpoint_arrivals<KIND>(t, A, M, e);
      endpoint_deposit(t, e, M, out);
      return kDeferNone;
    } else {
      zhs(t, A, M, out);
      return kDeferNone;
    }
  }

  // A near-Cherenkov pair (kFastBins) whose two linearised arrivals
  // u_m -/+ D_m (t1 - t0)/(2 dt) lie in one bin, or both before or both after
  // the window, contributes exactly 0 (reading C), and so does its adjoint.
  // Decided here from FP32 midpoint geometry, as arrival_bin_fast decides a
  // bin: the midpoint d_m = (s0 + s1)/2 from the endpoints' FP32 d (the
  // float-float path's high part; its roundings move each component by at most
  // 2u |s_i| + u L_i / 2, which moves x = R - w by at most 6u x + u L1 / 2, so
  // the arrival bound takes 3 more u k x and 2 u k L1, L1 >= L), the FP32
  // Doppler factor D_m (field_mixed: off the float-float D_m by at most
  // 8 u n + 16 u |D_m|, from the direction's rounding and its own), and two
  // more roundings on the interval ends.  True when the pair is decided to be
  // zero, false when the float-float evaluation must run (about 4 % of the
  // near-Cherenkov pairs of a shower).
  static __device__ __forceinline__ bool near_zero_fast(const void* Tv, int l, const AntRec& A, const MedParams& M) {
    if constexpr (kFastBins) {
      constexpr float u = 5.9604644775390625e-8f;  // 2^-24
      const float* T = static_cast<const float*>(Tv);
      const float x0 = TF(fm::X0), y0 = TF(fm::Y0), z0 = TF(fm::Z0);
      const float x1 = TF(fm::X1), y1 = TF(fm::Y1), z1 = TF(fm::Z1);
      const float a0x = __fadd_rn(A.xh, -x0), a0y = __fadd_rn(A.yh, -y0), a0z = __fadd_rn(A.zh, -z0);
      const float a1x = __fadd_rn(A.xh, -x1), a1y = __fadd_rn(A.yh, -y1), a1z = __fadd_rn(A.zh, -z1);
      GeoM g;
      g.s[0] = 0.5f * __fadd_rn(a0x, a1x);
      g.s[1] = 0.5f * __fadd_rn(a0y, a1y);
      g.s[2] = 0.5f * __fadd_rn(a0z, a1z);
      const float rho2 = __fmaf_rn(g.s[0], g.s[0], __fmul_rn(g.s[1], g.s[1]));
      const float S = __fmaf_rn(g.s[2], g.s[2], rho2);
      g.y = rsqrtf(S);
      g.R0 = __fmul_rn(S, g.y);
      g.R1 = 0.0f;
      if (g.R0 == 0.0f) return true;  // the midpoint on the antenna: no deposit
      const float L1 = fabsf(__fsub_rn(a0x, a1x)) + fabsf(__fsub_rn(a0y, a1y)) + fabsf(__fsub_rn(a0z, a1z));
      const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ), bmag = TF(fm::BMAG);
      float Eh = 1.0f, El = 0.0f, nm1 = M.nm1f;
      if (KIND != C8R_UNIFORM) {
        Eh = TF(fm::EMH);
        El = TF(fm::EML);
        nm1 = __fmul_rn(M.N0f, Eh);
      }
      const float om = __fsub_rn(TF(fm::OMB), __fmul_rn(nm1, bmag));
      FieldM f;
      field_mixed(g, bx, by, bz, bmag, om, __fadd_rn(1.0f, nm1), f);
      // midpoint time (t0 + t1)/(2 dt), float-float, as load_track_mixed forms
      // it, shifted by k z_m at the exact midpoint height z_m = (z0 + z1)/2
      float tmh, tml;
      two_sum(TF(fm::TAU0H), TF(fm::TAU1H), tmh, tml);
      tml = __fadd_rn(tml, __fadd_rn(TF(fm::TAU0L), TF(fm::TAU1L)));
      tmh *= 0.5f;
      tml *= 0.5f;
      float zmh, zml;
      two_sum(z0, z1, zmh, zml);
      const float kh = KIND == C8R_UNIFORM ? M.s_h : M.kc_h, kl = KIND == C8R_UNIFORM ? M.s_l : M.kc_l;
      float Tmh, Tml;
      shifted_time(tmh, tml, 0.5f * zmh, 0.5f * zml, kh, kl, Tmh, Tml);
      float uf;
      const float qv = KIND == C8R_EXPONENTIAL ? fast_quotient(M, A.Eah, A.Eal, g.s[2], Eh, El) : 0.0f;
      // the kernel's arrival form (either is exact to its own bound; one form
      // for every lane keeps the warp on one path)
      const float eps_a = arrival_fast<KIND, kSplit>(M, A, g, S, rho2, Tmh, Tml, qv, 3.0f, uf);
      const float eps_u = __fmaf_rn(2.0f * u * kh, L1, eps_a);
      const float dtau = TF(fm::DTAUH);
      const float aD = fabsf(f.D);
      const float h = 0.5f * __fmul_rn(aD, dtau);
      const float dh = __fmul_rn(__fmaf_rn(16.0f * u, aD, 8.0f * u * __fadd_rn(1.0f, nm1)), dtau);
      const float e = __fadd_rn(__fadd_rn(eps_u, dh), 2.0f * u * __fadd_rn(fabsf(uf), h));
      const float lo = __fsub_rn(__fsub_rn(uf, h), e), hi = __fadd_rn(__fadd_rn(uf, h), e);
      return hi < 0.0f || lo >= (float)M.n_bins || floorf(lo) == floorf(hi);
    } else {
      return false;
    }
  }

  // one endpoint set aside by the main pass (kFastBins; `end` is kDeferEnd0 or
  // kDeferEnd1), read from the staged tile (lane l): its float-float arrival
  // decides the bin.  The endpoint's fields are picked by index, so lanes with
  // different endpoints run one code path and only one endpoint's values are
  // live; they are formed as load_track_mixed forms them, and the deposit is
  // the one the main pass would have made (the same geometry and field
  // functions, so the same values)
  template <class Sink>
  static __device__ __forceinline__ void end_deferred(const void* Tv, int l, const AntRec& A, const MedParams& M,
                                                      Sink& out, int end) {
    if constexpr (kFastBins) {
      const float* T = static_cast<const float*>(Tv);
      const int N = M.n_bins;
      const int j = end == kDeferEnd1 ? 1 : 0;
      const float amp = TF(fm::AMPE);
      const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ), bmag = TF(fm::BMAG);
      float Eh = 1.0f, El = 0.0f, nm1 = M.nm1f;
      if (KIND != C8R_UNIFORM) {
        Eh = TF(fm::E0H + 2 * j);
        El = TF(fm::E0L + 2 * j);
        nm1 = __fmul_rn(M.N0f, Eh);
      }
      const float om = __fsub_rn(TF(fm::OMB), __fmul_rn(nm1, bmag));
      GeoM g;
      geo_lite(A, TF(fm::X0 + 3 * j), TF(fm::Y0 + 3 * j), TF(fm::Z0 + 3 * j), g);
      FieldM f;
      field_mixed(g, bx, by, bz, bmag, om, __fadd_rn(1.0f, nm1), f);
      geo_refine(g);
      const ff ua = arrival_mixed<KIND>(M, A, g, TF(fm::TAU0H + 2 * j), TF(fm::TAU0L + 2 * j), Eh, El);
      float fr;
      const int k = bin_raw(ua, N, fr);
      if (k < 0 || k >= N) return;
      const float c = __fdividef(j ? -amp : amp, f.D * g.R0) * (f.invR * f.invR);
      out.dep(k, c * f.V[0], c * f.V[1], c * f.V[2]);
    }
  }

  // a pair set aside by the main pass (Endpoint near the Cherenkov angle)
  template <class Sink>
  static __device__ __forceinline__ void pair_deferred(const TrackM& t, const AntRec& A, const MedParams& M,
                                                       Sink& out) {
    if constexpr (FORM == C8R_ENDPOINT) {
      EndpointEvalM e;
      if (!endpoint_fields<KIND>(t, A, M, e)) return;
      if (!endpoint_midpoint<KIND>(t, A, M, e)) return;
      endpoint_deposit(t, e, M, out);
    }
  }

  // one pair, complete, with float-float arrivals throughout (the arrival
  // listing records them)
  template <class Sink>
  static __device__ __forceinline__ void pair(const TrackM& t, const AntRec& A, const MedParams& M, Sink& out) {
    if constexpr (FORM == C8R_ENDPOINT) {
      EndpointEvalM e;
      endpoint_eval_mixed<KIND>(t, A, M, e);
      if (e.valid) endpoint_deposit(t, e, M, out);
    } else {
      zhs(t, A, M, out);
    }
  }

  // one pair from a staged tile (the arrival listing uses this)
  template <class Sink>
  static __device__ __forceinline__ void fwd(const void* Tv, int l, const AntRec& A, const MedParams& M, Sink& out) {
    TrackM t;
    load(Tv, l, M, t);
    if (!live(t)) return;
    pair(t, A, M, out);
  }

  // -------------------------------------------------------------------------
  // adjoint of `endpoint` with bins and branch held fixed
  // -------------------------------------------------------------------------
  static __device__ __forceinline__ void deposit_grad(const GeoM& g, const FieldM& f, float D, float n,
                                                      const float gv[3], float kappa, float dd[3], float db[3],
                                                      float& dns) {
    const float invR = f.invR;
    const float rh[3] = {g.s[0] * invR, g.s[1] * invR, g.s[2] * invR};
    const float inv2 = invR * invR;
    const float V[3] = {f.V[0] * inv2, f.V[1] * inv2, f.V[2] * inv2};
    const float c = f.bd * invR;
    deposit_adjoint<float>(rh, V, c, D, g.R0, n, gv, kappa, dd, db, dns);
  }
  static __device__ __forceinline__ void deposit_grad(const GeoM& g, const FieldM& f, float n, const float gv[3],
                                                      float kappa, float dd[3], float db[3], float& dns) {
    deposit_grad(g, f, f.D, n, gv, kappa, dd, db, dns);
  }

  // dL/dtrace seen by a unit deposit in cell J at s (reading LD), and its rate of
  // change with the arrival (bins outside the window read 0)
  static __device__ __forceinline__ void gather_lin(const float4* G, int N, int J, float s, float gv[3],
                                                    float slope[3]) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 g0 = (J >= 1 && J - 1 < N) ? G[J - 1] : z4;
    const float4 g1 = (J >= 0 && J < N) ? G[J] : z4;
    const float r = 1.0f - s;
    gv[0] = r * g0.x + s * g1.x;
    gv[1] = r * g0.y + s * g1.y;
    gv[2] = r * g0.z + s * g1.z;
    slope[0] = g1.x - g0.x;
    slope[1] = g1.y - g0.y;
    slope[2] = g1.z - g0.z;
  }

  // chain rule through an arrival position u = (t_e - t_a)/dt + (R + F)/(c dt)
  // of the emission point at d = x_a - x_e (refractivity factor E): adds
  // dL/dx_e x w_e (w_e = 1, or 1/2 to each endpoint for the midpoint), dL/dx_a,
  // dL/dN0; the caller adds dL/dt_e
  static __device__ __forceinline__ void arrival_grad(const GeoM& g, float invR, float E, const MedParams& M,
                                                      float dLdu, float* tg_pos0, float* tg_pos1, float w_e,
                                                      float ga[3], float& dn) {
    const RefrGrad<float> rg = refraction_grad<float>(KIND, g.R0, g.s[2] * M.invH_h, E, M.N0f, M.invH_h, M.nm1f);
    const float dLdopt = dLdu * M.kc_h;
    const float dLdR = dLdopt * (1.0f + rg.dF_dR);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = dLdR * g.s[k] * invR;
      ga[k] += v;
      tg_pos0[k] -= w_e * v;
      if (tg_pos1) tg_pos1[k] -= w_e * v;
    }
    tg_pos0[2] += w_e * dLdopt * rg.dF_dzm;
    if (tg_pos1) tg_pos1[2] += w_e * dLdopt * rg.dF_dzm;
    ga[2] += dLdopt * rg.dF_dza;
    dn += dLdopt * rg.dF_dN0;
  }

  // chain rule of one one-bin Endpoint deposit (endpoint J, bin held fixed,
  // dL/dtrace g4 at its bin) into the track gradients tg (positions of endpoint
  // J, beta), the antenna gradient ga and dL/dN0
  template <int J>
  static __device__ __forceinline__ void adj_end(const GeoM& g, const FieldM& f, float nm1, float E, float kappa,
                                                 const float4 g4, const MedParams& M, float tg[11], float ga[3],
                                                 float& dn) {
    const float dNdz_fac = (KIND == C8R_EXPONENTIAL) ? -M.N0f * M.invH_h : 0.0f;
    const float gv[3] = {g4.x, g4.y, g4.z};
    float dd[3], db[3], dns;
    deposit_grad(g, f, 1.0f + nm1, gv, kappa, dd, db, dns);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      tg[3 * J + c] -= dd[c];
      ga[c] += dd[c];
      tg[8 + c] += db[c];
    }
    tg[3 * J + 2] += dns * dNdz_fac * E;
    dn += dns * E;
  }

  // adjoint main pass: every pair except (Endpoint) the near-Cherenkov ones, for
  // which it adds nothing and returns kDeferPair, and (kFastBins) the endpoints
  // whose bin the FP32 arrival leaves open (kDeferEnd0/kDeferEnd1 bits), after
  // the other endpoint's part
  static __device__ __forceinline__ int adj_main(const TrackM& t, const AntRec& A, const MedParams& M,
                                                 const float4* G, const PrefixFF* Gp, float tg[11], float ga[3],
                                                 float& dn) {
    if constexpr (FORM == C8R_ZHS) {
      adj_zhs(t, A, M, G, Gp, tg, ga, dn);
      return kDeferNone;
    } else if constexpr (kFastBins) {
      GeoM g0, g1;
      float S0, S1, P0, P1;
      geo_fast(A, t.x0, t.y0, t.z0, g0, S0, P0);
      geo_fast(A, t.x1, t.y1, t.z1, g1, S1, P1);
      if (g0.R0 == 0.0f || g1.R0 == 0.0f) return kDeferNone;
      FieldM f0, f1;
      field_mixed(g0, t.bx, t.by, t.bz, t.bmag, t.om0, __fadd_rn(1.0f, t.nm1_0), f0);
      field_mixed(g1, t.bx, t.by, t.bz, t.bmag, t.om1, __fadd_rn(1.0f, t.nm1_1), f1);
      if (!(fminf(fabsf(f0.D), fabsf(f1.D)) >= M.eps_C)) return kDeferPair;
      int ka, kb;
      fast_bins(t, A, M, g0, g1, S0, S1, P0, P1, ka, kb);
      if (ka >= 0) adj_end<0>(g0, f0, t.nm1_0, t.E0h, t.amp, G[ka], M, tg, ga, dn);
      if (kb >= 0) adj_end<1>(g1, f1, t.nm1_1, t.E1h, -t.amp, G[kb], M, tg, ga, dn);
      return (ka == kFastUndecided ? kDeferEnd0 : 0) | (kb == kFastUndecided ? kDeferEnd1 : 0);
    } else {
      EndpointEvalM e;
      if (!endpoint_fields<KIND>(t, A, M, e)) return kDeferNone;
      if (endpoint_near_cherenkov(e, M)) return kDeferPair;
      endpoint_arrivals<KIND>(t, A, M, e);
      adj_deposits(t, e, M, G, tg, ga, dn);
      return kDeferNone;
    }
  }

  // the adjoint of one endpoint set aside by the main pass (kFastBins; `end` is
  // kDeferEnd0 or kDeferEnd1), read from the staged tile (lane l) as
  // end_deferred reads it: the float-float arrival gives the bin, the chain
  // rule is adj_end's, and the track gradients (positions of that endpoint,
  // beta) go to the output of track i with one reduction each; ga and dn
  // collect the antenna and N0 parts
  static __device__ __forceinline__ void adj_end_deferred(const void* Tv, int l, const AntRec& A, const MedParams& M,
                                                          const float4* G, const c8r_track_grads& out, int64_t i,
                                                          float ga[3], float& dn, int end) {
    if constexpr (kFastBins) {
      const float* T = static_cast<const float*>(Tv);
      const int N = M.n_bins;
      const int j = end == kDeferEnd1 ? 1 : 0;
      const float amp = TF(fm::AMPE);
      const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ), bmag = TF(fm::BMAG);
      float Eh = 1.0f, El = 0.0f, nm1 = M.nm1f;
      if (KIND != C8R_UNIFORM) {
        Eh = TF(fm::E0H + 2 * j);
        El = TF(fm::E0L + 2 * j);
        nm1 = __fmul_rn(M.N0f, Eh);
      }
      const float om = __fsub_rn(TF(fm::OMB), __fmul_rn(nm1, bmag));
      GeoM g;
      geo_lite(A, TF(fm::X0 + 3 * j), TF(fm::Y0 + 3 * j), TF(fm::Z0 + 3 * j), g);
      FieldM f;
      field_mixed(g, bx, by, bz, bmag, om, __fadd_rn(1.0f, nm1), f);
      GeoM gr = g;
      geo_refine(gr);
      const ff ua = arrival_mixed<KIND>(M, A, gr, TF(fm::TAU0H + 2 * j), TF(fm::TAU0L + 2 * j), Eh, El);
      float fr;
      const int k = bin_raw(ua, N, fr);
      if (k < 0 || k >= N) return;
      const float dNdz_fac = (KIND == C8R_EXPONENTIAL) ? -M.N0f * M.invH_h : 0.0f;
      const float4 g4 = G[k];
      const float gv[3] = {g4.x, g4.y, g4.z};
      float dd[3], db[3], dns;
      deposit_grad(g, f, 1.0f + nm1, gv, j ? -amp : amp, dd, db, dns);
      float* px = static_cast<float*>(j ? out.x1 : out.x0);
      float* py = static_cast<float*>(j ? out.y1 : out.y0);
      float* pz = static_cast<float*>(j ? out.z1 : out.z0);
      const float gz = -dd[2] + dns * dNdz_fac * Eh;
      if (dd[0] != 0.0f) atomicAdd(px + i, -dd[0]);
      if (dd[1] != 0.0f) atomicAdd(py + i, -dd[1]);
      if (gz != 0.0f) atomicAdd(pz + i, gz);
      if (db[0] != 0.0f) atomicAdd(static_cast<float*>(out.bx) + i, db[0]);
      if (db[1] != 0.0f) atomicAdd(static_cast<float*>(out.by) + i, db[1]);
      if (db[2] != 0.0f) atomicAdd(static_cast<float*>(out.bz) + i, db[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) ga[c] += dd[c];
      dn += dns * Eh;
    }
  }
  static __device__ __forceinline__ void adj_deferred(const TrackM& t, const AntRec& A, const MedParams& M,
                                                      const float4* G, const PrefixFF*, float tg[11], float ga[3],
                                                      float& dn) {
    if constexpr (FORM == C8R_ENDPOINT) {
      EndpointEvalM e;
      if (!endpoint_fields<KIND>(t, A, M, e)) return;
      if (!endpoint_midpoint<KIND>(t, A, M, e)) return;
      adj_deposits(t, e, M, G, tg, ga, dn);
    }
  }

  // G summed over bins kb..ke from the float-float running sums: the FP32
  // difference of the high parts is exact or rounded relative to the result,
  // and the low parts restore what the high parts dropped, so the sum comes out
  // rounded to FP32 plus the running sums' own error (~2k u^2 of the largest
  // partial sum after k bins), without the FP64 pipe
  static __device__ __forceinline__ void run_sum(const PrefixFF* Gp, int kb, int ke, float& ix, float& iy,
                                                 float& iz) {
    const PrefixFF p1 = Gp[ke + 1], p0 = Gp[kb];
    ix = __fadd_rn(__fsub_rn(p1.hx, p0.hx), __fsub_rn(p1.lx, p0.lx));
    iy = __fadd_rn(__fsub_rn(p1.hy, p0.hy), __fsub_rn(p1.ly, p0.ly));
    iz = __fadd_rn(__fsub_rn(p1.hz, p0.hz), __fsub_rn(p1.lz, p0.lz));
  }

  // ZHS adjoint (bins of the interval ends held fixed): the forward arithmetic
  // of `zhs`, then the chain rule through the one-bin deposit A = amp beta_perp/R
  // (amp = q K_A (t1 - t0)/dt) and the weights of [u_m - h, u_m + h] over its
  // bins: with S = sum_k w_k G_k, g_lo/g_hi = A.G at the first/last bin and W =
  // 2h, dL/du_m = (g_hi - g_lo)/W and dL/dh = (g_hi + g_lo - 2 A.S)/W (both 0
  // for a one-bin interval).  The sum of G over the whole bins in between comes
  // from the running sums Gp.  Times in ns, positions in m.
  static __device__ __forceinline__ void adj_zhs(const TrackM& t, const AntRec& A, const MedParams& M,
                                                 const float4* G, const PrefixFF* Gp, float tg[11], float ga[3],
                                                 float& dn) {
    const int N = M.n_bins;
    GeoM gm;
    if constexpr (kFlat)
      geo_lite(A, t.mx, t.my, t.mxl, t.myl, t.zm, gm);
    else
      geo_lite(A, t.mx, t.my, t.mz, t.mxl, t.myl, t.mzl, gm);
    if (gm.R0 == 0.0f) return;
    FieldM f;
    field_mixed(gm, t.bx, t.by, t.bz, t.bmag, t.om_m, __fadd_rn(1.0f, t.nm1_m), f);
    ff um, aD;
    if constexpr (kFlat) {
      geo_refine(gm, t.zm);
      um = arrival_mixed_q<KIND>(M, A, gm, t.tmh, t.tml, t.qmh, t.qml);
      aD = doppler_ff(gm, t.bx, t.by, t.zm, t.nm1_m);
    } else {
      geo_refine(gm);
      um = arrival_mixed<KIND>(M, A, gm, t.tmh, t.tml, t.Emh, t.Eml);
      aD = doppler_ff(gm, t.bx, t.by, t.bz, t.nm1_m);
    }
    const float sgn = aD.h < 0.0f ? -1.0f : 1.0f;
    if (aD.h < 0.0f) {
      aD.h = -aD.h;
      aD.l = -aD.l;
    }
    float hh, hl;
    two_prod(aD.h, t.dtauh, hh, hl);
    hl = __fmaf_rn(aD.h, t.dtaul, __fmaf_rn(aD.l, t.dtauh, hl));
    hh *= 0.5f;
    hl *= 0.5f;
    ff ulo, uhi;
    two_sum(um.h, -hh, ulo.h, ulo.l);
    ulo.l = __fadd_rn(ulo.l, __fsub_rn(um.l, hl));
    two_sum(um.h, hh, uhi.h, uhi.l);
    uhi.l = __fadd_rn(uhi.l, __fadd_rn(um.l, hl));
    float flo, fhi;
    const int klo = bin_raw(ulo, N, flo);
    const int khi = bin_raw(uhi, N, fhi);
    const float invR = f.invR;
    const float rh[3] = {gm.s[0] * invR, gm.s[1] * invR, gm.s[2] * invR};
    const float b[3] = {t.bx, t.by, t.bz};
    const float c = f.bd * invR;
    const float Av[3] = {t.amp * (b[0] - c * rh[0]) * invR, t.amp * (b[1] - c * rh[1]) * invR,
                         t.amp * (b[2] - c * rh[2]) * invR};
    float S[3];
    float dLdu = 0.0f, dLdh = 0.0f;
    if constexpr (LIN) {
      float slo, shi;
      const int Jlo = lin_cell(ulo, N, slo);
      const int Jhi = lin_cell(uhi, N, shi);
      float sl[3];
      if (Jlo == Jhi) {
        if (Jlo < 0 || Jlo > N) return;
        gather_lin(G, N, Jlo, 0.5f * (slo + shi), S, sl);
        dLdu = Av[0] * sl[0] + Av[1] * sl[1] + Av[2] * sl[2];
      } else {
        const float invW = __fdividef(1.0f, 2.0f * hh);
        const LinEnds z = lin_ends(Jlo, slo, Jhi, shi, invW);
        float ix = 0.0f, iy = 0.0f, iz = 0.0f;  // G summed over the bins strictly between the ends
        const int kb = Jlo + 1 < 0 ? 0 : Jlo + 1;
        const int ke = Jhi - 2 > N - 1 ? N - 1 : Jhi - 2;
        if (kb <= ke) run_sum(Gp, kb, ke, ix, iy, iz);
        S[0] = invW * ix;
        S[1] = invW * iy;
        S[2] = invW * iz;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (i < z.n && z.k[i] >= 0 && z.k[i] < N) {
            const float4 g = G[z.k[i]];
            S[0] += z.w[i] * g.x;
            S[1] += z.w[i] * g.y;
            S[2] += z.w[i] * g.z;
          }
        }
        float glo[3], ghi[3];
        gather_lin(G, N, Jlo, slo, glo, sl);
        gather_lin(G, N, Jhi, shi, ghi, sl);
        const float p_lo = Av[0] * glo[0] + Av[1] * glo[1] + Av[2] * glo[2];
        const float p_hi = Av[0] * ghi[0] + Av[1] * ghi[1] + Av[2] * ghi[2];
        const float AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
        dLdu = (p_hi - p_lo) * invW;
        dLdh = (p_hi + p_lo - 2.0f * AS) * invW;
      }
    } else {
      // one path for intervals inside one bin (weight 1 on its bin, 1 G = G
      // exactly, and no dependence on the interval's ends: 1/W taken as 0) and
      // for intervals over several bins
      const bool one = klo == khi;
      const bool inlo = klo >= 0 && klo < N, inhi = !one && khi >= 0 && khi < N;
      if (one && !inlo) return;
      const float invW = one ? 0.0f : __fdividef(1.0f, 2.0f * hh);
      const float4 glo = inlo ? G[klo] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 ghi = inhi ? G[khi] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float wlo = inlo ? (one ? 1.0f : gap_to_next_edge(ulo, klo) * invW) : 0.0f, whi = fhi * invW;
      float ix = 0.0f, iy = 0.0f, iz = 0.0f;  // G summed over the whole bins between
      const int kb = klo + 1 < 0 ? 0 : klo + 1;
      const int ke = khi - 1 > N - 1 ? N - 1 : khi - 1;
      if (kb <= ke) run_sum(Gp, kb, ke, ix, iy, iz);
      S[0] = wlo * glo.x + invW * ix + whi * ghi.x;
      S[1] = wlo * glo.y + invW * iy + whi * ghi.y;
      S[2] = wlo * glo.z + invW * iz + whi * ghi.z;
      const float g_lo = Av[0] * glo.x + Av[1] * glo.y + Av[2] * glo.z;
      const float g_hi = Av[0] * ghi.x + Av[1] * ghi.y + Av[2] * ghi.z;
      const float AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
      dLdu = (g_hi - g_lo) * invW;
      dLdh = (g_hi + g_lo - 2.0f * AS) * invW;
    }
    const float AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
    // through A
    const float ka = t.amp * invR;
    const float sb[3] = {ka * S[0], ka * S[1], ka * S[2]};
    const float sbr = sb[0] * rh[0] + sb[1] * rh[1] + sb[2] * rh[2];
    float dLdb[3], dLdr[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dLdb[k] = sb[k] - sbr * rh[k];
      dLdr[k] = -c * sb[k] - sbr * b[k];
    }
    const float dtau = t.dtauh;  // (t1 - t0)/dt
    float dLd_dtau = __fdividef(AS, dtau);
    float dLdR = -AS * invR;
    // through h = |D| dtau / 2
    const float absD = aD.h;
    const float dLdD = dLdh * sgn * 0.5f * dtau;
    dLd_dtau += dLdh * 0.5f * absD;
    // D = 1 - n c
    const float n = 1.0f + t.nm1_m;
    const float dLdn = -c * dLdD;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dLdb[k] -= n * rh[k] * dLdD;
      dLdr[k] -= n * b[k] * dLdD;
    }
    // u_m = tau_m - tau_a + (R + F) / (c dt)
    const float R = gm.R0;
    const RefrGrad<float> rg = refraction_grad<float>(KIND, R, gm.s[2] * M.invH_h, t.Emh, M.N0f, M.invH_h, M.nm1f);
    const float dLdopt = dLdu * M.kc_h;
    dLdR += dLdopt * (1.0f + rg.dF_dR);
    const float dLdzm = dLdopt * rg.dF_dzm + dLdn * rg.dn_dzm;
    const float dLdza = dLdopt * rg.dF_dza;
    dn += dLdopt * rg.dF_dN0 + dLdn * rg.dn_dN0;
    // rhat = d/R, d = x_a - x_m
    const float rdr = dLdr[0] * rh[0] + dLdr[1] * rh[1] + dLdr[2] * rh[2];
    float dLdd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dLdd[k] = (dLdr[k] - rdr * rh[k]) * invR + dLdR * rh[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float dm = -dLdd[k] + (k == 2 ? dLdzm : 0.0f);
      tg[k] += 0.5f * dm;
      tg[3 + k] += 0.5f * dm;
      tg[8 + k] += dLdb[k];
      ga[k] += dLdd[k] + (k == 2 ? dLdza : 0.0f);
    }
    const float idt = M.idt_h;  // 1/dt (per ns)
    tg[6] += (0.5f * dLdu - dLd_dtau) * idt;
    tg[7] += (0.5f * dLdu + dLd_dtau) * idt;
  }

  // gradients of the linear (two-bin) Endpoint deposits of an evaluated pair:
  // the amplitude as for one bin, against the spread of dL/dtrace that the
  // deposit sees, plus its slide with the arrival, dL/du = l(G_J - G_{J-1}),
  // taken through the arrival time (and near Cherenkov through
  // u_a, u_b = u_m -/+ D (t1 - t0)/(2 dt)).  Times in ns, positions in m.
  static __device__ __forceinline__ void adj_deposits_lin(const TrackM& t, const EndpointEvalM& e,
                                                          const MedParams& M, const float4* G, float tg[11],
                                                          float ga[3], float& dn) {
    const int N = M.n_bins;
    float sa, sb;
    const int Ja = lin_cell(e.ua, N, sa);
    const int Jb = lin_cell(e.ub, N, sb);
    const float dNdz_fac = (KIND == C8R_EXPONENTIAL) ? -M.N0f * M.invH_h : 0.0f;
    const float idt = M.idt_h;
    const float amp = t.amp;
    float dd[3], db[3], dns, gv[3], sl[3];
    if (e.branch == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int J = j == 0 ? Ja : Jb;
        if (J < 0 || J > N) continue;
        const GeoM& g = j == 0 ? e.g0 : e.g1;
        const FieldM& f = j == 0 ? e.f0 : e.f1;
        const float E = j == 0 ? t.E0h : t.E1h;
        const float kap = j == 0 ? amp : -amp;
        gather_lin(G, N, J, j == 0 ? sa : sb, gv, sl);
        deposit_grad(g, f, 1.0f + (j == 0 ? t.nm1_0 : t.nm1_1), gv, kap, dd, db, dns);
        for (int c = 0; c < 3; ++c) {
          tg[3 * j + c] -= dd[c];
          ga[c] += dd[c];
          tg[8 + c] += db[c];
        }
        tg[3 * j + 2] += dns * dNdz_fac * E;
        dn += dns * E;
        const float cj = __fdividef(kap, f.D * g.R0) * (f.invR * f.invR);
        const float dLdu = cj * (f.V[0] * sl[0] + f.V[1] * sl[1] + f.V[2] * sl[2]);
        arrival_grad(g, f.invR, E, M, dLdu, tg + 3 * j, nullptr, 1.0f, ga, dn);
        tg[6 + j] += dLdu * idt;
      }
      return;
    }
    const float invR = e.fm.invR;
    if (Ja == Jb) {
      // l = amp (t1 - t0)/dt (g.V)/R with g = G_{J-1} - G_J: the deposit adjoint
      // with D = 1 and n = 0, and dl/d(t1 - t0) = l/(t1 - t0)
      if (Ja < 0 || Ja > N) return;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 g0 = (Ja >= 1 && Ja - 1 < N) ? G[Ja - 1] : z4;
      const float4 g1 = (Ja < N) ? G[Ja] : z4;
      gv[0] = g0.x - g1.x;
      gv[1] = g0.y - g1.y;
      gv[2] = g0.z - g1.z;
      const float kap = amp * t.dtauh;
      deposit_grad(e.gm, e.fm, 1.0f, 0.0f, gv, kap, dd, db, dns);
      for (int c = 0; c < 3; ++c) {
        tg[c] -= 0.5f * dd[c];
        tg[3 + c] -= 0.5f * dd[c];
        ga[c] += dd[c];
        tg[8 + c] += db[c];
      }
      const float l_dtau =
          amp * (gv[0] * e.fm.V[0] + gv[1] * e.fm.V[1] + gv[2] * e.fm.V[2]) * (invR * invR * invR);
      tg[6] -= l_dtau * idt;
      tg[7] += l_dtau * idt;
      return;
    }
    float ga_[3], gb_[3], sla[3], slb[3];
    gather_lin(G, N, Ja, sa, ga_, sla);
    gather_lin(G, N, Jb, sb, gb_, slb);
    gv[0] = ga_[0] - gb_[0];
    gv[1] = ga_[1] - gb_[1];
    gv[2] = ga_[2] - gb_[2];
    deposit_grad(e.gm, e.fm, 1.0f + t.nm1_m, gv, amp, dd, db, dns);
    for (int c = 0; c < 3; ++c) {
      tg[c] -= 0.5f * dd[c];
      tg[3 + c] -= 0.5f * dd[c];
      ga[c] += dd[c];
      tg[8 + c] += db[c];
    }
    tg[2] += 0.5f * dns * dNdz_fac * t.Emh;
    tg[5] += 0.5f * dns * dNdz_fac * t.Emh;
    dn += dns * t.Emh;
    // the slide of the two spread deposits +/- c V
    const float Dm = e.fm.D;
    const float cm = __fdividef(amp, Dm * e.gm.R0) * (invR * invR);
    const float dLdua = cm * (e.fm.V[0] * sla[0] + e.fm.V[1] * sla[1] + e.fm.V[2] * sla[2]);
    const float dLdub = -cm * (e.fm.V[0] * slb[0] + e.fm.V[1] * slb[1] + e.fm.V[2] * slb[2]);
    const float dLdum = dLdua + dLdub;
    const float dLdD = (dLdub - dLdua) * 0.5f * t.dtauh;
    const float dLd_dtau = (dLdub - dLdua) * 0.5f * Dm;
    // D = 1 - n (beta.rhat), rhat = d/R, d = x_a - x_m
    const float n = 1.0f + t.nm1_m;
    const float rh[3] = {e.gm.s[0] * invR, e.gm.s[1] * invR, e.gm.s[2] * invR};
    const float b[3] = {t.bx, t.by, t.bz};
    const float cr = e.fm.bd * invR;
    float dLdr[3];
    for (int k = 0; k < 3; ++k) {
      tg[8 + k] -= n * rh[k] * dLdD;
      dLdr[k] = -n * b[k] * dLdD;
    }
    const float rdr = dLdr[0] * rh[0] + dLdr[1] * rh[1] + dLdr[2] * rh[2];
    for (int k = 0; k < 3; ++k) {
      const float v = (dLdr[k] - rdr * rh[k]) * invR;
      tg[k] -= 0.5f * v;
      tg[3 + k] -= 0.5f * v;
      ga[k] += v;
    }
    const float dLdn = -cr * dLdD;
    tg[2] += 0.5f * dLdn * dNdz_fac * t.Emh;
    tg[5] += 0.5f * dLdn * dNdz_fac * t.Emh;
    dn += dLdn * t.Emh;
    arrival_grad(e.gm, invR, t.Emh, M, dLdum, tg, tg + 3, 0.5f, ga, dn);
    tg[6] += (0.5f * dLdum - dLd_dtau) * idt;
    tg[7] += (0.5f * dLdum + dLd_dtau) * idt;
  }

  // gradients of the deposits of an evaluated pair
  static __device__ __forceinline__ void adj_deposits(const TrackM& t, const EndpointEvalM& e, const MedParams& M,
                                                      const float4* G, float tg[11], float ga[3], float& dn) {
    if constexpr (LIN) {
      adj_deposits_lin(t, e, M, G, tg, ga, dn);
      return;
    }
    const int N = M.n_bins;
    float fa, fb;
    const int ka = bin_raw(e.ua, N, fa);
    const int kb = bin_raw(e.ub, N, fb);
    const bool ina = ka >= 0 && ka < N, inb = kb >= 0 && kb < N;
    const float dNdz_fac = (KIND == C8R_EXPONENTIAL) ? -M.N0f * M.invH_h : 0.0f;
    const float amp = t.amp;
    float dd[3], db[3], dns;
    if (e.branch == 0) {
      for (int j = 0; j < 2; ++j) {
        const bool in = j == 0 ? ina : inb;
        if (!in) continue;
        const int k = j == 0 ? ka : kb;
        const float4 g4 = G[k];
        const float gv[3] = {g4.x, g4.y, g4.z};
        deposit_grad(j == 0 ? e.g0 : e.g1, j == 0 ? e.f0 : e.f1, 1.0f + (j == 0 ? t.nm1_0 : t.nm1_1), gv,
                     j == 0 ? amp : -amp, dd, db, dns);
        const float E = j == 0 ? t.E0h : t.E1h;
        for (int c = 0; c < 3; ++c) {
          tg[3 * j + c] -= dd[c];
          ga[c] += dd[c];
          tg[8 + c] += db[c];
        }
        tg[3 * j + 2] += dns * dNdz_fac * E;
        dn += dns * E;
      }
      return;
    }
    if (ka == kb) return;
    float gv[3];
    const float4 ga4 = ina ? G[ka] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 gb4 = inb ? G[kb] : make_float4(0.f, 0.f, 0.f, 0.f);
    gv[0] = ga4.x - gb4.x;
    gv[1] = ga4.y - gb4.y;
    gv[2] = ga4.z - gb4.z;
    deposit_grad(e.gm, e.fm, 1.0f + t.nm1_m, gv, amp, dd, db, dns);
    for (int c = 0; c < 3; ++c) {
      tg[c] -= 0.5f * dd[c];
      tg[3 + c] -= 0.5f * dd[c];
      ga[c] += dd[c];
      tg[8 + c] += db[c];
    }
    tg[2] += 0.5f * dns * dNdz_fac * t.Emh;
    tg[5] += 0.5f * dns * dNdz_fac * t.Emh;
    dn += dns * t.Emh;
  }
};

#undef TF

// forward and adjoint launches for one deposit shape (one-bin, or linear in a
// translation unit of its own so that the two compile in parallel)
template <bool LIN>
cudaError_t forward_mixed(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                          const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                          cudaStream_t st) {
  FwdArgs a{tiles, n_tiles, ants, n_ant, shape.a_tile, acc, err, FwdGrid{}, M};
  auto go = [&](auto ops) {
    using O = decltype(ops);
    a.replicas = shape.replicas > 1 ? shape.replicas : 1;
    a.replica_stride = (int64_t)n_ant * M.n_bins * O::kAccRows;
    const int64_t ctas = forward_grid(a, shape, sm_count * forward_blocks_per_sm<O>(shape.a_tile),
                                      sizeof(float4) * O::kAccRows);
    return launch_forward_ops<O>(a, ctas, st);
  };
  const bool ex = M.kind == C8R_EXPONENTIAL;
  if (M.kind == C8R_EXPONENTIAL_SPHERICAL)
    return formalism == C8R_ENDPOINT ? go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL_SPHERICAL, LIN>{})
                                     : go(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL_SPHERICAL, LIN>{});
  if (M.kind == C8R_EXPONENTIAL_RAY)
    return formalism == C8R_ENDPOINT ? go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL_RAY, LIN>{})
                                     : go(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL_RAY, LIN>{});
  if constexpr (!LIN) {
    // the one-bin Endpoint kernels come in both arrival forms (M.split) and,
    // for the direct form in the exponential medium, for a flat antenna array
    // (M.flat, OpsMixed::kFlat)
    if (formalism == C8R_ENDPOINT) {
      if (!ex)
        return M.split ? go(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, false, true>{})
                       : go(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, false, false>{});
      if (M.split) return go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, true>{});
      return M.flat ? go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, false, true>{})
                    : go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, false>{});
    }
  }
  if (formalism == C8R_ENDPOINT)
    return ex ? go(OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, LIN>{}) : go(OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, LIN>{});
  // ZHS in the exponential medium: for a flat array the kernel that forms the
  // midpoint's refractivity quotient and the z part of its d once per track
  // (OpsMixed::kFlat)
  if (ex && M.flat) return go(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL, LIN, false, true>{});
  return ex ? go(OpsMixed<C8R_ZHS, C8R_EXPONENTIAL, LIN>{}) : go(OpsMixed<C8R_ZHS, C8R_UNIFORM, LIN>{});
}

template <bool LIN>
cudaError_t backward_mixed(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count, cudaStream_t st) {
  const bool ex = a.M.kind == C8R_EXPONENTIAL;
  if (formalism == C8R_ZHS) {
    if (ex && a.M.flat)
      return launch_backward_ops<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL, LIN, false, true>>(a, shape, sm_count, st);
    return ex ? launch_backward_ops<OpsMixed<C8R_ZHS, C8R_EXPONENTIAL, LIN>>(a, shape, sm_count, st)
              : launch_backward_ops<OpsMixed<C8R_ZHS, C8R_UNIFORM, LIN>>(a, shape, sm_count, st);
  }
  if constexpr (!LIN) {
    if (a.M.split)
      return ex ? launch_backward_ops<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, false, true>>(a, shape, sm_count, st)
                : launch_backward_ops<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, false, true>>(a, shape, sm_count, st);
  }
  return ex ? launch_backward_ops<OpsMixed<C8R_ENDPOINT, C8R_EXPONENTIAL, LIN>>(a, shape, sm_count, st)
            : launch_backward_ops<OpsMixed<C8R_ENDPOINT, C8R_UNIFORM, LIN>>(a, shape, sm_count, st);
}

}  // namespace c8r
