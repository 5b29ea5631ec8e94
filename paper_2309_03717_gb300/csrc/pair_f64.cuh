// pair_f64.cuh -- per (track, antenna) arithmetic of the FP64 path: the plain
// formulas of the two formalisms (§1) and the straight-line propagator (§2) in
// FP64, in the order of their definitions (one exception: the ZHS factor
// K_A/(R |D_m| dt) is formed once per interval rather than once per bin).  This
// translation unit is compiled without FMA contraction so that every operation
// rounds as written.
#pragma once

#include "kernels.cuh"

namespace c8r {

#define TF(f) T[(f) * kTileT + l]

struct EndpointEvalD {
  GeoD g0, g1, gm;
  double V0[3], V1[3], Vm[3];
  double D0, D1, Dm;
  double E0, E1, Em;
  int branch;
  double ua, ub;
  bool valid;
};

__device__ __forceinline__ void field_vec_f64(const double b[3], const GeoD& g, double V[3], double& D) {
  const double c = b[0] * g.rh[0] + b[1] * g.rh[1] + b[2] * g.rh[2];
  V[0] = c * g.rh[0] - b[0];
  V[1] = c * g.rh[1] - b[1];
  V[2] = c * g.rh[2] - b[2];
  D = 1.0 - g.n_src * c;
}

// stop_near: a near-Cherenkov pair stops after the branch decision (branch 1,
// valid false), for a caller that evaluates those pairs in a later pass
__device__ __forceinline__ void endpoint_eval_f64(const double* T, int l, const AntRec& A, const MedParams& M,
                                                  EndpointEvalD& e, bool stop_near = false) {
  e.valid = false;
  e.branch = 0;
  const double b[3] = {TF(fd::BX), TF(fd::BY), TF(fd::BZ)};
  const double x0 = TF(fd::X0), y0 = TF(fd::Y0), z0 = TF(fd::Z0);
  const double x1 = TF(fd::X1), y1 = TF(fd::Y1), z1 = TF(fd::Z1);
  const double t0 = TF(fd::T0), t1 = TF(fd::T1);
  e.E0 = TF(fd::E0);
  e.E1 = TF(fd::E1);
  e.Em = TF(fd::EM);
  geo_f64(M, A, x0, y0, z0, e.E0, e.g0);
  geo_f64(M, A, x1, y1, z1, e.E1, e.g1);
  if (e.g0.R == 0.0 || e.g1.R == 0.0) return;
  field_vec_f64(b, e.g0, e.V0, e.D0);
  field_vec_f64(b, e.g1, e.V1, e.D1);
  if (fmin(fabs(e.D0), fabs(e.D1)) >= M.eps_Cd) {
    e.branch = 0;
    e.ua = arrival_f64(M, e.g0, t0, A.t_ref);
    e.ub = arrival_f64(M, e.g1, t1, A.t_ref);
    e.valid = true;
    return;
  }
  e.branch = 1;
  if (stop_near) return;
  geo_f64(M, A, 0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (z0 + z1), e.Em, e.gm);
  if (e.gm.R == 0.0) return;
  field_vec_f64(b, e.gm, e.Vm, e.Dm);
  const double dte = t1 - t0;
  const double tm = 0.5 * (t0 + t1);
  const double tarr_rel = (tm - A.t_ref) + e.gm.n_avg * e.gm.R * M.inv_c_ns;
  e.ua = (tarr_rel - e.Dm * dte / 2.0) / M.dt_ns;
  e.ub = (tarr_rel + e.Dm * dte / 2.0) / M.dt_ns;
  e.valid = true;
}

// Linear (two-bin) deposit (reading LD), in FP64: a deposit arriving at u
// covers [u - 1/2, u + 1/2]; bin k0 = floor(u - 1/2) receives
// (k0 + 1) - (u - 1/2) of it and bin k0 + 1 receives (u + 1/2) - (k0 + 1).
template <class Sink>
__device__ __forceinline__ void dep_lin_f64(Sink& out, int N, double u, double x, double y, double z) {
  const double k0 = floor(u - 0.5);
  const double w0 = (k0 + 1.0) - (u - 0.5), w1 = (u + 0.5) - (k0 + 1.0);
  if (k0 >= 0.0 && k0 < (double)N && w0 > 0.0) out.dep((int)k0, x * w0, y * w0, z * w0);
  if (k0 + 1.0 >= 0.0 && k0 + 1.0 < (double)N && w1 > 0.0) out.dep((int)k0 + 1, x * w1, y * w1, z * w1);
}

// the share of bin k of a deposit arriving at u (the tent max(0, 1 - |u - k - 1/2|))
__device__ __forceinline__ double lin_share_f64(double u, double k) {
  const double lo = fmax(u - 0.5, k), hi = fmin(u + 0.5, k + 1.0);
  return hi > lo ? hi - lo : 0.0;
}

// integral of that share over u in [a, b]: the tent is linear between its knots
// k - 1/2, k + 1/2, k + 3/2, so each piece is its length times the tent at its
// middle
__device__ __forceinline__ double lin_share_integral_f64(double a, double b, double k) {
  double sum = 0.0;
  for (int p = 0; p < 2; ++p) {
    const double lo = fmax(a, k - 0.5 + p), hi = fmin(b, k + 0.5 + p);
    if (hi > lo) sum += (hi - lo) * lin_share_f64(0.5 * (lo + hi), k);
  }
  return sum;
}

// dL/dtrace seen by a unit deposit at u, and its rate of change with u
__device__ __forceinline__ void gather_lin_f64(const Acc4D* G, int N, double u, double g[3], double slope[3]) {
  const double k0 = floor(u - 0.5);
  const double w0 = (k0 + 1.0) - (u - 0.5), w1 = (u + 0.5) - (k0 + 1.0);
  const Acc4D zero{0.0, 0.0, 0.0, 0.0};
  const Acc4D g0 = (k0 >= 0.0 && k0 < (double)N) ? G[(int)k0] : zero;
  const Acc4D g1 = (k0 + 1.0 >= 0.0 && k0 + 1.0 < (double)N) ? G[(int)k0 + 1] : zero;
  g[0] = w0 * g0.x + w1 * g1.x;
  g[1] = w0 * g0.y + w1 * g1.y;
  g[2] = w0 * g0.z + w1 * g1.z;
  slope[0] = g1.x - g0.x;
  slope[1] = g1.y - g0.y;
  slope[2] = g1.z - g0.z;
}

// a track of a staged tile: the FP64 path reads its fields where it needs them
struct TrackD {
  const double* T;
  int l;
  double q;
};

template <int FORM, bool LIN = false>
struct OpsF64 {
  using acc_t = double;
  using Track = TrackD;
  static constexpr int kPrec = C8R_FP64;
  static constexpr int kTileBytes = kTileBytesF64;
  static constexpr int kMinBlocks = 4;
  // Endpoint (one-bin deposit): the near-Cherenkov pairs (about one in ten on a
  // shower, in most warps) are set aside by the main pass and evaluated
  // together afterwards, so that the midpoint form's FP64 arithmetic runs in
  // full warps instead of holding the other lanes of nearly every warp.  The
  // arithmetic of each pair is the same either way.  (The adjoint, adj_main,
  // evaluates every pair in its main pass; its set-aside lists stay empty.)
  static constexpr bool kDefers = FORM == C8R_ENDPOINT && !LIN;
  static constexpr bool kFastBins = false;
  static constexpr int kBwdMinBlocks = 2;
  static constexpr int kAccRows = 1;      // no box deposits

  static __device__ __forceinline__ AntRec load_ant(const AntRec* p) { return *p; }

  static __device__ __forceinline__ void load(const void* Tv, int l, const MedParams&, TrackD& t) {
    t.T = static_cast<const double*>(Tv);
    t.l = l;
    t.q = t.T[fd::Q * kTileT + l];
  }
  static __device__ __forceinline__ bool live(const TrackD& t) { return t.q != 0.0; }
  template <class Sink>
  static __device__ __forceinline__ void pair(const TrackD& t, const AntRec& A, const MedParams& M, Sink& out) {
    if constexpr (FORM == C8R_ENDPOINT)
      endpoint(t.T, t.l, A, M, out);
    else
      zhs(t.T, t.l, A, M, out);
  }
  // main pass: every pair but (kDefers) the near-Cherenkov ones, returned as
  // kDeferPair with nothing deposited; pair_deferred evaluates those in full
  template <class Sink>
  static __device__ __forceinline__ int pair_main(const TrackD& t, const AntRec& A, const MedParams& M, Sink& out) {
    if constexpr (kDefers) return endpoint(t.T, t.l, A, M, out, true);
    pair(t, A, M, out);
    return kDeferNone;
  }
  template <class Sink>
  static __device__ __forceinline__ void pair_deferred(const TrackD& t, const AntRec& A, const MedParams& M,
                                                       Sink& out) {
    if constexpr (kDefers) pair(t, A, M, out);
  }
  template <class Sink>
  static __device__ __forceinline__ void end_deferred(const void*, int, const AntRec&, const MedParams&, Sink&, int) {}
  static __device__ __forceinline__ bool near_zero_fast(const void*, int, const AntRec&, const MedParams&) {
    return false;
  }

  // returns kDeferPair (nothing deposited) for a near-Cherenkov pair when
  // defer_near is set, kDeferNone otherwise
  template <class Sink>
  static __device__ __forceinline__ int endpoint(const double* T, int l, const AntRec& A, const MedParams& M,
                                                 Sink& out, bool defer_near = false) {
    const double q = TF(fd::Q);
    if (q == 0.0) return kDeferNone;
    const int N = M.n_bins;
    EndpointEvalD e;
    endpoint_eval_f64(T, l, A, M, e, defer_near);
    if (defer_near && e.branch == 1) return kDeferPair;
    if (!e.valid) return kDeferNone;
    out.rec(e.branch, e.ua, e.ub);
    const double K = q * kKendpoint;
    const double dt_s = M.dt_ns * 1e-9;
    if constexpr (LIN) {
      // reading LD
      if (e.branch == 0) {
        const double s0 = +K / (e.D0 * e.g0.R * dt_s);
        const double s1 = -K / (e.D1 * e.g1.R * dt_s);
        dep_lin_f64(out, N, e.ua, s0 * e.V0[0], s0 * e.V0[1], s0 * e.V0[2]);
        dep_lin_f64(out, N, e.ub, s1 * e.V1[0], s1 * e.V1[1], s1 * e.V1[2]);
        return kDeferNone;
      }
      const double Ja = floor(e.ua + 0.5), Jb = floor(e.ub + 0.5);
      if (Ja == Jb) {
        // both arrivals in one cell: the exact limit K (dt_e/dt) V/(R dt) into
        // bin J - 1 and its negative into bin J
        const double B = K * ((TF(fd::T1) - TF(fd::T0)) / M.dt_ns) / (e.gm.R * dt_s);
        if (Ja - 1.0 >= 0.0 && Ja - 1.0 < (double)N) out.dep((int)Ja - 1, B * e.Vm[0], B * e.Vm[1], B * e.Vm[2]);
        if (Ja >= 0.0 && Ja < (double)N) out.dep((int)Ja, -B * e.Vm[0], -B * e.Vm[1], -B * e.Vm[2]);
        return kDeferNone;
      }
      const double s = K / (e.Dm * e.gm.R * dt_s);
      dep_lin_f64(out, N, e.ua, s * e.Vm[0], s * e.Vm[1], s * e.Vm[2]);
      dep_lin_f64(out, N, e.ub, -s * e.Vm[0], -s * e.Vm[1], -s * e.Vm[2]);
      return kDeferNone;
    }
    const double ka = floor(e.ua), kb = floor(e.ub);
    const bool ina = ka >= 0.0 && ka < (double)N, inb = kb >= 0.0 && kb < (double)N;
    if (e.branch == 0) {
      const double s0 = +K / (e.D0 * e.g0.R * dt_s);
      const double s1 = -K / (e.D1 * e.g1.R * dt_s);
      if (ina) out.dep((int)ka, s0 * e.V0[0], s0 * e.V0[1], s0 * e.V0[2]);
      if (inb) out.dep((int)kb, s1 * e.V1[0], s1 * e.V1[1], s1 * e.V1[2]);
      return kDeferNone;
    }
    if (ka == kb) return kDeferNone;  // both linearised arrivals in one bin: zero
    const double s = K / (e.Dm * e.gm.R * dt_s);
    if (ina) out.dep((int)ka, s * e.Vm[0], s * e.Vm[1], s * e.Vm[2]);
    if (inb) out.dep((int)kb, -s * e.Vm[0], -s * e.Vm[1], -s * e.Vm[2]);
    return kDeferNone;
  }

  template <class Sink>
  static __device__ __forceinline__ void zhs(const double* T, int l, const AntRec& A, const MedParams& M, Sink& out) {
    const double q = TF(fd::Q);
    if (q == 0.0) return;
    const int N = M.n_bins;
    const double b[3] = {TF(fd::BX), TF(fd::BY), TF(fd::BZ)};
    const double x0 = TF(fd::X0), y0 = TF(fd::Y0), z0 = TF(fd::Z0);
    const double x1 = TF(fd::X1), y1 = TF(fd::Y1), z1 = TF(fd::Z1);
    const double t0 = TF(fd::T0), t1 = TF(fd::T1);
    const double KA = q * kKzhs;
    GeoD gm;
    geo_f64(M, A, 0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (z0 + z1), TF(fd::EM), gm);
    if (gm.R == 0.0) return;
    const double c = b[0] * gm.rh[0] + b[1] * gm.rh[1] + b[2] * gm.rh[2];
    const double Dm = 1.0 - gm.n_src * c;
    const double bp[3] = {b[0] - c * gm.rh[0], b[1] - c * gm.rh[1], b[2] - c * gm.rh[2]};
    const double dte = t1 - t0;
    const double tm = 0.5 * (t0 + t1);
    const double tarr_rel = (tm - A.t_ref) + gm.n_avg * gm.R * M.inv_c_ns;
    const double half = fabs(Dm) * dte / 2.0;
    const double t_lo = tarr_rel - half, t_hi = tarr_rel + half;
    const double dt = M.dt_ns;
    const double u_lo = t_lo / dt, u_hi = t_hi / dt;
    const double k_lo = floor(u_lo), k_hi = floor(u_hi);
    out.rec(k_lo == k_hi ? 2 : 3, u_lo, u_hi);
    if (!(u_lo < (double)N + 1.0 && u_hi > -1.0)) return;
    if constexpr (LIN) {
      // reading LD: the tent weights averaged over [u_lo, u_hi]
      const double A1 = KA * dte / (gm.R * dt);
      if (floor(u_lo + 0.5) == floor(u_hi + 0.5)) {
        dep_lin_f64(out, N, 0.5 * (u_lo + u_hi), A1 * bp[0], A1 * bp[1], A1 * bp[2]);
        return;
      }
      const double W = u_hi - u_lo;
      const double kb = fmax(floor(u_lo - 0.5), 0.0), ke = fmin(floor(u_hi + 0.5), (double)(N - 1));
      for (double kd = kb; kd <= ke; kd += 1.0) {
        const double w = lin_share_integral_f64(u_lo, u_hi, kd) / W;
        if (w > 0.0) out.dep((int)kd, A1 * w * bp[0], A1 * w * bp[1], A1 * w * bp[2]);
      }
      return;
    }
    if (k_lo == k_hi) {
      const double s = KA * dte / (gm.R * dt);
      if (k_lo >= 0.0 && k_lo < (double)N) out.dep((int)k_lo, s * bp[0], s * bp[1], s * bp[2]);
      return;
    }
    const double kb = fmax(k_lo, 0.0), ke = fmin(k_hi, (double)(N - 1));
    // K_A beta_perp/(R |D_m|) times the overlap o of the interval with the bin,
    // over dt; the factor is formed once for the interval's bins
    const double sc = KA / (gm.R * fabs(Dm) * dt);
    for (double kd = kb; kd <= ke; kd += 1.0) {
      const double e_lo = kd * dt, e_hi = (kd + 1.0) * dt;
      const double o = fmin(t_hi, e_hi) - fmax(t_lo, e_lo);
      if (o <= 0.0) continue;
      const double s = sc * o;
      out.dep((int)kd, s * bp[0], s * bp[1], s * bp[2]);
    }
  }

  template <class Sink>
  static __device__ __forceinline__ void fwd(const void* Tv, int l, const AntRec& A, const MedParams& M, Sink& out) {
    const double* T = static_cast<const double*>(Tv);
    if constexpr (FORM == C8R_ENDPOINT)
      endpoint(T, l, A, M, out);
    else
      zhs(T, l, A, M, out);
  }

  static __device__ __forceinline__ int adj_main(const TrackD& tr, const AntRec& A, const MedParams& M,
                                                 const Acc4D* G, const PrefixFF* Gp, double tg[11], double ga[3],
                                                 double& dn) {
    if constexpr (FORM == C8R_ZHS)
      adj_zhs(tr, A, M, G, Gp, tg, ga, dn);
    else
      adj(tr, A, M, G, tg, ga, dn);
    return kDeferNone;
  }
  static __device__ __forceinline__ void adj_deferred(const TrackD&, const AntRec&, const MedParams&, const Acc4D*,
                                                      const PrefixFF*, double*, double*, double&) {}
  static __device__ __forceinline__ void adj_end_deferred(const void*, int, const AntRec&, const MedParams&,
                                                          const Acc4D*, const c8r_track_grads&, int64_t, double*,
                                                          double&, int) {}

  // ZHS adjoint (bins of the interval ends held fixed; see the mixed path for
  // the formulas): in FP64, times in ns, positions in m
  static __device__ __forceinline__ void adj_zhs(const TrackD& tr, const AntRec& A, const MedParams& M,
                                                 const Acc4D* G, const PrefixFF*, double tg[11], double ga[3],
                                                 double& dn) {
    const double* T = tr.T;
    const int l = tr.l;
    const double q = TF(fd::Q);
    if (q == 0.0) return;
    const int N = M.n_bins;
    const double b[3] = {TF(fd::BX), TF(fd::BY), TF(fd::BZ)};
    const double x0 = TF(fd::X0), y0 = TF(fd::Y0), z0 = TF(fd::Z0);
    const double x1 = TF(fd::X1), y1 = TF(fd::Y1), z1 = TF(fd::Z1);
    const double t0 = TF(fd::T0), t1 = TF(fd::T1);
    const double Em = TF(fd::EM);
    GeoD gm;
    geo_f64(M, A, 0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (z0 + z1), Em, gm);
    if (gm.R == 0.0) return;
    const double c = b[0] * gm.rh[0] + b[1] * gm.rh[1] + b[2] * gm.rh[2];
    const double Dm = 1.0 - gm.n_src * c;
    const double dte = t1 - t0;
    const double tm = 0.5 * (t0 + t1);
    const double tarr_rel = (tm - A.t_ref) + gm.n_avg * gm.R * M.inv_c_ns;
    const double half = fabs(Dm) * dte / 2.0;
    const double dt = M.dt_ns;
    const double u_lo = (tarr_rel - half) / dt, u_hi = (tarr_rel + half) / dt;
    const double k_lo = floor(u_lo), k_hi = floor(u_hi);
    const double KA = q * kKzhs;
    double Av[3];
    for (int k = 0; k < 3; ++k) Av[k] = KA * (b[k] - c * gm.rh[k]) * dte / (gm.R * dt);
    double S[3] = {0.0, 0.0, 0.0};
    double dLdu = 0.0, dLdh = 0.0;  // per bin of u, per bin of h = half/dt
    if constexpr (LIN) {
      // reading LD: S = sum_k w_k G_k with the tent weights averaged over the
      // interval; the interval-end values p = A.(G seen by a deposit at the end)
      double sl[3];
      if (floor(u_lo + 0.5) == floor(u_hi + 0.5)) {
        gather_lin_f64(G, N, 0.5 * (u_lo + u_hi), S, sl);
        dLdu = Av[0] * sl[0] + Av[1] * sl[1] + Av[2] * sl[2];
      } else {
        const double W = u_hi - u_lo;
        const double kb = fmax(floor(u_lo - 0.5), 0.0), ke = fmin(floor(u_hi + 0.5), (double)(N - 1));
        for (double kd = kb; kd <= ke; kd += 1.0) {
          const double w = lin_share_integral_f64(u_lo, u_hi, kd) / W;
          const Acc4D g = G[(int)kd];
          S[0] += w * g.x;
          S[1] += w * g.y;
          S[2] += w * g.z;
        }
        double glo[3], ghi[3];
        gather_lin_f64(G, N, u_lo, glo, sl);
        gather_lin_f64(G, N, u_hi, ghi, sl);
        const double p_lo = Av[0] * glo[0] + Av[1] * glo[1] + Av[2] * glo[2];
        const double p_hi = Av[0] * ghi[0] + Av[1] * ghi[1] + Av[2] * ghi[2];
        const double AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
        dLdu = (p_hi - p_lo) / W;
        dLdh = (p_hi + p_lo - 2.0 * AS) / W;
      }
    } else if (k_lo == k_hi) {
      if (!(k_lo >= 0.0 && k_lo < (double)N)) return;
      const Acc4D g = G[(int)k_lo];
      S[0] = g.x; S[1] = g.y; S[2] = g.z;
    } else {
      // S = sum of (overlap / width) G over the bins of the interval inside the
      // window, bin by bin (the FP64 path does not use the running sums)
      const double W = u_hi - u_lo;
      const bool inlo = k_lo >= 0.0 && k_lo < (double)N, inhi = k_hi >= 0.0 && k_hi < (double)N;
      const Acc4D zero{0.0, 0.0, 0.0, 0.0};
      const Acc4D glo = inlo ? G[(int)k_lo] : zero, ghi = inhi ? G[(int)k_hi] : zero;
      const double kb = fmax(k_lo, 0.0), ke = fmin(k_hi, (double)(N - 1));
      for (double kd = kb; kd <= ke; kd += 1.0) {
        const double o = fmin(u_hi, kd + 1.0) - fmax(u_lo, kd);
        if (o <= 0.0) continue;
        const Acc4D g = G[(int)kd];
        S[0] += (o / W) * g.x;
        S[1] += (o / W) * g.y;
        S[2] += (o / W) * g.z;
      }
      const double g_lo = Av[0] * glo.x + Av[1] * glo.y + Av[2] * glo.z;
      const double g_hi = Av[0] * ghi.x + Av[1] * ghi.y + Av[2] * ghi.z;
      const double AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
      dLdu = (g_hi - g_lo) / W;
      dLdh = (g_hi + g_lo - 2.0 * AS) / W;
    }
    const double AS = Av[0] * S[0] + Av[1] * S[1] + Av[2] * S[2];
    const double ka = KA * dte / (gm.R * dt);
    double sb[3], dLdb[3], dLdr[3];
    for (int k = 0; k < 3; ++k) sb[k] = ka * S[k];
    const double sbr = sb[0] * gm.rh[0] + sb[1] * gm.rh[1] + sb[2] * gm.rh[2];
    for (int k = 0; k < 3; ++k) {
      dLdb[k] = sb[k] - sbr * gm.rh[k];
      dLdr[k] = -c * sb[k] - sbr * b[k];
    }
    // dte enters A and h = |D| dte / (2 dt); u_m = tau_m - tau_a + n_avg R / (c dt)
    double dLd_dte = AS / dte + dLdh * fabs(Dm) / (2.0 * dt);
    double dLdR = -AS / gm.R;
    const double dLdD = dLdh * (Dm < 0.0 ? -1.0 : 1.0) * dte / (2.0 * dt);
    const double dLdn = -c * dLdD;
    for (int k = 0; k < 3; ++k) {
      dLdb[k] -= gm.n_src * gm.rh[k] * dLdD;
      dLdr[k] -= gm.n_src * b[k] * dLdD;
    }
    const RefrGrad<double> rg =
        refraction_grad<double>(M.kind, gm.R, gm.d[2] * M.invH, Em, M.N0, M.invH, M.n - 1.0);
    const double dLdopt = dLdu * M.inv_c_ns / dt;
    dLdR += dLdopt * (1.0 + rg.dF_dR);
    const double dLdzm = dLdopt * rg.dF_dzm + dLdn * rg.dn_dzm;
    const double dLdza = dLdopt * rg.dF_dza;
    dn += dLdopt * rg.dF_dN0 + dLdn * rg.dn_dN0;
    const double rdr = dLdr[0] * gm.rh[0] + dLdr[1] * gm.rh[1] + dLdr[2] * gm.rh[2];
    for (int k = 0; k < 3; ++k) {
      const double dd = (dLdr[k] - rdr * gm.rh[k]) / gm.R + dLdR * gm.rh[k];
      const double dm = -dd + (k == 2 ? dLdzm : 0.0);
      tg[k] += 0.5 * dm;
      tg[3 + k] += 0.5 * dm;
      tg[8 + k] += dLdb[k];
      ga[k] += dd + (k == 2 ? dLdza : 0.0);
    }
    tg[6] += 0.5 * dLdu / dt - dLd_dte;
    tg[7] += 0.5 * dLdu / dt + dLd_dte;
  }

  // chain rule through an arrival position u = (t_e - t_a)/dt + n_avg R/(c dt)
  // of the emission point at d = x_a - x_e (refractivity factor E): adds dL/dx_e
  // x w_e to pos0 (and pos1), dL/dx_a and dL/dN0 (the caller adds dL/dt_e)
  static __device__ __forceinline__ void arrival_grad(const GeoD& g, double E, const MedParams& M, double dLdu,
                                                      double* pos0, double* pos1, double w_e, double ga[3],
                                                      double& dn) {
    const RefrGrad<double> rg = refraction_grad<double>(M.kind, g.R, g.d[2] * M.invH, E, M.N0, M.invH, M.n - 1.0);
    const double dLdopt = dLdu * M.inv_c_ns / M.dt_ns;
    const double dLdR = dLdopt * (1.0 + rg.dF_dR);
    for (int k = 0; k < 3; ++k) {
      const double v = dLdR * g.rh[k];
      ga[k] += v;
      pos0[k] -= w_e * v;
      if (pos1) pos1[k] -= w_e * v;
    }
    pos0[2] += w_e * dLdopt * rg.dF_dzm;
    if (pos1) pos1[2] += w_e * dLdopt * rg.dF_dzm;
    ga[2] += dLdopt * rg.dF_dza;
    dn += dLdopt * rg.dF_dN0;
  }

  // Endpoint adjoint with the linear deposit (reading LD): the amplitude against
  // the spread of dL/dtrace each deposit sees, plus the slide of the deposits with
  // their arrivals (dL/du = l(G_{k0+1} - G_{k0})), through the arrival times and,
  // near Cherenkov, through u_a, u_b = u_m -/+ D dt_e/(2 dt).  Times in ns.
  static __device__ __forceinline__ void adj_lin(const double* T, int l, const EndpointEvalD& e, const double b[3],
                                                 double K, double dt_s, const MedParams& M, const Acc4D* G,
                                                 double tg[11], double ga[3], double& dn) {
    const int N = M.n_bins;
    const double dt = M.dt_ns;
    double dd[3], db[3], dns, gv[3], sl[3];
    if (e.branch == 0) {
      for (int j = 0; j < 2; ++j) {
        const GeoD& g = j == 0 ? e.g0 : e.g1;
        const double* V = j == 0 ? e.V0 : e.V1;
        const double D = j == 0 ? e.D0 : e.D1;
        const double E = j == 0 ? e.E0 : e.E1;
        const double kap = (j == 0 ? K : -K) / dt_s;
        gather_lin_f64(G, N, j == 0 ? e.ua : e.ub, gv, sl);
        const double c = b[0] * g.rh[0] + b[1] * g.rh[1] + b[2] * g.rh[2];
        deposit_adjoint<double>(g.rh, V, c, D, g.R, g.n_src, gv, kap, dd, db, dns);
        const RefrGrad<double> rg =
            refraction_grad<double>(M.kind, g.R, g.d[2] * M.invH, E, M.N0, M.invH, M.n - 1.0);
        for (int cc = 0; cc < 3; ++cc) {
          tg[3 * j + cc] -= dd[cc];
          ga[cc] += dd[cc];
          tg[8 + cc] += db[cc];
        }
        tg[3 * j + 2] += dns * rg.dn_dzm;
        dn += dns * rg.dn_dN0;
        const double dLdu = kap * (V[0] * sl[0] + V[1] * sl[1] + V[2] * sl[2]) / (D * g.R);
        arrival_grad(g, E, M, dLdu, tg + 3 * j, nullptr, 1.0, ga, dn);
        tg[6 + j] += dLdu / dt;
      }
      return;
    }
    const GeoD& g = e.gm;
    const double c = b[0] * g.rh[0] + b[1] * g.rh[1] + b[2] * g.rh[2];
    const double dte = TF(fd::T1) - TF(fd::T0);
    const double Ja = floor(e.ua + 0.5), Jb = floor(e.ub + 0.5);
    if (Ja == Jb) {
      // l = kap (g.V)/R, kap = K (dt_e/dt)/dt_s, g = G_{J-1} - G_J: the deposit
      // adjoint with D = 1 and n = 0, and dl/d dt_e = l/dt_e
      const Acc4D zero{0.0, 0.0, 0.0, 0.0};
      const Acc4D g0 = (Ja - 1.0 >= 0.0 && Ja - 1.0 < (double)N) ? G[(int)Ja - 1] : zero;
      const Acc4D g1 = (Ja >= 0.0 && Ja < (double)N) ? G[(int)Ja] : zero;
      gv[0] = g0.x - g1.x;
      gv[1] = g0.y - g1.y;
      gv[2] = g0.z - g1.z;
      const double kap = K * (dte / dt) / dt_s;
      deposit_adjoint<double>(g.rh, e.Vm, c, 1.0, g.R, 0.0, gv, kap, dd, db, dns);
      for (int cc = 0; cc < 3; ++cc) {
        tg[cc] -= 0.5 * dd[cc];
        tg[3 + cc] -= 0.5 * dd[cc];
        ga[cc] += dd[cc];
        tg[8 + cc] += db[cc];
      }
      const double lv = kap * (gv[0] * e.Vm[0] + gv[1] * e.Vm[1] + gv[2] * e.Vm[2]) / g.R;
      tg[6] -= lv / dte;
      tg[7] += lv / dte;
      return;
    }
    double gav[3], gbv[3], sla[3], slb[3];
    gather_lin_f64(G, N, e.ua, gav, sla);
    gather_lin_f64(G, N, e.ub, gbv, slb);
    for (int cc = 0; cc < 3; ++cc) gv[cc] = gav[cc] - gbv[cc];
    deposit_adjoint<double>(g.rh, e.Vm, c, e.Dm, g.R, g.n_src, gv, K / dt_s, dd, db, dns);
    const RefrGrad<double> rg = refraction_grad<double>(M.kind, g.R, g.d[2] * M.invH, e.Em, M.N0, M.invH, M.n - 1.0);
    for (int cc = 0; cc < 3; ++cc) {
      tg[cc] -= 0.5 * dd[cc];
      tg[3 + cc] -= 0.5 * dd[cc];
      ga[cc] += dd[cc];
      tg[8 + cc] += db[cc];
    }
    tg[2] += 0.5 * dns * rg.dn_dzm;
    tg[5] += 0.5 * dns * rg.dn_dzm;
    dn += dns * rg.dn_dN0;
    // the slide of the two spread deposits +/- s V, s = K/(D R dt_s)
    const double sm = K / (e.Dm * g.R * dt_s);
    const double dLdua = sm * (e.Vm[0] * sla[0] + e.Vm[1] * sla[1] + e.Vm[2] * sla[2]);
    const double dLdub = -sm * (e.Vm[0] * slb[0] + e.Vm[1] * slb[1] + e.Vm[2] * slb[2]);
    const double dLdum = dLdua + dLdub;
    const double dtau = dte / dt;
    const double dLdD = (dLdub - dLdua) * dtau / 2.0;
    const double dLd_dtau = (dLdub - dLdua) * e.Dm / 2.0;
    // D = 1 - n_src (beta.rhat), rhat = d/R, d = x_a - x_m
    double dLdr[3];
    for (int k = 0; k < 3; ++k) {
      tg[8 + k] -= g.n_src * g.rh[k] * dLdD;
      dLdr[k] = -g.n_src * b[k] * dLdD;
    }
    const double rdr = dLdr[0] * g.rh[0] + dLdr[1] * g.rh[1] + dLdr[2] * g.rh[2];
    for (int k = 0; k < 3; ++k) {
      const double v = (dLdr[k] - rdr * g.rh[k]) / g.R;
      tg[k] -= 0.5 * v;
      tg[3 + k] -= 0.5 * v;
      ga[k] += v;
    }
    const double dLdn = -c * dLdD;
    tg[2] += 0.5 * dLdn * rg.dn_dzm;
    tg[5] += 0.5 * dLdn * rg.dn_dzm;
    dn += dLdn * rg.dn_dN0;
    arrival_grad(g, e.Em, M, dLdum, tg, tg + 3, 0.5, ga, dn);
    tg[6] += (0.5 * dLdum - dLd_dtau) / dt;
    tg[7] += (0.5 * dLdum + dLd_dtau) / dt;
  }

  static __device__ __forceinline__ void adj(const TrackD& tr, const AntRec& A, const MedParams& M,
                                             const Acc4D* G, double tg[11], double ga[3], double& dn) {
    static_assert(FORM == C8R_ENDPOINT, "adjoint is defined for the Endpoint formalism");
    const double* T = tr.T;
    const int l = tr.l;
    const double q = TF(fd::Q);
    if (q == 0.0) return;
    const int N = M.n_bins;
    EndpointEvalD e;
    endpoint_eval_f64(T, l, A, M, e);
    if (!e.valid) return;
    const double b[3] = {TF(fd::BX), TF(fd::BY), TF(fd::BZ)};
    const double K = q * kKendpoint;
    const double dt_s = M.dt_ns * 1e-9;
    if constexpr (LIN) {
      adj_lin(T, l, e, b, K, dt_s, M, G, tg, ga, dn);
      return;
    }
    const double ka = floor(e.ua), kb = floor(e.ub);
    const bool ina = ka >= 0.0 && ka < (double)N, inb = kb >= 0.0 && kb < (double)N;
    const bool expo = M.kind == C8R_EXPONENTIAL;
    double dd[3], db[3], dns;
    if (e.branch == 0) {
      for (int j = 0; j < 2; ++j) {
        const bool in = j == 0 ? ina : inb;
        if (!in) continue;
        const int k = (int)(j == 0 ? ka : kb);
        const double gv[3] = {G[k].x, G[k].y, G[k].z};
        const GeoD& g = j == 0 ? e.g0 : e.g1;
        const double* V = j == 0 ? e.V0 : e.V1;
        const double c = b[0] * g.rh[0] + b[1] * g.rh[1] + b[2] * g.rh[2];
        deposit_adjoint<double>(g.rh, V, c, j == 0 ? e.D0 : e.D1, g.R, g.n_src, gv, (j == 0 ? K : -K) / dt_s, dd,
                                db, dns);
        const double E = j == 0 ? e.E0 : e.E1;
        for (int cc = 0; cc < 3; ++cc) {
          tg[3 * j + cc] -= dd[cc];
          ga[cc] += dd[cc];
          tg[8 + cc] += db[cc];
        }
        if (expo) {
          tg[3 * j + 2] += dns * (-M.N0 * E / M.H);
          dn += dns * E;
        } else {
          dn += dns;
        }
      }
      return;
    }
    if (ka == kb) return;
    double gv[3];
    for (int cc = 0; cc < 3; ++cc)
      gv[cc] = (ina ? (&G[(int)ka].x)[cc] : 0.0) - (inb ? (&G[(int)kb].x)[cc] : 0.0);
    const double c = b[0] * e.gm.rh[0] + b[1] * e.gm.rh[1] + b[2] * e.gm.rh[2];
    deposit_adjoint<double>(e.gm.rh, e.Vm, c, e.Dm, e.gm.R, e.gm.n_src, gv, K / dt_s, dd, db, dns);
    for (int cc = 0; cc < 3; ++cc) {
      tg[cc] -= 0.5 * dd[cc];
      tg[3 + cc] -= 0.5 * dd[cc];
      ga[cc] += dd[cc];
      tg[8 + cc] += db[cc];
    }
    if (expo) {
      tg[2] += 0.5 * dns * (-M.N0 * e.Em / M.H);
      tg[5] += 0.5 * dns * (-M.N0 * e.Em / M.H);
      dn += dns * e.Em;
    } else {
      dn += dns;
    }
  }
};

#undef TF

// forward and adjoint launches for one deposit shape
template <bool LIN>
cudaError_t forward_f64(int formalism, const void* tiles, int64_t n_tiles, const AntRec* ants, int n_ant,
                        const MedParams& M, void* acc, const FwdShape& shape, int sm_count, int* err,
                        cudaStream_t st) {
  FwdArgs a{tiles, n_tiles, ants, n_ant, shape.a_tile, acc, err, FwdGrid{}, M};
  auto go = [&](auto ops) {
    using O = decltype(ops);
    const int64_t ctas =
        forward_grid(a, shape, sm_count * forward_blocks_per_sm<O>(shape.a_tile), sizeof(Acc4D) * O::kAccRows);
    return launch_forward_ops<O>(a, ctas, st);
  };
  return formalism == C8R_ENDPOINT ? go(OpsF64<C8R_ENDPOINT, LIN>{}) : go(OpsF64<C8R_ZHS, LIN>{});
}

template <bool LIN>
cudaError_t backward_f64(int formalism, BwdArgs& a, const FwdShape& shape, int sm_count, cudaStream_t st) {
  if (formalism == C8R_ZHS) return launch_backward_ops<OpsF64<C8R_ZHS, LIN>>(a, shape, sm_count, st);
  return launch_backward_ops<OpsF64<C8R_ENDPOINT, LIN>>(a, shape, sm_count, st);
}

}  // namespace c8r
