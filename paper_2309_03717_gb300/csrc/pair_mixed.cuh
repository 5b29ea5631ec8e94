// pair_mixed.cuh -- per (track, antenna) arithmetic of the mixed-precision path.
//
// FP32 field arithmetic; the arrival time, the bin index and the ends of the
// arrival interval are float-float (about 48 significant bits), which keeps the
// bin of every deposit identical to an FP64 evaluation except within ~1e-7 bin
// of an edge.  The Doppler factor D = 1 - n beta.rhat is formed without the
// cancellation of the direct form (see field_mixed), from 1 - n|beta| computed
// per track in FP64 by the ingest kernel.
#pragma once

#include "kernels.cuh"

namespace c8r {

// track fields of lane l in a field-major tile
#define TF(f) T[(f) * kTileT + l]

// geometry shared by the forward and the adjoint Endpoint evaluation
struct EndpointEvalM {
  GeoM g0, g1, gm;
  FieldM f0, f1, fm;
  float n0, n1, nm;
  float E0h, E1h, Emh;
  int branch;     // 0 two endpoints, 1 midpoint
  ff ua, ub;      // arrivals (start/end, or the two linearised midpoint arrivals)
  bool valid;
};

template <int KIND>
__device__ __forceinline__ void endpoint_eval_mixed(const float* T, int l, const AntRec& A, const MedParams& M,
                                                    EndpointEvalM& e) {
  e.valid = false;
  const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ);
  const float bmag = TF(fm::BMAG), omb = TF(fm::OMB);
  e.E0h = e.E1h = e.Emh = 1.0f;
  // n - 1 is formed directly (N0 E, or the uniform n - 1 rounded from FP64): as
  // (1 + x) - 1 in FP32 it would lose ~6e-8, comparable to D near Cherenkov
  float nm1_0 = M.nm1f, nm1_1 = M.nm1f;
  if (KIND == C8R_EXPONENTIAL) {
    e.E0h = TF(fm::E0H);
    e.E1h = TF(fm::E1H);
    nm1_0 = __fmul_rn(M.N0f, e.E0h);
    nm1_1 = __fmul_rn(M.N0f, e.E1h);
  }
  e.n0 = __fadd_rn(1.0f, nm1_0);
  e.n1 = __fadd_rn(1.0f, nm1_1);
  // 1 - n|beta| = (1 - |beta|) - (n - 1)|beta|
  const float om0 = __fsub_rn(omb, __fmul_rn(nm1_0, bmag));
  const float om1 = __fsub_rn(omb, __fmul_rn(nm1_1, bmag));
  geo_lite(A, TF(fm::X0), TF(fm::Y0), TF(fm::Z0), 0.f, 0.f, 0.f, e.g0);
  geo_lite(A, TF(fm::X1), TF(fm::Y1), TF(fm::Z1), 0.f, 0.f, 0.f, e.g1);
  if (e.g0.R0 == 0.0f || e.g1.R0 == 0.0f) return;  // emission point on the antenna: outside the domain
  field_mixed(e.g0, bx, by, bz, bmag, om0, e.n0, e.f0);
  field_mixed(e.g1, bx, by, bz, bmag, om1, e.n1, e.f1);
  const bool mid = !(fminf(fabsf(e.f0.D), fabsf(e.f1.D)) >= M.eps_C);
  e.branch = mid ? 1 : 0;
  float Eml = 0.0f;
  if (mid) {
    // near-Cherenkov: midpoint geometry, arrivals t_m -/+ D_m dt_e/2
    float nm1_m = M.nm1f;
    if (KIND == C8R_EXPONENTIAL) {
      e.Emh = TF(fm::EMH);
      Eml = TF(fm::EML);
      nm1_m = __fmul_rn(M.N0f, e.Emh);
    }
    e.nm = __fadd_rn(1.0f, nm1_m);
    midpoint_from_endpoints(e.g0, e.g1, e.f0, e.f1, bmag, __fsub_rn(omb, __fmul_rn(nm1_m, bmag)), e.nm, e.gm, e.fm);
    if (e.gm.R0 == 0.0f) return;
  }
  // arrival times: both endpoints, or the midpoint alone (one code path for both
  // branches, so a warp mixing them does not run two copies of it)
  ff u0 = {0.0f, 0.0f}, u1 = {0.0f, 0.0f};
#pragma unroll 1
  for (int j = 0; j < (mid ? 1 : 2); ++j) {
    GeoM g = (j == 0) ? (mid ? e.gm : e.g0) : e.g1;
    float th, tl, Eh, El;
    if (mid) {
      two_sum(TF(fm::TAU0H), TF(fm::TAU1H), th, tl);
      tl = __fadd_rn(tl, __fadd_rn(TF(fm::TAU0L), TF(fm::TAU1L)));
      th *= 0.5f;
      tl *= 0.5f;
      Eh = e.Emh;
      El = Eml;
    } else {
      th = j == 0 ? TF(fm::TAU0H) : TF(fm::TAU1H);
      tl = j == 0 ? TF(fm::TAU0L) : TF(fm::TAU1L);
      Eh = j == 0 ? e.E0h : e.E1h;
      El = KIND == C8R_EXPONENTIAL ? (j == 0 ? TF(fm::E0L) : TF(fm::E1L)) : 0.0f;
    }
    geo_refine(g);
    const ff u = arrival_mixed(M, A, g, th, tl, Eh, El);
    if (j == 0)
      u0 = u;
    else
      u1 = u;
  }
  if (!mid) {
    e.ua = u0;
    e.ub = u1;
  } else {
    float hh, hl;  // D_m (t1 - t0)/(2 dt)
    two_prod(e.fm.D, TF(fm::DTAUH), hh, hl);
    hl = __fmaf_rn(e.fm.D, TF(fm::DTAUL), hl);
    hh *= 0.5f;
    hl *= 0.5f;
    const ff um = u0;
    two_sum(um.h, -hh, e.ua.h, e.ua.l);
    e.ua.l = __fadd_rn(e.ua.l, __fsub_rn(um.l, hl));
    two_sum(um.h, hh, e.ub.h, e.ub.l);
    e.ub.l = __fadd_rn(e.ub.l, __fadd_rn(um.l, hl));
  }
  e.valid = true;
}

template <int FORM, int KIND>
struct OpsMixed {
  using acc_t = float;
  static constexpr int kPrec = C8R_MIXED;
  static constexpr int kTileBytes = kTileBytesMixed;

  // -------------------------------------------------------------------------
  // Endpoint (§1; James et al.): +amp V/(D R) at the start's arrival bin and
  // -amp V/(D R) at the end's, amp = q K / dt; midpoint form near Cherenkov.
  // -------------------------------------------------------------------------
  template <class Sink>
  static __device__ __forceinline__ void endpoint(const float* T, int l, const AntRec& A, const MedParams& M,
                                                  Sink& out) {
    const float amp = TF(fm::AMPE);
    if (amp == 0.0f) return;  // filtered track or padding
    const int N = M.n_bins;
    EndpointEvalM e;
    endpoint_eval_mixed<KIND>(T, l, A, M, e);
    if (!e.valid) return;
    out.rec(e.branch, e.ua, e.ub);
    float fa, fb;
    const int ka = bin_raw(e.ua, N, fa);
    const int kb = bin_raw(e.ub, N, fb);
    const bool ina = ka >= 0 && ka < N, inb = kb >= 0 && kb < N;
    if (e.branch == 0) {
      const float c0 = __fdividef(amp, e.f0.D * e.g0.R0) * (e.f0.invR * e.f0.invR);
      const float c1 = __fdividef(-amp, e.f1.D * e.g1.R0) * (e.f1.invR * e.f1.invR);
      if (ina && inb && ka == kb) {
        // both deposits in one bin: add them in registers, one set of atomics
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
  static __device__ __forceinline__ void zhs(const float* T, int l, const AntRec& A, const MedParams& M, Sink& out) {
    if (TF(fm::AMPE) == 0.0f) return;
    const float ampz = TF(fm::AMPZ);
    const int N = M.n_bins;
    const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ);
    const float bmag = TF(fm::BMAG), omb = TF(fm::OMB);
    float mx, mxl, my, myl, mz, mzl;
    two_sum(TF(fm::X0), TF(fm::X1), mx, mxl);
    two_sum(TF(fm::Y0), TF(fm::Y1), my, myl);
    two_sum(TF(fm::Z0), TF(fm::Z1), mz, mzl);
    mx *= 0.5f; mxl *= 0.5f; my *= 0.5f; myl *= 0.5f; mz *= 0.5f; mzl *= 0.5f;
    GeoM gm;
    geo_mixed(A, mx, my, mz, mxl, myl, mzl, gm);
    if (gm.R0 == 0.0f) return;
    float Emh = 1.0f, Eml = 0.0f, nm1 = M.nm1f;
    if (KIND == C8R_EXPONENTIAL) {
      Emh = TF(fm::EMH);
      Eml = TF(fm::EML);
      nm1 = __fmul_rn(M.N0f, Emh);
    }
    FieldM f;
    field_mixed(gm, bx, by, bz, bmag, __fsub_rn(omb, __fmul_rn(nm1, bmag)), __fadd_rn(1.0f, nm1), f);
    float th, tl;
    two_sum(TF(fm::TAU0H), TF(fm::TAU1H), th, tl);
    tl = __fadd_rn(tl, __fadd_rn(TF(fm::TAU0L), TF(fm::TAU1L)));
    const ff um = arrival_mixed(M, A, gm, 0.5f * th, 0.5f * tl, Emh, Eml);
    const float aD = fabsf(f.D);
    float hh, hl;  // |D| (t1 - t0)/(2 dt)
    two_prod(aD, TF(fm::DTAUH), hh, hl);
    hl = __fmaf_rn(aD, TF(fm::DTAUL), hl);
    hh *= 0.5f;
    hl *= 0.5f;
    ff ulo, uhi;
    two_sum(um.h, -hh, ulo.h, ulo.l);
    ulo.l = __fadd_rn(ulo.l, __fsub_rn(um.l, hl));
    two_sum(um.h, hh, uhi.h, uhi.l);
    uhi.l = __fadd_rn(uhi.l, __fadd_rn(um.l, hl));
    const float s = -ampz * (f.invR * f.invR) * f.invR;  // beta_perp = -V
    const float Mx = s * f.V[0], My = s * f.V[1], Mz = s * f.V[2];
    float flo, fhi;
    const int klo = bin_raw(ulo, N, flo);
    const int khi = bin_raw(uhi, N, fhi);
    out.rec(klo == khi ? 2 : 3, ulo, uhi);
    if (klo == khi) {
      if (klo >= 0 && klo < N) out.dep(klo, Mx, My, Mz);
      return;
    }
    const float invW = __fdividef(1.0f, 2.0f * hh);  // 1 / interval length in bins
    const int kb = klo < 0 ? 0 : klo;
    const int ke = khi > N - 1 ? N - 1 : khi;
    for (int k = kb; k <= ke; ++k) {
      float o = 1.0f;
      if (k == klo) o = 1.0f - flo;
      if (k == khi) o = fhi;
      const float w = o * invW;
      if (w > 0.0f) out.dep(k, Mx * w, My * w, Mz * w);
    }
  }

  template <class Sink>
  static __device__ __forceinline__ void fwd(const void* Tv, int l, const AntRec& A, const MedParams& M, Sink& out) {
    const float* T = static_cast<const float*>(Tv);
    if constexpr (FORM == C8R_ENDPOINT)
      endpoint(T, l, A, M, out);
    else
      zhs(T, l, A, M, out);
  }

  // -------------------------------------------------------------------------
  // adjoint of `endpoint` with bins and branch held fixed
  // -------------------------------------------------------------------------
  static __device__ __forceinline__ void deposit_grad(const GeoM& g, const FieldM& f, float bx, float by, float bz,
                                                      float n, const float gv[3], float kappa, float dd[3],
                                                      float db[3], float& dns) {
    const float invR = f.invR;
    const float rh[3] = {g.s[0] * invR, g.s[1] * invR, g.s[2] * invR};
    const float inv2 = invR * invR;
    const float V[3] = {f.V[0] * inv2, f.V[1] * inv2, f.V[2] * inv2};
    const float c = f.bd * invR;
    deposit_adjoint<float>(rh, V, c, f.D, g.R0, n, gv, kappa, dd, db, dns);
    (void)bx;
    (void)by;
    (void)bz;
  }

  static __device__ __forceinline__ void adj(const void* Tv, int l, const AntRec& A, const MedParams& M,
                                             const float* G, float tg[11], float ga[3], float& dn) {
    static_assert(FORM == C8R_ENDPOINT, "adjoint is defined for the Endpoint formalism");
    const float* T = static_cast<const float*>(Tv);
    const float amp = TF(fm::AMPE);
    if (amp == 0.0f) return;
    const int N = M.n_bins;
    EndpointEvalM e;
    endpoint_eval_mixed<KIND>(T, l, A, M, e);
    if (!e.valid) return;
    float fa, fb;
    const int ka = bin_raw(e.ua, N, fa);
    const int kb = bin_raw(e.ub, N, fb);
    const bool ina = ka >= 0 && ka < N, inb = kb >= 0 && kb < N;
    const float bx = TF(fm::BX), by = TF(fm::BY), bz = TF(fm::BZ);
    const float dNdz_fac = (KIND == C8R_EXPONENTIAL) ? -M.N0f * M.invH_h : 0.0f;
    float dd[3], db[3], dns;
    if (e.branch == 0) {
      for (int j = 0; j < 2; ++j) {
        const bool in = j == 0 ? ina : inb;
        if (!in) continue;
        const int k = j == 0 ? ka : kb;
        const float gv[3] = {G[k], G[N + k], G[2 * N + k]};
        deposit_grad(j == 0 ? e.g0 : e.g1, j == 0 ? e.f0 : e.f1, bx, by, bz, j == 0 ? e.n0 : e.n1, gv,
                     j == 0 ? amp : -amp, dd, db, dns);
        const float E = j == 0 ? e.E0h : e.E1h;
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
    for (int c = 0; c < 3; ++c) gv[c] = (ina ? G[c * N + ka] : 0.0f) - (inb ? G[c * N + kb] : 0.0f);
    deposit_grad(e.gm, e.fm, bx, by, bz, e.nm, gv, amp, dd, db, dns);
    for (int c = 0; c < 3; ++c) {
      tg[c] -= 0.5f * dd[c];
      tg[3 + c] -= 0.5f * dd[c];
      ga[c] += dd[c];
      tg[8 + c] += db[c];
    }
    tg[2] += 0.5f * dns * dNdz_fac * e.Emh;
    tg[5] += 0.5f * dns * dNdz_fac * e.Emh;
    dn += dns * e.Emh;
  }
};

#undef TF

}  // namespace c8r
