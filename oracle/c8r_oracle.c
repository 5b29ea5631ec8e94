/*
 * c8r_oracle.c -- plain, slow, single-threaded FP64 reference ("oracle") of the
 * track x antenna radio-emission step that the CORSIKA 8 radio module runs for
 * every particle track and every antenna (paper §2, the radio process flow:
 * track -> track filter -> formalism -> propagator -> antenna store).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may use it.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * The paper names the two formalisms (§1: "Endpoint", after James et al.,
 * Phys. Rev. E 84, 056602 (2011); "ZHS", after Zas, Halzen & Stanev,
 * Phys. Rev. D 45, 362 (1992)) and the flow (§2), but prints no equation.  The
 * formulas below are those of the cited works, written in SI units for a charge
 * q*e moving with constant velocity beta*c along a straight track inside a
 * medium of refractive index n.  Readings of points where the paper is silent:
 *
 *  F  track filter (§2 names it, no criteria): keep a track iff q != 0, all
 *     twelve fields are finite, t1 > t0, |x1 - x0| > 0 and 0 < |beta| < 1.
 *  M  straight-line propagator (§2, §4 "simple" propagator): one straight path
 *     x_e -> x_a; uniform medium n_avg = n_src = n; exponential medium
 *     n(z) = 1 + N0 exp(-z/H), n_src = n(z_e), n_avg = path average of n(z),
 *     evaluated in the expm1 form that is exact for every dz; arrival time
 *     t_arr = t_e + n_avg R / c.  The Doppler factor uses n_src.
 *  MS the exponential atmosphere over a spherical Earth (the straight path is
 *     kept; only the altitude is measured from the sphere): centre (0, 0, -R_E),
 *     h(x) = |x - centre| - R_E, n(x) = 1 + N0 exp(-h(x)/H); n_avg R is the
 *     integral of n along the path, by composite 8-point Gauss-Legendre
 *     quadrature (64 panels).
 *  RB curved rays in the flat exponential atmosphere (the propagator's "heavier"
 *     form, §2): the signal follows the ray from x_e to x_a in the vertical plane
 *     through both that keeps n(z) sin(theta) = p (theta from the vertical;
 *     Snell's law for horizontal layers), with rho = horizontal distance,
 *     rho = integral over z between z_a and z_e of p / sqrt(n^2 - p^2), and
 *     arrival delay (1/c) integral of n^2 / sqrt(n^2 - p^2).  The field and the
 *     Doppler factor use the ray's direction at x_e, (sin(theta_e) rhat_h,
 *     +/- cos(theta_e)) with sin(theta_e) = p / n(z_e); the amplitude keeps the
 *     straight distance R (the ray's spreading differs from 1/R by the relative
 *     bending, ~1e-4).  In n decreasing upward the direct ray is the only one for
 *     rho below its grazing limit (some 1e2 km here); a path within 1e-3 of the
 *     horizontal (|z_a - z_e| < 1e-3 R) keeps the straight line.  Integrals by
 *     composite 8-point Gauss-Legendre quadrature (16 panels); p by Newton's
 *     method safeguarded by bisection.
 *  T  binning: bin k of antenna a covers [t_ref + k dt, t_ref + (k+1) dt); a
 *     deposit with k outside [0, N) is dropped.
 *  E  Endpoint: at the start (sign +1) and the end (sign -1) of the track a
 *     field s K V / (D R dt) lands in the arrival bin, K = q e / (4 pi eps0 c),
 *     V = rhat x (rhat x beta), D = 1 - n_src beta.rhat (signed).
 *  C  near-Cherenkov Endpoint: if min(|D0|,|D1|) < eps_C the pair is evaluated
 *     at the track midpoint with linearised arrival times t_arr,m -/+ D_m dt_e/2;
 *     a pair whose two arrivals share a bin contributes exactly zero.
 *  Z  ZHS: bin average of the midpoint step potential K_A beta_perp/(R |D|) over
 *     the arrival interval t_arr,m -/+ |D| dt_e / 2; if the interval lies in one
 *     bin the deposit is K_A beta_perp dt_e / (R dt) (no division by D).
 *  G  adjoint (Endpoint): gradient of a scalar loss whose derivative with respect
 *     to the traces is given, with every bin index and branch decision held
 *     fixed (the traces are piecewise constant in the times).
 *  GZ adjoint (ZHS): the same with the bins of the two interval ends held fixed;
 *     the fractions of the interval that fall in its first and last bin vary
 *     with the interval ends, so the ZHS traces are piecewise linear in the
 *     arrival time and the times get non-zero gradients.
 *  LD linear (two-bin) deposit, an alternative to T for both formalisms: a
 *     deposit arriving at u (in bins from the window start) is spread evenly
 *     over one bin width centred on u, so bin k receives the fraction
 *     |[u - 1/2, u + 1/2] & [k, k + 1)| of it (bins floor(u - 1/2) and the next;
 *     the weight is the tent max(0, 1 - |u - (k + 1/2)|)).  ZHS: the bin weights
 *     are that tent averaged over the arrival interval; when the interval lies
 *     between two consecutive bin centres the tents are linear over it and the
 *     average is the tent at the interval's middle (no division by D).
 *     Endpoint near Cherenkov (C): the two linearised arrivals +/- K V/(D R dt)
 *     are spread the same way; when they lie between the same two bin centres
 *     J - 1/2 and J + 1/2 the result is the exact limit K V dt_e/(R dt^2) into
 *     bin J - 1 and its negative into bin J (no division by D).  The traces are
 *     then continuous in the arrival times, which gives the times informative
 *     gradients; the adjoints hold the bins of the deposits fixed.
 *
 * Parity unpinned: the value eps_C = 1e-3 itself (any value gives a consistent
 * result; the tests pin the branch's formula, not the threshold), the choice
 * of n_src over n_avg in the Doppler factor for a non-uniform medium (the two
 * coincide in a uniform medium, where the closed-form pins run), and, for
 * curved rays (RB), keeping the straight distance R in the amplitude (the ray's
 * path, time and direction are pinned; the amplitude rule is a choice).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define OR_C_LIGHT 299792458.0          /* m/s                        */
#define OR_EPS0 8.8541878128e-12        /* F/m                        */
#define OR_QE 1.602176634e-19           /* C                          */
#define OR_PI 3.14159265358979323846

/* OR_RAY_LINEAR_N2 is an oracle-only profile for the ray tracer's pins:
   n(z)^2 = n^2 + dn2dz z, whose rays have closed forms */
enum { OR_UNIFORM = 0, OR_EXPONENTIAL = 1, OR_EXPONENTIAL_SPHERICAL = 2, OR_EXPONENTIAL_RAY = 3, OR_RAY_LINEAR_N2 = 4 };
enum { OR_ENDPOINT = 0, OR_ZHS = 1 };
/* oracle-only evaluation modes used by the tests: the identity tests force the
   Endpoint midpoint form or sample the ZHS potential at bin edges; MODE_ABS
   accumulates |deposit| per component (the magnitude of the summed terms, the
   scale of the rounding error of any evaluation of the sum) */
enum { OR_MODE_NORMAL = 0, OR_MODE_FORCE_MIDPOINT = 1, OR_MODE_ZHS_EDGE_SAMPLED = 2, OR_MODE_ABS = 3 };
/* deposit shapes: reading T (one bin) or reading LD (spread over one bin width) */
enum { OR_DEPOSIT_BIN = 0, OR_DEPOSIT_LINEAR = 1 };

typedef struct {
  const double *x0, *y0, *z0, *x1, *y1, *z1; /* m                          */
  const double *t0, *t1;                     /* s                          */
  const double *bx, *by, *bz;                /* velocity / c               */
  const double *q;                           /* charge in units of e       */
} or_tracks;

typedef struct {
  int kind;        /* OR_UNIFORM, OR_EXPONENTIAL or OR_EXPONENTIAL_SPHERICAL */
  double n;        /* uniform: refractive index                             */
  double N0;       /* exponential: refractivity at z = 0                    */
  double H;        /* exponential: scale height, m                          */
  double R_E;      /* spherical: Earth radius, m                            */
  double dn2dz;    /* OR_RAY_LINEAR_N2: d(n^2)/dz, 1/m                       */
} or_medium;

typedef struct {
  const double* xyz;   /* [n_ant][3] m                                       */
  const double* t_ref; /* [n_ant] s, start time of bin 0                     */
  int n_ant;
  int n_bins;
  double dt;           /* s                                                  */
} or_antennas;

/* ------------------------------------------------------------------------ */
/* reading F: the track filter                                               */
static int track_kept(const or_tracks* T, int64_t i) {
  double v[12] = {T->x0[i], T->y0[i], T->z0[i], T->x1[i], T->y1[i], T->z1[i],
                  T->t0[i], T->t1[i], T->bx[i], T->by[i], T->bz[i], T->q[i]};
  for (int k = 0; k < 12; ++k)
    if (!isfinite(v[k])) return 0;
  if (T->q[i] == 0.0) return 0;
  if (!(T->t1[i] > T->t0[i])) return 0;
  double lx = v[3] - v[0], ly = v[4] - v[1], lz = v[5] - v[2];
  if (!(lx * lx + ly * ly + lz * lz > 0.0)) return 0;
  double b = sqrt(v[8] * v[8] + v[9] * v[9] + v[10] * v[10]);
  if (!(b > 0.0 && b < 1.0)) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* reading M: refractive index at the source and averaged over the path      */
static void medium_indices(const or_medium* m, double z_e, double z_a, double* n_src, double* n_avg,
                           double* dn_src_dN0, double* dn_src_dze) {
  if (m->kind == OR_UNIFORM) {
    *n_src = m->n;
    *n_avg = m->n;
    *dn_src_dN0 = 1.0; /* n = 1 + N0 in the uniform case */
    *dn_src_dze = 0.0;
    return;
  }
  double E_e = exp(-z_e / m->H);
  *n_src = 1.0 + m->N0 * E_e;
  /* (1/dz) * integral_{z_e}^{z_a} N0 exp(-z/H) dz = N0 E_e (1 - exp(-x)) / x, x = dz/H */
  double x = (z_a - z_e) / m->H;
  double ratio = (x == 0.0) ? 1.0 : (-expm1(-x)) / x;
  *n_avg = 1.0 + m->N0 * E_e * ratio;
  *dn_src_dN0 = E_e;
  *dn_src_dze = -m->N0 * E_e / m->H;
}

/* straight emission path from x_e to antenna x_a (reading M) */
typedef struct {
  double d[3];   /* x_a - x_e                                               */
  double R;      /* |d|                                                     */
  double rh[3];  /* d / R                                                   */
  double n_src, n_avg, dn_src_dN0, dn_src_dze;
} or_path;

/* reading MS: altitude above the sphere, without the cancellation of |x - c| - R_E */
static double sphere_altitude(const or_medium* m, const double x[3]) {
  double zr = x[2] + m->R_E;
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + zr * zr);
  return (x[0] * x[0] + x[1] * x[1] + x[2] * (x[2] + 2.0 * m->R_E)) / (r + m->R_E);
}

/* integral of N0 exp(-h/H) along the straight path xe -> xe + R rhat */
static double sphere_refractive_path(const or_medium* m, const double xe[3], const double rh[3], double R) {
  static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  const int panels = 64;
  double sum = 0.0, hw = 0.5 * R / panels;
  for (int pn = 0; pn < panels; ++pn) {
    double mid = (pn + 0.5) * (R / panels);
    for (int j = 0; j < 4; ++j) {
      for (int sg = -1; sg <= 1; sg += 2) {
        double sdist = mid + sg * hw * xg[j], x[3];
        for (int c = 0; c < 3; ++c) x[c] = xe[c] + sdist * rh[c];
        sum += wg[j] * hw * m->N0 * exp(-sphere_altitude(m, x) / m->H);
      }
    }
  }
  return sum;
}

/* reading RB: the index profile the ray sees */
static double ray_index(const or_medium* m, double z) {
  if (m->kind == OR_RAY_LINEAR_N2) return sqrt(m->n * m->n + m->dn2dz * z);
  return 1.0 + m->N0 * exp(-z / m->H);
}

/* integrals over z in [zlo, zhi] for ray parameter p: out[0] = int p/sqrt(n^2-p^2),
   out[1] = its derivative in p, int n^2/(n^2-p^2)^(3/2), out[2] = int n^2/sqrt(n^2-p^2) */
static void ray_integrals(const or_medium* m, double zlo, double zhi, double p, double out[3]) {
  static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  const int panels = 16;
  double h = (zhi - zlo) / panels, hw = 0.5 * h;
  out[0] = out[1] = out[2] = 0.0;
  for (int pn = 0; pn < panels; ++pn) {
    double mid = zlo + (pn + 0.5) * h;
    for (int j = 0; j < 4; ++j) {
      for (int sg = -1; sg <= 1; sg += 2) {
        double n = ray_index(m, mid + sg * hw * xg[j]);
        double q = n * n - p * p;
        double rq = sqrt(q);
        out[0] += wg[j] * hw * p / rq;
        out[1] += wg[j] * hw * n * n / (q * rq);
        out[2] += wg[j] * hw * n * n / rq;
      }
    }
  }
}

/* reading RB: direction at x_e and arrival delay of the ray from x_e to x_a */
static void ray_path(const or_medium* m, const double xe[3], const double xa[3], or_path* p) {
  double dz = xa[2] - xe[2];
  double rho = sqrt(p->d[0] * p->d[0] + p->d[1] * p->d[1]);
  double n_e = ray_index(m, xe[2]);
  p->n_src = n_e;
  p->dn_src_dN0 = NAN; /* the adjoint is not defined for this medium */
  p->dn_src_dze = NAN;
  double zlo = fmin(xe[2], xa[2]), zhi = fmax(xe[2], xa[2]);
  if (fabs(dz) < 1e-3 * p->R) {
    /* near-horizontal path: the straight line; n_avg = mean of n along it */
    double sum = 0.0;
    static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    for (int pn = 0; pn < 64; ++pn)
      for (int j = 0; j < 4; ++j)
        for (int sg = -1; sg <= 1; sg += 2) {
          double f = ((pn + 0.5) + sg * 0.5 * xg[j]) / 64.0;
          sum += wg[j] * 0.5 / 64.0 * ray_index(m, xe[2] + f * dz);
        }
    p->n_avg = sum;
    return;
  }
  if (rho == 0.0) {
    double I[3];
    ray_integrals(m, zlo, zhi, 0.0, I);
    p->n_avg = I[2] / p->R;
    return;
  }
  /* Newton's method for p in (0, n_top), safeguarded by bisection, from the
     straight line's sine times the mean index over the heights crossed */
  double n_top = ray_index(m, zhi);
  double n_mean = 0.0;
  {
    static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    for (int j = 0; j < 4; ++j)
      for (int sg = -1; sg <= 1; sg += 2) n_mean += 0.5 * wg[j] * ray_index(m, 0.5 * (zlo + zhi) + sg * 0.5 * (zhi - zlo) * xg[j]);
  }
  double lo = 0.0, hi = n_top, pp = fmin(n_mean * rho / p->R, 0.5 * (n_top + n_mean * rho / p->R)), I[3];
  for (int it = 0; it < 100; ++it) {
    ray_integrals(m, zlo, zhi, pp, I);
    double F = I[0] - rho;
    if (F == 0.0) break;
    if (F > 0.0) hi = pp; else lo = pp;
    double step = F / I[1];
    double next = pp - step;
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    /* converged once the step is within a few rounding units of p */
    int done = fabs(next - pp) <= 4e-16 * pp;
    pp = next;
    if (done) break;
  }
  ray_integrals(m, zlo, zhi, pp, I);
  double s_e = pp / n_e, c_e = sqrt(1.0 - s_e * s_e);
  p->rh[0] = s_e * p->d[0] / rho;
  p->rh[1] = s_e * p->d[1] / rho;
  p->rh[2] = (dz < 0.0 ? -1.0 : 1.0) * c_e;
  p->n_avg = I[2] / p->R; /* so that n_avg R / c is the ray's delay */
}

static void propagate(const or_medium* m, const double xe[3], const double xa[3], or_path* p) {
  for (int c = 0; c < 3; ++c) p->d[c] = xa[c] - xe[c];
  p->R = sqrt(p->d[0] * p->d[0] + p->d[1] * p->d[1] + p->d[2] * p->d[2]);
  for (int c = 0; c < 3; ++c) p->rh[c] = p->d[c] / p->R;
  if (m->kind == OR_EXPONENTIAL_RAY || m->kind == OR_RAY_LINEAR_N2) {
    ray_path(m, xe, xa, p);
    return;
  }
  if (m->kind == OR_EXPONENTIAL_SPHERICAL) {
    double E = exp(-sphere_altitude(m, xe) / m->H);
    p->n_src = 1.0 + m->N0 * E;
    p->n_avg = 1.0 + sphere_refractive_path(m, xe, p->rh, p->R) / p->R;
    p->dn_src_dN0 = E;
    p->dn_src_dze = NAN; /* the adjoint is not defined for this medium */
    return;
  }
  medium_indices(m, xe[2], xa[2], &p->n_src, &p->n_avg, &p->dn_src_dN0, &p->dn_src_dze);
}

/* arrival time relative to the antenna's bin-0 edge, in units of dt (reading T) */
static double arrival_in_bins(const or_path* p, double t_e, double t_ref, double dt) {
  return ((t_e - t_ref) + p->n_avg * p->R / OR_C_LIGHT) / dt;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int g_abs_mode = 0; /* set by oracle_forward for OR_MODE_ABS; single-threaded */

static void deposit(double* trace_a, int n_bins, int64_t k, const double v[3], double scale) {
  if (k < 0 || k >= n_bins) return;
  for (int c = 0; c < 3; ++c) trace_a[(int64_t)c * n_bins + k] += g_abs_mode ? fabs(scale * v[c]) : scale * v[c];
}

/* reading LD: the share of a deposit arriving at u that falls in bin k */
static double lin_weight(double u, int64_t k) {
  double lo = fmax(u - 0.5, (double)k), hi = fmin(u + 0.5, (double)(k + 1));
  return hi > lo ? hi - lo : 0.0;
}

static void deposit_linear(double* trace_a, int n_bins, double u, const double v[3], double scale) {
  int64_t k0 = (int64_t)floor(u - 0.5);
  for (int64_t k = k0; k <= k0 + 1; ++k) {
    double w = lin_weight(u, k);
    if (w > 0.0) deposit(trace_a, n_bins, k, v, scale * w);
  }
}

/* integral over [a, b] of lin_weight(u, k) du: the tent is linear between its
   knots k - 1/2, k + 1/2, k + 3/2, so each piece contributes its length times the
   tent at the piece's middle */
static double lin_weight_integral(double a, double b, int64_t k) {
  double knot[3] = {(double)k - 0.5, (double)k + 0.5, (double)k + 1.5};
  double sum = 0.0;
  for (int p = 0; p < 2; ++p) {
    double lo = fmax(a, knot[p]), hi = fmin(b, knot[p + 1]);
    if (hi > lo) sum += (hi - lo) * lin_weight(0.5 * (lo + hi), k);
  }
  return sum;
}

static double K_endpoint(double q) { return q * OR_QE / (4.0 * OR_PI * OR_EPS0 * OR_C_LIGHT); }
static double K_zhs(double q) {
  double mu0 = 1.0 / (OR_EPS0 * OR_C_LIGHT * OR_C_LIGHT);
  return mu0 * q * OR_QE * OR_C_LIGHT / (4.0 * OR_PI);
}

static void track_points(const or_tracks* T, int64_t i, double x0[3], double x1[3], double xm[3], double beta[3]) {
  x0[0] = T->x0[i]; x0[1] = T->y0[i]; x0[2] = T->z0[i];
  x1[0] = T->x1[i]; x1[1] = T->y1[i]; x1[2] = T->z1[i];
  for (int c = 0; c < 3; ++c) xm[c] = 0.5 * (x0[c] + x1[c]);
  beta[0] = T->bx[i]; beta[1] = T->by[i]; beta[2] = T->bz[i];
}

/* V = rhat x (rhat x beta) = (beta.rhat) rhat - beta = -beta_perp */
static void endpoint_vector(const double beta[3], const double rh[3], double V[3]) {
  double c = dot3(beta, rh);
  for (int k = 0; k < 3; ++k) V[k] = c * rh[k] - beta[k];
}

/* ------------------------------------------------------------------------ */
/* Per (track, antenna) evaluation shared by the forward pass and the bin    */
/* listing.  Returns the branch taken: 0 two-endpoint, 1 midpoint (C),       */
/* 2 ZHS single bin, 3 ZHS multi-bin.  u_a/u_b are arrival positions in bins */
/* (start/end, or t1/t2 for branch C, or interval ends for ZHS).             */
typedef struct {
  int branch;
  double u_a, u_b;
} or_pair_info;

static or_pair_info endpoint_pair(const or_tracks* T, int64_t i, const double xa[3], double t_ref, double dt,
                                  int n_bins, const or_medium* m, double eps_C, int mode, int lin, double* trace_a) {
  double x0[3], x1[3], xm[3], beta[3];
  track_points(T, i, x0, x1, xm, beta);
  double K = K_endpoint(T->q[i]);
  double t0 = T->t0[i], t1 = T->t1[i], dte = t1 - t0;
  or_pair_info info;
  or_path p0, p1;
  propagate(m, x0, xa, &p0);
  propagate(m, x1, xa, &p1);
  double D0 = 1.0 - p0.n_src * dot3(beta, p0.rh);
  double D1 = 1.0 - p1.n_src * dot3(beta, p1.rh);
  if (mode != OR_MODE_FORCE_MIDPOINT && fmin(fabs(D0), fabs(D1)) >= eps_C) {
    /* reading E: one deposit per endpoint, start +, end - */
    double u0 = arrival_in_bins(&p0, t0, t_ref, dt);
    double u1 = arrival_in_bins(&p1, t1, t_ref, dt);
    double V[3];
    if (trace_a && lin) {
      endpoint_vector(beta, p0.rh, V);
      deposit_linear(trace_a, n_bins, u0, V, +K / (D0 * p0.R * dt));
      endpoint_vector(beta, p1.rh, V);
      deposit_linear(trace_a, n_bins, u1, V, -K / (D1 * p1.R * dt));
    } else if (trace_a) {
      endpoint_vector(beta, p0.rh, V);
      deposit(trace_a, n_bins, (int64_t)floor(u0), V, +K / (D0 * p0.R * dt));
      endpoint_vector(beta, p1.rh, V);
      deposit(trace_a, n_bins, (int64_t)floor(u1), V, -K / (D1 * p1.R * dt));
    }
    info.branch = 0; info.u_a = u0; info.u_b = u1;
    return info;
  }
  /* reading C: midpoint geometry, linearised arrival times */
  or_path pm;
  propagate(m, xm, xa, &pm);
  double Dm = 1.0 - pm.n_src * dot3(beta, pm.rh);
  double tm = 0.5 * (t0 + t1);
  double tarr_rel = (tm - t_ref) + pm.n_avg * pm.R / OR_C_LIGHT;
  double ua = (tarr_rel - Dm * dte / 2.0) / dt; /* arrival of the start */
  double ub = (tarr_rel + Dm * dte / 2.0) / dt; /* arrival of the end   */
  int64_t ka = (int64_t)floor(ua), kb = (int64_t)floor(ub);
  info.branch = 1; info.u_a = ua; info.u_b = ub;
  if (!trace_a) return info;
  double V[3];
  endpoint_vector(beta, pm.rh, V);
  if (lin) {
    int64_t Ja = (int64_t)floor(ua + 0.5), Jb = (int64_t)floor(ub + 0.5);
    if (Ja == Jb) {
      /* both between the bin centres Ja - 1/2 and Ja + 1/2: the exact limit */
      double B = K * dte / (pm.R * dt * dt);
      deposit(trace_a, n_bins, Ja - 1, V, +B);
      deposit(trace_a, n_bins, Ja, V, -B);
    } else {
      double amp = K / (Dm * pm.R * dt);
      deposit_linear(trace_a, n_bins, ua, V, +amp);
      deposit_linear(trace_a, n_bins, ub, V, -amp);
    }
    return info;
  }
  if (ka != kb) {
    double amp = K / (Dm * pm.R * dt);
    deposit(trace_a, n_bins, ka, V, +amp);
    deposit(trace_a, n_bins, kb, V, -amp);
  }
  return info;
}

static or_pair_info zhs_pair(const or_tracks* T, int64_t i, const double xa[3], double t_ref, double dt, int n_bins,
                             const or_medium* m, int mode, int lin, double* trace_a) {
  double x0[3], x1[3], xm[3], beta[3];
  track_points(T, i, x0, x1, xm, beta);
  double KA = K_zhs(T->q[i]);
  double t0 = T->t0[i], t1 = T->t1[i], dte = t1 - t0;
  or_path pm;
  propagate(m, xm, xa, &pm);
  double bdr = dot3(beta, pm.rh);
  double Dm = 1.0 - pm.n_src * bdr;
  double bperp[3];
  for (int c = 0; c < 3; ++c) bperp[c] = beta[c] - bdr * pm.rh[c];
  double tm = 0.5 * (t0 + t1);
  double tarr_rel = (tm - t_ref) + pm.n_avg * pm.R / OR_C_LIGHT;
  double half = fabs(Dm) * dte / 2.0;
  double t_lo = tarr_rel - half, t_hi = tarr_rel + half;
  double u_lo = t_lo / dt, u_hi = t_hi / dt;
  int64_t k_lo = (int64_t)floor(u_lo), k_hi = (int64_t)floor(u_hi);
  or_pair_info info;
  info.u_a = u_lo; info.u_b = u_hi;
  if (mode == OR_MODE_ZHS_EDGE_SAMPLED) {
    /* the step potential sampled at bin edges e_k = t_ref + k dt, nonzero for
       t_lo < e_k <= t_hi: the form whose edge differences equal the Endpoint
       field of the same track forced to its midpoint */
    info.branch = 3;
    if (trace_a) {
      for (int64_t k = k_lo + 1; k <= k_hi; ++k) {
        if (k < 0 || k >= n_bins) continue;
        deposit(trace_a, n_bins, k, bperp, KA / (pm.R * fabs(Dm)));
      }
    }
    return info;
  }
  if (lin) {
    /* reading LD: the tent weights averaged over [u_lo, u_hi] */
    info.branch = (k_lo == k_hi) ? 2 : 3;
    if (!trace_a) return info;
    double A1 = KA * dte / (pm.R * dt); /* the whole interval's deposit */
    if (floor(u_lo + 0.5) == floor(u_hi + 0.5)) {
      deposit_linear(trace_a, n_bins, 0.5 * (u_lo + u_hi), bperp, A1);
      return info;
    }
    double W = u_hi - u_lo;
    for (int64_t k = (int64_t)floor(u_lo - 0.5); k <= (int64_t)floor(u_hi + 0.5); ++k) {
      if (k < 0 || k >= n_bins) continue;
      double w = lin_weight_integral(u_lo, u_hi, k) / W;
      if (w > 0.0) deposit(trace_a, n_bins, k, bperp, A1 * w);
    }
    return info;
  }
  if (k_lo == k_hi) {
    info.branch = 2;
    if (trace_a) deposit(trace_a, n_bins, k_lo, bperp, KA * dte / (pm.R * dt));
    return info;
  }
  info.branch = 3;
  if (trace_a) {
    int64_t kb = k_lo < 0 ? 0 : k_lo;
    int64_t ke = k_hi > n_bins - 1 ? n_bins - 1 : k_hi;
    for (int64_t k = kb; k <= ke; ++k) {
      double e_lo = (double)k * dt, e_hi = (double)(k + 1) * dt;
      double o = fmin(t_hi, e_hi) - fmax(t_lo, e_lo);
      if (o <= 0.0) continue;
      deposit(trace_a, n_bins, k, bperp, KA / pm.R * (o / fabs(Dm)) / dt);
    }
  }
  return info;
}

/* ------------------------------------------------------------------------ */
/* Forward: traces[a][c][k] (row-major [n_ant][3][n_bins]) are ACCUMULATED.  */
/* Returns the number of tracks kept by the filter.                          */
int64_t oracle_forward(const or_tracks* T, int64_t n, const or_antennas* A, const or_medium* m, int formalism,
                       double eps_C, int mode, int deposit_kind, double* traces) {
  int lin = deposit_kind == OR_DEPOSIT_LINEAR;
  int64_t kept = 0;
  g_abs_mode = (mode == OR_MODE_ABS);
  if (g_abs_mode) mode = OR_MODE_NORMAL;
  for (int64_t i = 0; i < n; ++i) {
    if (!track_kept(T, i)) continue;
    ++kept;
    for (int a = 0; a < A->n_ant; ++a) {
      const double* xa = A->xyz + 3 * (int64_t)a;
      double* tr = traces + (int64_t)a * 3 * A->n_bins;
      if (formalism == OR_ENDPOINT)
        endpoint_pair(T, i, xa, A->t_ref[a], A->dt, A->n_bins, m, eps_C, mode, lin, tr);
      else
        zhs_pair(T, i, xa, A->t_ref[a], A->dt, A->n_bins, m, mode, lin, tr);
    }
  }
  g_abs_mode = 0;
  return kept;
}

/* Per (track, antenna) arrival positions: branch[i*n_ant+a] (-1 if the track is
   filtered out), u[2*(i*n_ant+a)+{0,1}] in bins relative to the antenna's bin-0
   edge: Endpoint start/end (branch 0), t1/t2 (branch C), ZHS interval ends. */
void oracle_arrivals(const or_tracks* T, int64_t n, const or_antennas* A, const or_medium* m, int formalism,
                     double eps_C, int32_t* branch, double* u) {
  for (int64_t i = 0; i < n; ++i) {
    int keep = track_kept(T, i);
    for (int a = 0; a < A->n_ant; ++a) {
      int64_t j = i * A->n_ant + a;
      if (!keep) { branch[j] = -1; u[2 * j] = u[2 * j + 1] = 0.0; continue; }
      const double* xa = A->xyz + 3 * (int64_t)a;
      or_pair_info info = (formalism == OR_ENDPOINT)
                              ? endpoint_pair(T, i, xa, A->t_ref[a], A->dt, A->n_bins, m, eps_C, OR_MODE_NORMAL, 0, 0)
                              : zhs_pair(T, i, xa, A->t_ref[a], A->dt, A->n_bins, m, OR_MODE_NORMAL, 0, 0);
      branch[j] = info.branch;
      u[2 * j] = info.u_a;
      u[2 * j + 1] = info.u_b;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* the refractivity part F of the optical path n_avg R = R + F from x_e to    */
/* x_a (reading M), with its derivatives                                      */
static void refractive_part(const or_medium* m, const double xm[3], const double xa[3], double R, double* F,
                            double* dF_dR, double* dF_dzm, double* dF_dza, double* dF_dN0) {
  if (m->kind == OR_UNIFORM) {
    *F = (m->n - 1.0) * R;
    *dF_dR = m->n - 1.0;
    *dF_dzm = *dF_dza = 0.0;
    *dF_dN0 = R; /* d/d(n - 1) */
    return;
  }
  /* F = N0 E_m R rho(x), rho(x) = (1 - exp(-x))/x, x = (z_a - z_m)/H; rho' = (exp(-x) - rho)/x */
  double E = exp(-xm[2] / m->H);
  double x = (xa[2] - xm[2]) / m->H;
  double rho, drho;
  if (fabs(x) < 1e-3) {
    rho = 1.0 - x / 2.0 + x * x / 6.0 - x * x * x / 24.0;
    drho = -0.5 + x / 3.0 - x * x / 8.0 + x * x * x / 30.0;
  } else {
    rho = -expm1(-x) / x;
    drho = (exp(-x) - rho) / x;
  }
  *F = m->N0 * E * R * rho;
  *dF_dR = m->N0 * E * rho;
  *dF_dzm = -m->N0 * R * E * (rho + drho) / m->H;
  *dF_dza = m->N0 * R * E * drho / m->H;
  *dF_dN0 = E * R * rho;
}

/* chain rule through an arrival time t_e + (R + F)/c: adds dL/dx_e and dL/dx_a
   (into gxe, gxa) and dL/dN0 for a given dL/dt_arr (dL/dt_e is dL/dt_arr) */
static void arrival_adjoint(const or_medium* m, const double xe[3], const double xa[3], const or_path* p,
                            double dL_dtarr, double gxe[3], double gxa[3], double* dN0) {
  double F, dF_dR, dF_dze, dF_dza, dF_dN0;
  refractive_part(m, xe, xa, p->R, &F, &dF_dR, &dF_dze, &dF_dza, &dF_dN0);
  double g = dL_dtarr / OR_C_LIGHT;
  double dR = g * (1.0 + dF_dR);
  for (int k = 0; k < 3; ++k) {
    gxe[k] -= dR * p->rh[k];
    gxa[k] += dR * p->rh[k];
  }
  gxe[2] += g * dF_dze;
  gxa[2] += g * dF_dza;
  *dN0 += g * dF_dN0;
}

/* ------------------------------------------------------------------------ */
/* reading G: reverse-mode gradient of the Endpoint traces.                  */
/* One deposit l = kappa (g.V)/(D R) with upstream g = dL/dtrace at its bin: */
/*   dl/dd    = kappa/(D R^2) [ -(rhat.g) V + c (g - rhat (rhat.g))           */
/*                               - (g.V) (n V / D + rhat) ]                  */
/*   dl/dbeta = kappa/(D R)   [ (rhat.g) rhat - g + (g.V) n rhat / D ]        */
/*   dl/dn    = kappa (g.V) c / (D^2 R)                                       */
/* with d = x_a - x_e, c = beta.rhat, V = c rhat - beta, D = 1 - n c.        */
static void deposit_adjoint(const or_path* p, const double beta[3], const double g[3], double kappa,
                            double gd[3], double gbeta[3], double* gn) {
  const double* rh = p->rh;
  double R = p->R, n = p->n_src;
  double c = dot3(beta, rh);
  double V[3];
  for (int k = 0; k < 3; ++k) V[k] = c * rh[k] - beta[k];
  double D = 1.0 - n * c;
  double gV = dot3(g, V), rg = dot3(rh, g);
  for (int k = 0; k < 3; ++k) {
    gd[k] = kappa / (D * R * R) * (-rg * V[k] + c * (g[k] - rh[k] * rg) - gV * (n * V[k] / D + rh[k]));
    gbeta[k] = kappa / (D * R) * (rg * rh[k] - g[k] + gV * n * rh[k] / D);
  }
  *gn = kappa * gV * c / (D * D * R);
}

static void gather_g(const double* G_a, int n_bins, int64_t k, double g[3]) {
  for (int c = 0; c < 3; ++c) g[c] = (k >= 0 && k < n_bins) ? G_a[(int64_t)c * n_bins + k] : 0.0;
}

/* reading LD: the combination of dL/dtrace that a unit deposit arriving at u
   sees, and its rate of change with u (the deposit slides from bin k0 to k0 + 1) */
static void gather_lin(const double* G_a, int n_bins, double u, double g[3], double slope[3]) {
  int64_t k0 = (int64_t)floor(u - 0.5);
  double w0 = lin_weight(u, k0), w1 = lin_weight(u, k0 + 1), g0[3], g1[3];
  gather_g(G_a, n_bins, k0, g0);
  gather_g(G_a, n_bins, k0 + 1, g1);
  for (int c = 0; c < 3; ++c) {
    g[c] = w0 * g0[c] + w1 * g1[c];
    slope[c] = g1[c] - g0[c];
  }
}

/* G: dL/dtraces [n_ant][3][n_bins].  Outputs are ACCUMULATED:
   track_grad[i][11] = d/d{x0,y0,z0,x1,y1,z1,t0,t1,bx,by,bz}, ant_grad[a][3],
   *dN0 = d/dN0 (exponential) or d/d(n-1) (uniform).  With the linear deposit
   (reading LD) the deposits also slide with their arrival times u: a deposit
   l(g) = kappa (g.V)/(D R) at u adds dL/du = l(G_{k0+1} - G_{k0}), which the
   chain rule takes through the arrival time (arrival_adjoint) and, near
   Cherenkov, through u_a, u_b = tau -/+ D dt_e/(2 dt). */
void oracle_backward(const or_tracks* T, int64_t n, const or_antennas* A, const or_medium* m, double eps_C,
                     int deposit_kind, const double* G, double* track_grad, double* ant_grad, double* dN0) {
  int lin = deposit_kind == OR_DEPOSIT_LINEAR;
  for (int64_t i = 0; i < n; ++i) {
    if (!track_kept(T, i)) continue;
    double x0[3], x1[3], xm[3], beta[3];
    track_points(T, i, x0, x1, xm, beta);
    double K = K_endpoint(T->q[i]);
    double t0 = T->t0[i], t1 = T->t1[i], dte = t1 - t0;
    double* tg = track_grad + 11 * i;
    for (int a = 0; a < A->n_ant; ++a) {
      const double* xa = A->xyz + 3 * (int64_t)a;
      const double* G_a = G + (int64_t)a * 3 * A->n_bins;
      double dt = A->dt, t_ref = A->t_ref[a];
      or_path p0, p1;
      propagate(m, x0, xa, &p0);
      propagate(m, x1, xa, &p1);
      double D0 = 1.0 - p0.n_src * dot3(beta, p0.rh);
      double D1 = 1.0 - p1.n_src * dot3(beta, p1.rh);
      double gd[3], gb[3], gn, g[3];
      if (fmin(fabs(D0), fabs(D1)) >= eps_C) {
        const or_path* ps[2] = {&p0, &p1};
        double ts[2] = {t0, t1};
        for (int j = 0; j < 2; ++j) {
          double u = arrival_in_bins(ps[j], ts[j], t_ref, dt), slope[3];
          if (lin)
            gather_lin(G_a, A->n_bins, u, g, slope);
          else
            gather_g(G_a, A->n_bins, (int64_t)floor(u), g);
          double kappa = (j == 0 ? +K : -K) / dt;
          deposit_adjoint(ps[j], beta, g, kappa, gd, gb, &gn);
          for (int k = 0; k < 3; ++k) {
            tg[3 * j + k] -= gd[k];
            ant_grad[3 * a + k] += gd[k];
            tg[8 + k] += gb[k];
          }
          tg[3 * j + 2] += gn * ps[j]->dn_src_dze;
          *dN0 += gn * ps[j]->dn_src_dN0;
          if (lin) {
            double V[3], gxe[3] = {0.0, 0.0, 0.0};
            endpoint_vector(beta, ps[j]->rh, V);
            double Dj = j == 0 ? D0 : D1;
            double dL_du = kappa * dot3(slope, V) / (Dj * ps[j]->R);
            arrival_adjoint(m, j == 0 ? x0 : x1, xa, ps[j], dL_du / dt, gxe, ant_grad + 3 * a, dN0);
            for (int k = 0; k < 3; ++k) tg[3 * j + k] += gxe[k];
            tg[6 + j] += dL_du / dt;
          }
        }
      } else if (lin) {
        /* reading LD near Cherenkov */
        or_path pm;
        propagate(m, xm, xa, &pm);
        double c = dot3(beta, pm.rh);
        double Dm = 1.0 - pm.n_src * c;
        double tm = 0.5 * (t0 + t1);
        double tarr_rel = (tm - t_ref) + pm.n_avg * pm.R / OR_C_LIGHT;
        double ua = (tarr_rel - Dm * dte / 2.0) / dt;
        double ub = (tarr_rel + Dm * dte / 2.0) / dt;
        double V[3], ga[3], gbv[3];
        endpoint_vector(beta, pm.rh, V);
        int64_t Ja = (int64_t)floor(ua + 0.5), Jb = (int64_t)floor(ub + 0.5);
        if (Ja == Jb) {
          /* l = kappa (g.V)/R with kappa = K dt_e/dt^2 and g = G_{J-1} - G_J: the
             deposit adjoint with D = 1 (n = 0), plus dl/d dt_e = l/dt_e */
          gather_g(G_a, A->n_bins, Ja - 1, ga);
          gather_g(G_a, A->n_bins, Ja, gbv);
          for (int k = 0; k < 3; ++k) g[k] = ga[k] - gbv[k];
          or_path pz = pm;
          pz.n_src = 0.0;
          double kap = K * dte / (dt * dt);
          deposit_adjoint(&pz, beta, g, kap, gd, gb, &gn);
          for (int k = 0; k < 3; ++k) {
            tg[k] -= 0.5 * gd[k];
            tg[3 + k] -= 0.5 * gd[k];
            ant_grad[3 * a + k] += gd[k];
            tg[8 + k] += gb[k];
          }
          double l = kap * dot3(g, V) / pm.R;
          tg[6] -= l / dte;
          tg[7] += l / dte;
          continue;
        }
        double sa[3], sb[3];
        gather_lin(G_a, A->n_bins, ua, ga, sa);
        gather_lin(G_a, A->n_bins, ub, gbv, sb);
        for (int k = 0; k < 3; ++k) g[k] = ga[k] - gbv[k];
        deposit_adjoint(&pm, beta, g, K / dt, gd, gb, &gn);
        for (int k = 0; k < 3; ++k) {
          tg[k] -= 0.5 * gd[k];
          tg[3 + k] -= 0.5 * gd[k];
          ant_grad[3 * a + k] += gd[k];
          tg[8 + k] += gb[k];
        }
        tg[2] += 0.5 * gn * pm.dn_src_dze;
        tg[5] += 0.5 * gn * pm.dn_src_dze;
        *dN0 += gn * pm.dn_src_dN0;
        /* the arrivals slide the deposits +/- amp V, amp = K/(D R dt) */
        double amp = K / (Dm * pm.R * dt);
        double dL_dua = amp * dot3(sa, V), dL_dub = -amp * dot3(sb, V);
        double dL_dtau = (dL_dua + dL_dub) / dt; /* per second of tarr_rel */
        double dL_dD = (dL_dub - dL_dua) * dte / (2.0 * dt);
        double dL_ddte = (dL_dub - dL_dua) * Dm / (2.0 * dt);
        /* D = 1 - n_src (beta.rhat), rhat = d/R, d = x_a - x_m */
        double dL_drh[3];
        for (int k = 0; k < 3; ++k) {
          tg[8 + k] -= pm.n_src * pm.rh[k] * dL_dD;
          dL_drh[k] = -pm.n_src * beta[k] * dL_dD;
        }
        double rdr = dot3(dL_drh, pm.rh);
        for (int k = 0; k < 3; ++k) {
          double dd = (dL_drh[k] - rdr * pm.rh[k]) / pm.R;
          tg[k] -= 0.5 * dd;
          tg[3 + k] -= 0.5 * dd;
          ant_grad[3 * a + k] += dd;
        }
        double dL_dn = -c * dL_dD;
        tg[2] += 0.5 * dL_dn * pm.dn_src_dze;
        tg[5] += 0.5 * dL_dn * pm.dn_src_dze;
        *dN0 += dL_dn * pm.dn_src_dN0;
        double gxm[3] = {0.0, 0.0, 0.0};
        arrival_adjoint(m, xm, xa, &pm, dL_dtau, gxm, ant_grad + 3 * a, dN0);
        for (int k = 0; k < 3; ++k) {
          tg[k] += 0.5 * gxm[k];
          tg[3 + k] += 0.5 * gxm[k];
        }
        tg[6] += 0.5 * dL_dtau - dL_ddte;
        tg[7] += 0.5 * dL_dtau + dL_ddte;
      } else {
        or_path pm;
        propagate(m, xm, xa, &pm);
        double Dm = 1.0 - pm.n_src * dot3(beta, pm.rh);
        double tm = 0.5 * (t0 + t1);
        double tarr_rel = (tm - t_ref) + pm.n_avg * pm.R / OR_C_LIGHT;
        double ua = (tarr_rel - Dm * dte / 2.0) / dt;
        double ub = (tarr_rel + Dm * dte / 2.0) / dt;
        int64_t ka = (int64_t)floor(ua), kb = (int64_t)floor(ub);
        if (ka == kb) continue;
        double ga[3], gbv[3];
        gather_g(G_a, A->n_bins, ka, ga);
        gather_g(G_a, A->n_bins, kb, gbv);
        for (int k = 0; k < 3; ++k) g[k] = ga[k] - gbv[k];
        deposit_adjoint(&pm, beta, g, K / dt, gd, gb, &gn);
        for (int k = 0; k < 3; ++k) {
          tg[k] -= 0.5 * gd[k];
          tg[3 + k] -= 0.5 * gd[k];
          ant_grad[3 * a + k] += gd[k];
          tg[8 + k] += gb[k];
        }
        tg[2] += 0.5 * gn * pm.dn_src_dze;
        tg[5] += 0.5 * gn * pm.dn_src_dze;
        *dN0 += gn * pm.dn_src_dN0;
      }
      /* with the one-bin deposit d/dt0 and d/dt1 stay zero: with bins held
         fixed the deposits do not depend on the times (reading G). */
    }
  }
}

/* ------------------------------------------------------------------------ */
/* reading GZ: reverse-mode gradient of the ZHS traces.  Per pair, with the   */
/* midpoint path (d = x_a - x_m, R, rhat, c = beta.rhat, D = 1 - n_src c,     */
/* beta_perp = beta - c rhat) the deposit into bin k is A w_k, with          */
/*   A   = K_A beta_perp dt_e / (R dt)           (the one-bin deposit),       */
/*   w_k = |[t_lo, t_hi] & bin k| / (t_hi - t_lo)  (1 for a one-bin interval), */
/*   t_lo, t_hi = tau -/+ |D| dt_e / 2,  tau = (t_m - t_ref) + n_avg R / c.   */
/* With S = sum_k w_k G_k, g_lo/g_hi = A.G at the first/last bin (0 outside  */
/* the window) and W = t_hi - t_lo, for a multi-bin interval                 */
/*   dL/dtau  = (g_hi - g_lo) / W,  dL/dhalf = (g_hi + g_lo - 2 A.S) / W,     */
/* and both vanish for a one-bin interval (w = 1).  The rest is the chain     */
/* rule through A, |D|, tau and the path (n_avg R = R + F, F the             */
/* refractivity part of the optical path).                                   */
/* With the linear deposit (reading LD) w_k is the tent of bin k averaged over */
/* the interval; S and the two formulas keep their form, with g_lo, g_hi the */
/* tent-weighted A.G at the interval ends, and for an interval between two   */
/* consecutive bin centres dL/dtau = A.(G_{k0+1} - G_{k0})/dt, dL/dhalf = 0.  */
/* G: dL/dtraces [n_ant][3][n_bins].  Outputs are ACCUMULATED, as for
   oracle_backward (track_grad [n][11], ant_grad [n_ant][3], dN0). */
void oracle_backward_zhs(const or_tracks* T, int64_t n, const or_antennas* A, const or_medium* m, int deposit_kind,
                         const double* G, double* track_grad, double* ant_grad, double* dN0) {
  int lin = deposit_kind == OR_DEPOSIT_LINEAR;
  for (int64_t i = 0; i < n; ++i) {
    if (!track_kept(T, i)) continue;
    double x0[3], x1[3], xm[3], beta[3];
    track_points(T, i, x0, x1, xm, beta);
    double KA = K_zhs(T->q[i]);
    double t0 = T->t0[i], t1 = T->t1[i], dte = t1 - t0, tm = 0.5 * (t0 + t1);
    double* tg = track_grad + 11 * i;
    for (int a = 0; a < A->n_ant; ++a) {
      const double* xa = A->xyz + 3 * (int64_t)a;
      const double* G_a = G + (int64_t)a * 3 * A->n_bins;
      double dt = A->dt, t_ref = A->t_ref[a];
      int nb = A->n_bins;
      or_path pm;
      propagate(m, xm, xa, &pm);
      double c = dot3(beta, pm.rh);
      double D = 1.0 - pm.n_src * c;
      double bperp[3], Av[3];
      for (int k = 0; k < 3; ++k) {
        bperp[k] = beta[k] - c * pm.rh[k];
        Av[k] = KA * bperp[k] * dte / (pm.R * dt);
      }
      double tau = (tm - t_ref) + pm.n_avg * pm.R / OR_C_LIGHT;
      double half = fabs(D) * dte / 2.0;
      double t_lo = tau - half, t_hi = tau + half;
      int64_t k_lo = (int64_t)floor(t_lo / dt), k_hi = (int64_t)floor(t_hi / dt);
      /* S = sum_k w_k G_k over the bins inside the window */
      double S[3] = {0.0, 0.0, 0.0}, g[3];
      double dL_dtau = 0.0, dL_dhalf = 0.0;
      double u_lo = t_lo / dt, u_hi = t_hi / dt;
      if (lin && floor(u_lo + 0.5) == floor(u_hi + 0.5)) {
        double slope[3];
        gather_lin(G_a, nb, 0.5 * (u_lo + u_hi), S, slope);
        dL_dtau = dot3(Av, slope) / dt;
      } else if (lin) {
        double W = t_hi - t_lo, Wb = u_hi - u_lo, slope[3];
        for (int64_t k = (int64_t)floor(u_lo - 0.5); k <= (int64_t)floor(u_hi + 0.5); ++k) {
          double w = lin_weight_integral(u_lo, u_hi, k) / Wb;
          gather_g(G_a, nb, k, g);
          for (int q = 0; q < 3; ++q) S[q] += w * g[q];
        }
        gather_lin(G_a, nb, u_lo, g, slope);
        double g_lo = dot3(Av, g);
        gather_lin(G_a, nb, u_hi, g, slope);
        double g_hi = dot3(Av, g);
        double AS = dot3(Av, S);
        dL_dtau = (g_hi - g_lo) / W;
        dL_dhalf = (g_hi + g_lo - 2.0 * AS) / W;
      } else if (k_lo == k_hi) {
        gather_g(G_a, nb, k_lo, S);
      } else {
        double W = t_hi - t_lo;
        int64_t kb = k_lo < 0 ? 0 : k_lo, ke = k_hi > nb - 1 ? nb - 1 : k_hi;
        for (int64_t k = kb; k <= ke; ++k) {
          double o = fmin(t_hi, (double)(k + 1) * dt) - fmax(t_lo, (double)k * dt);
          if (o <= 0.0) continue;
          gather_g(G_a, nb, k, g);
          for (int q = 0; q < 3; ++q) S[q] += (o / W) * g[q];
        }
        gather_g(G_a, nb, k_lo, g);
        double g_lo = dot3(Av, g);
        gather_g(G_a, nb, k_hi, g);
        double g_hi = dot3(Av, g);
        double AS = dot3(Av, S);
        dL_dtau = (g_hi - g_lo) / W;
        dL_dhalf = (g_hi + g_lo - 2.0 * AS) / W;
      }
      double AS = dot3(Av, S);
      if (AS == 0.0 && dL_dtau == 0.0 && dL_dhalf == 0.0) continue;
      /* through A = K_A beta_perp dt_e / (R dt) */
      double sb[3], dL_dbeta[3], dL_drh[3];
      for (int k = 0; k < 3; ++k) sb[k] = KA * dte / (pm.R * dt) * S[k];
      double sbr = dot3(sb, pm.rh);
      for (int k = 0; k < 3; ++k) {
        dL_dbeta[k] = sb[k] - sbr * pm.rh[k];
        dL_drh[k] = -c * sb[k] - sbr * beta[k];
      }
      double dL_ddte = AS / dte;
      double dL_dR = -AS / pm.R;
      /* through half = |D| dt_e / 2 */
      double sgn = D < 0.0 ? -1.0 : 1.0;
      double dL_dD = dL_dhalf * sgn * dte / 2.0;
      dL_ddte += dL_dhalf * fabs(D) / 2.0;
      /* D = 1 - n_src c */
      double dL_dnsrc = -c * dL_dD;
      for (int k = 0; k < 3; ++k) {
        dL_dbeta[k] += -pm.n_src * pm.rh[k] * dL_dD;
        dL_drh[k] += -pm.n_src * beta[k] * dL_dD;
      }
      /* tau = (t_m - t_ref) + (R + F) / c */
      double F, dF_dR, dF_dzm, dF_dza, dF_dN0;
      refractive_part(m, xm, xa, pm.R, &F, &dF_dR, &dF_dzm, &dF_dza, &dF_dN0);
      double dL_dopt = dL_dtau / OR_C_LIGHT;
      dL_dR += dL_dopt * (1.0 + dF_dR);
      double dL_dzm = dL_dopt * dF_dzm + dL_dnsrc * pm.dn_src_dze;
      double dL_dza = dL_dopt * dF_dza;
      *dN0 += dL_dopt * dF_dN0 + dL_dnsrc * pm.dn_src_dN0;
      /* rhat = d/R, d = x_a - x_m */
      double rdr = dot3(dL_drh, pm.rh), dL_dd[3];
      for (int k = 0; k < 3; ++k) dL_dd[k] = (dL_drh[k] - rdr * pm.rh[k]) / pm.R + dL_dR * pm.rh[k];
      for (int k = 0; k < 3; ++k) {
        double dm = -dL_dd[k] + (k == 2 ? dL_dzm : 0.0);
        tg[k] += 0.5 * dm;
        tg[3 + k] += 0.5 * dm;
        tg[8 + k] += dL_dbeta[k];
        ant_grad[3 * a + k] += dL_dd[k] + (k == 2 ? dL_dza : 0.0);
      }
      tg[6] += 0.5 * dL_dtau - dL_ddte;
      tg[7] += 0.5 * dL_dtau + dL_ddte;
    }
  }
}

/* filter only: writes keep[i] in {0,1}, returns the kept count */
int64_t oracle_filter(const or_tracks* T, int64_t n, uint8_t* keep) {
  int64_t kept = 0;
  for (int64_t i = 0; i < n; ++i) {
    keep[i] = (uint8_t)track_kept(T, i);
    kept += keep[i];
  }
  return kept;
}

/* propagator quantities for one emission point / antenna pair:
   out = {R, n_src, n_avg, arrival delay n_avg R / c (s), direction at x_e (3)} */
void oracle_propagate(const or_medium* m, const double* xe, const double* xa, double* out) {
  or_path p;
  propagate(m, xe, xa, &p);
  out[0] = p.R;
  out[1] = p.n_src;
  out[2] = p.n_avg;
  out[3] = p.n_avg * p.R / OR_C_LIGHT;
  for (int c = 0; c < 3; ++c) out[4 + c] = p.rh[c];
}
