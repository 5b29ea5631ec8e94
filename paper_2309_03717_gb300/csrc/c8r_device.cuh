// c8r_device.cuh -- device-side building blocks of libc8r (sm_103a).
//
// The per-pair arithmetic follows the step the paper (§2) describes for every
// track and antenna: straight-line propagator -> formalism (Endpoint or ZHS,
// §1) -> deposit into the antenna's time-binned trace.  The formulas are those
// of the cited formalism papers (Endpoint: James et al., PRE 84 056602; ZHS:
// Zas, Halzen & Stanev, PRD 45 362), in SI units with times in ns at the
// interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/c8r.h"

namespace c8r {

// ---------------------------------------------------------------------------
// physical constants (SI) and units
// ---------------------------------------------------------------------------
constexpr double kC = 299792458.0;              // m/s
constexpr double kCns = 0.299792458;            // m/ns
constexpr double kEps0 = 8.8541878128e-12;      // F/m
constexpr double kQe = 1.602176634e-19;         // C
constexpr double kPi = 3.14159265358979323846;
// Endpoint: K = e / (4 pi eps0 c)  [V s] per unit charge
constexpr double kKendpoint = kQe / (4.0 * kPi * kEps0 * kC);
// ZHS: K_A = mu0 e c / (4 pi), mu0 = 1/(eps0 c^2)  [V s] per unit charge
constexpr double kKzhs = (1.0 / (kEps0 * kC * kC)) * kQe * kC / (4.0 * kPi);

// tracks per derived tile (the unit of the TMA bulk copies)
constexpr int kTileT = 128;

// ---------------------------------------------------------------------------
// derived-track tiles written by the ingest kernel: per tile of kTileT tracks,
// field-major ([field][kTileT]) so one bulk copy moves a whole tile and lane i
// of a warp reads track i of a field without bank conflicts.
// ---------------------------------------------------------------------------
namespace fm {  // mixed precision (float fields)
enum : int {
  X0, Y0, Z0, X1, Y1, Z1,         // FP32 positions, m
  BX, BY, BZ,                     // beta
  AMPE,                           // q K / dt  [V]; 0 => track dropped by the filter
  AMPZ,                           // q K_A (t1 - t0)/dt  [V s]
  BMAG,                           // |beta|
  OMB,                            // 1 - |beta|
  TAU0H, TAU0L, TAU1H, TAU1L,     // t/dt, float-float
  DTAUH, DTAUL,                   // (t1 - t0)/dt, float-float
  E0H, E0L, E1H, E1L, EMH, EML,   // exp(-z/H) at start, end, midpoint (float-float)
  NFIELDS
};
}
namespace fd {  // FP64 path (double fields)
enum : int { X0, Y0, Z0, X1, Y1, Z1, BX, BY, BZ, Q, T0, T1, E0, E1, EM, NFIELDS };
}
constexpr int kTileBytesMixed = fm::NFIELDS * kTileT * 4;
constexpr int kTileBytesF64 = fd::NFIELDS * kTileT * 8;
static_assert(kTileBytesMixed % 16 == 0 && kTileBytesF64 % 16 == 0, "bulk copies move multiples of 16 bytes");

// ---------------------------------------------------------------------------
// antenna record (device table, built on the host in FP64)
// ---------------------------------------------------------------------------
struct AntRec {
  double x, y, z;        // m
  double t_ref;          // ns, first bin edge
  double Ea;             // exp(-z/H) (exponential medium), 1 otherwise
  // t_ref/dt + k z (k = n/(c dt) in the uniform medium, 1/(c dt) in the
  // exponential one) as float-float: the antenna's part of the shifted arrival
  // time of the FP32 arrival (arrival_fast)
  float Tah, Tal;
  float xh, yh, zh, xl, yl, zl;  // position as float-float
  float tauh, taul;              // t_ref / dt as float-float
  float Eah, Eal;                // Ea as float-float
  // constants of the error bound of the FP32 arrival (arrival_bin_fast):
  // fb_abs = 2 x bins per metre x |low part of the position| + 16 u^2 |T_a| +
  // 1e-6 bin, and fb_rel_v = |z_l| / (1e-3 H), the relative error of the
  // refractivity term from the low part of the altitude (exponential medium;
  // 0 otherwise)
  float fb_abs, fb_rel_v;
};
static_assert(sizeof(AntRec) == 96, "antenna record layout");
static_assert(offsetof(AntRec, xh) % 16 == 0 && offsetof(AntRec, Tah) % 8 == 0,
              "the mixed path loads the float part as float4s and the shifted time as a float2");

// medium + binning parameters (kernel argument)
struct MedParams {
  int kind;              // C8R_UNIFORM / C8R_EXPONENTIAL
  int n_bins;
  double n;              // uniform index
  double N0, H, invH;    // exponential
  double R_E;            // spherical: Earth radius (m)
  double dt_ns;
  double inv_c_ns;       // 1 / c in ns/m
  double eps_Cd;         // near-Cherenkov threshold (FP64 path)
  // float-float constants of the mixed path
  float kc_h, kc_l;      // 1/(c dt): bins per metre
  float s_h, s_l;        // uniform: n/(c dt)
  float cN_h, cN_l;      // exponential: N0 H /(c dt)
  float invH_h, invH_l;  // 1/H
  float N0f, nf;         // N0 and n as floats
  float idt_h, idt_l;    // 1/dt (per ns)
  float ampE;            // K/dt of the Endpoint amplitude (per unit charge), FP64 rounded once
  float kzhs;            // K_A of the ZHS amplitude
  float nm1f;            // uniform: n - 1 formed in FP64, then rounded (never (1 + x) - 1 in FP32)
  float RE_f;            // spherical: Earth radius (m)
  float eps_C;           // near-Cherenkov threshold
  uint32_t wait_limit;   // polls of a bounded wait on a staged track tile before it gives up
  // the form of the FP32 arrival (Endpoint, one-bin deposit, plain media): the
  // centroid of the antenna array, which the ingest's count of tracks seen
  // from above within 45 degrees refers to, and the host's choice from that
  // count (1: the split form of x = R - w)
  float cen_x, cen_y, cen_z;
  int split;
  // a flat antenna array (every antenna at one altitude z_a, exponential
  // medium): z_a and exp(-z_a/H) as float-float, the same values the antenna
  // records hold, so that the quotient (E_e - E_a)/(z_a - z_e) of the
  // refractivity term, the same for every antenna, can be formed once per
  // track (OpsMixed::kFlat)
  int flat;
  float flat_zh, flat_zl, flat_Eh, flat_El;
};

// ---------------------------------------------------------------------------
// float-float ("double-float") arithmetic: error-free transformations after
// Knuth (TwoSum) and Dekker / the FMA form (TwoProd).  Intrinsics pin the
// rounding of every step; nothing here may be contracted or reassociated.
// ---------------------------------------------------------------------------
struct ff {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// Dekker's Fast2Sum: exact when the exponent of a is at least that of b
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy; dst/src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each try_wait itself suspends for a
// while) and returns false.  Callers turn a give-up into an error status.
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

// error word written by kernels that gave up a bounded wait
enum : int { kErrNone = 0, kErrWaitTimeout = 1, kErrCancelled = 2 };

// ---------------------------------------------------------------------------
// FP64 path: the plain formulas in FP64, in the order of their definition.
// ---------------------------------------------------------------------------
struct GeoD {
  double d[3], R, rh[3], n_src, n_avg;
};

// ---------------------------------------------------------------------------
// exponential atmosphere over a spherical Earth (centre (0, 0, -R_E)): the
// altitude excess of a point over the flat altitude z,
//   delta = h - z = |x - centre| - R_E - z = rho^2 / (|x - centre| + z + R_E),
// written without the cancellation of the first form.  The optical path is the
// flat closed form plus the integral along the straight path of
// N0 exp(-z/H) (exp(-delta/H) - 1), by 8-point Gauss-Legendre quadrature (nodes
// sigma_j on [0, 1] from the emission point, weights w_j summing to 1).
// ---------------------------------------------------------------------------
// Quotient, square root and exponential for the small corrections (the
// sphere's curvature part of the optical path, the curved ray's turn and time
// saved): their FP32 forms need ~1e-6 relative accuracy, so they use the
// approximate hardware operations; the FP64 forms round as written.
template <typename T>
__device__ __forceinline__ T approx_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float approx_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename T>
__device__ __forceinline__ T approx_sqrt(T x) { return sqrt(x); }  // x > 0
template <>
__device__ __forceinline__ float approx_sqrt<float>(float x) { return x * rsqrtf(x); }
template <typename T>
__device__ __forceinline__ T approx_exp(T x) { return exp(x); }
template <>
__device__ __forceinline__ float approx_exp<float>(float x) { return __expf(x); }

constexpr int kSphNodes = 8;
__device__ __constant__ const double kSphSigma[kSphNodes] = {
    0.019855071751231856, 0.10166676129318664, 0.2372337950418355, 0.4082826787521751,
    0.5917173212478249,   0.7627662049581645,  0.8983332387068134, 0.9801449282487681};
__device__ __constant__ const double kSphWeight[kSphNodes] = {
    0.05061426814518813, 0.11119051722668724, 0.15685332293894363, 0.18134189168918100,
    0.18134189168918100, 0.15685332293894363, 0.11119051722668724, 0.05061426814518813};

template <typename T>
__device__ __forceinline__ T sphere_excess(T x, T y, T z, T R_E) {
  const T rho2 = x * x + y * y;
  const T zr = z + R_E;
  return approx_div(rho2, approx_sqrt(rho2 + zr * zr) + zr);
}
// exp(-x) - 1 for x >= 0 without cancellation
template <typename T>
__device__ __forceinline__ T exp_m1_neg(T x) {
  if (x < T(0.1)) return -x * (T(1) + x * (T(-0.5) + x * (T(1) / T(6) + x * (T(-1) / T(24) + x * (T(1) / T(120))))));
  return approx_exp(-x) - T(1);
}
// the curvature part of the optical path from x_e to the antenna a, d = a - x_e
template <typename T>
__device__ __forceinline__ T sphere_path_correction(T ax, T ay, T az, T dx, T dy, T dz, T R, T N0, T invH, T R_E) {
  T sum = T(0);
#pragma unroll
  for (int j = 0; j < kSphNodes; ++j) {
    const T f = T(1) - T(kSphSigma[j]);  // the node at x_e + sigma d = a - (1 - sigma) d
    const T x = ax - f * dx, y = ay - f * dy, z = az - f * dz;
    const T ex = sphere_excess(x, y, z, R_E);
    sum += T(kSphWeight[j]) * approx_exp(-z * invH) * exp_m1_neg(ex * invH);
  }
  return N0 * R * sum;
}

// ---------------------------------------------------------------------------
// curved rays in the flat exponential atmosphere (C8R_EXPONENTIAL_RAY).  The ray
// from x_e to the antenna keeps n(z) sin(theta) = p.  Written p = S m, with S =
// rho/R and C = |dz|/R the straight line's sine and cosine from the vertical and
// mu = m - 1 an effective refractivity, the ray's turn away from the straight
// line at height z is
//   sin(theta - theta_s) = S Q,  Q = (mu - nu)(2 + mu + nu) / (n^2 (C m/n + cos theta)),
// nu = n - 1, free of the cancellation of the direct difference.  The end-point
// condition, integral over z of (tan theta - tan theta_s) = 0, reads
// sum_j w_j k_j (mu - nu_j) = 0 with k_j = (2 + mu + nu_j)/(n_j^2 (C m/n_j +
// cos theta_j) cos theta_j) > 0 at the Gauss-Legendre nodes, so mu is the
// k-weighted mean of nu: a fixed point whose contraction factor is ~1e-4 (each
// iteration gains about four digits; from the plain mean, one iteration leaves
// < 1e-12 of mu for paths up to 40 km, three leave < 1e-18).  The optical path then differs from the
// straight line's by exactly
//   - integral over z of 2 n sin^2((theta - theta_s)/2)/C
//   = - R S^2 sum_j w_j n_j Q_j^2 / (1 + cos(theta_j - theta_s))
// (Fermat: from n sin(theta) = p and the shared end points), a small negative
// quantity formed directly, which is added to the straight path's closed form.
// Paths within 1e-3 of the horizontal, and vertical ones, keep the straight line.
// ---------------------------------------------------------------------------
template <typename T>
struct RayFix {
  T Q;    // sin(turn at x_e) = S Q
  T dop;  // ray's optical path minus the straight line's (m, <= 0)
};
template <typename T, int ITERS>
__device__ __forceinline__ RayFix<T> ray_fix(T rho2, T dz, T R, T nu_e, T invH) {
  RayFix<T> r{T(0), T(0)};
  const T adz = fabs(dz);
  if (!(rho2 > T(0)) || !(adz >= T(1e-3) * R)) return r;
  const T invR = approx_div(T(1), R);
  const T S = approx_sqrt(rho2) * invR, C = adz * invR;
  T nu[kSphNodes];
  T mu = T(0);
#pragma unroll
  for (int j = 0; j < kSphNodes; ++j) {
    nu[j] = nu_e * approx_exp(-T(kSphSigma[j]) * dz * invH);  // z = z_e + sigma dz
    mu += T(kSphWeight[j]) * nu[j];
  }
#pragma unroll
  for (int it = 0; it < ITERS; ++it) {
    const T m = T(1) + mu;
    T num = T(0), den = T(0);
#pragma unroll
    for (int j = 0; j < kSphNodes; ++j) {
      const T in = approx_div(T(1), T(1) + nu[j]);
      const T a = S * m * in;
      const T c2 = T(1) - a * a;
      if (!(c2 > T(0))) return RayFix<T>{T(0), T(0)};
      const T c = approx_sqrt(c2);
      const T k = approx_div((T(2) + mu + nu[j]) * in * in, (C * m * in + c) * c);
      num += T(kSphWeight[j]) * k * nu[j];
      den += T(kSphWeight[j]) * k;
    }
    mu = approx_div(num, den);
  }
  const T m = T(1) + mu;
  T sum = T(0);
#pragma unroll
  for (int j = 0; j < kSphNodes; ++j) {
    const T n = T(1) + nu[j];
    const T in = approx_div(T(1), n);
    const T a = S * m * in;
    const T c2 = T(1) - a * a;
    if (!(c2 > T(0))) return RayFix<T>{T(0), T(0)};
    const T Q = approx_div((mu - nu[j]) * (T(2) + mu + nu[j]) * in * in, C * m * in + approx_sqrt(c2));
    const T sd = S * Q;
    sum += T(kSphWeight[j]) * approx_div(n * Q * Q, T(1) + approx_sqrt(T(1) - sd * sd));
  }
  r.dop = -R * S * S * sum;
  const T in = approx_div(T(1), T(1) + nu_e);
  const T a = S * m * in;
  const T c2 = T(1) - a * a;
  if (!(c2 > T(0))) return RayFix<T>{T(0), T(0)};
  r.Q = approx_div((mu - nu_e) * (T(2) + mu + nu_e) * in * in, C * m * in + approx_sqrt(c2));
  return r;
}

// the turn of the direction d = x_a - x_e (length R) at x_e in the vertical plane,
// as the change of R rhat: sin(delta) R t + (cos(delta) - 1) d, with t the unit
// vector away from the vertical, R t = (|dz| d_h/rho, -sgn(dz) rho) and
// sin(delta) = (rho/R) Q
template <typename T>
__device__ __forceinline__ void ray_turn_vector(T dx, T dy, T dz, T R, T Q, T out[3]) {
  const T rho2 = dx * dx + dy * dy;
  const T invR = approx_div(T(1), R);
  const T sd = approx_sqrt(rho2) * invR * Q;
  const T cdm1 = approx_div(-sd * sd, T(1) + approx_sqrt(T(1) - sd * sd));
  const T f = cdm1 + Q * fabs(dz) * invR;
  out[0] = f * dx;
  out[1] = f * dy;
  out[2] = cdm1 * dz - (dz < T(0) ? T(-1) : T(1)) * Q * rho2 * invR;
}

// straight emission path x_e -> antenna (propagator, §2): distance, direction,
// source index and path-averaged index of the medium
__device__ __forceinline__ void geo_f64(const MedParams& M, const AntRec& A, double xe, double ye, double ze,
                                        double Ee, GeoD& g) {
  g.d[0] = A.x - xe;
  g.d[1] = A.y - ye;
  g.d[2] = A.z - ze;
  g.R = sqrt(g.d[0] * g.d[0] + g.d[1] * g.d[1] + g.d[2] * g.d[2]);
  double invR = 1.0 / g.R;
  g.rh[0] = g.d[0] * invR;
  g.rh[1] = g.d[1] * invR;
  g.rh[2] = g.d[2] * invR;
  if (M.kind == C8R_UNIFORM) {
    g.n_src = M.n;
    g.n_avg = M.n;
  } else {
    g.n_src = 1.0 + M.N0 * Ee;
    // path average of N0 exp(-z/H) between z_e and z_a: N0 H (E_e - E_a) / dz,
    // or its series in x = dz/H when the two altitudes nearly coincide
    double dz = g.d[2];
    double x = dz * M.invH;
    double ratio;
    if (fabs(x) > 1e-3)
      ratio = (Ee - A.Ea) / x;
    else
      ratio = Ee * (1.0 + x * (-0.5 + x * (1.0 / 6.0 + x * (-1.0 / 24.0 + x * (1.0 / 120.0)))));
    g.n_avg = 1.0 + M.N0 * ratio;
    if (M.kind == C8R_EXPONENTIAL_SPHERICAL) {
      g.n_src = 1.0 + M.N0 * Ee * exp(-sphere_excess(xe, ye, ze, M.R_E) * M.invH);
      g.n_avg += sphere_path_correction<double>(A.x, A.y, A.z, g.d[0], g.d[1], g.d[2], g.R, M.N0, M.invH, M.R_E) /
                 g.R;
    } else if (M.kind == C8R_EXPONENTIAL_RAY) {
      // the refracted ray: its direction at x_e and its optical path
      const RayFix<double> r =
          ray_fix<double, 3>(g.d[0] * g.d[0] + g.d[1] * g.d[1], g.d[2], g.R, M.N0 * Ee, M.invH);
      double t[3];
      ray_turn_vector<double>(g.d[0], g.d[1], g.d[2], g.R, r.Q, t);
      for (int c = 0; c < 3; ++c) g.rh[c] = (g.d[c] + t[c]) * invR;
      g.n_avg += r.dop * invR;
    }
  }
}

// arrival position in bins relative to the antenna's first bin edge
__device__ __forceinline__ double arrival_f64(const MedParams& M, const GeoD& g, double t_e, double t_ref) {
  return ((t_e - t_ref) + g.n_avg * g.R * M.inv_c_ns) / M.dt_ns;
}

// ---------------------------------------------------------------------------
// mixed path: FP32 field arithmetic; arrival time in float-float
// ---------------------------------------------------------------------------
struct GeoM {
  float s[3], e[3];  // d = x_a - x_e as float-float per component
  float R0, R1;      // |d| as float-float (R1 = 0 until geo_refine)
  float y;           // ~1/R0 (rsqrt estimate)
};

// d = a - p (p given as float-float; p_l = 0 for the FP32-exact endpoints) and
// an FP32 estimate of R = |d| (enough for the Doppler factor and amplitudes)
__device__ __forceinline__ void geo_lite(const AntRec& A, float pxh, float pyh, float pzh, float pxl, float pyl,
                                         float pzl, GeoM& g) {
  two_sum(A.xh, -pxh, g.s[0], g.e[0]);
  two_sum(A.yh, -pyh, g.s[1], g.e[1]);
  two_sum(A.zh, -pzh, g.s[2], g.e[2]);
  g.e[0] = __fadd_rn(g.e[0], __fsub_rn(A.xl, pxl));
  g.e[1] = __fadd_rn(g.e[1], __fsub_rn(A.yl, pyl));
  g.e[2] = __fadd_rn(g.e[2], __fsub_rn(A.zl, pzl));
  const float S = __fmaf_rn(g.s[2], g.s[2], __fmaf_rn(g.s[0], g.s[0], __fmul_rn(g.s[1], g.s[1])));
  g.y = rsqrtf(S);
  g.R0 = __fmul_rn(S, g.y);
  g.R1 = 0.0f;
}

// R = |d| in float-float: the three exact squares are summed with TwoSum, then
// one Newton step corrects the FP32 estimate R0 (its square is formed exactly)
// the same for an FP32-exact point (no low part)
__device__ __forceinline__ void geo_lite(const AntRec& A, float px, float py, float pz, GeoM& g) {
  two_sum(A.xh, -px, g.s[0], g.e[0]);
  two_sum(A.yh, -py, g.s[1], g.e[1]);
  two_sum(A.zh, -pz, g.s[2], g.e[2]);
  g.e[0] = __fadd_rn(g.e[0], A.xl);
  g.e[1] = __fadd_rn(g.e[1], A.yl);
  g.e[2] = __fadd_rn(g.e[2], A.zl);
  const float S = __fmaf_rn(g.s[2], g.s[2], __fmaf_rn(g.s[0], g.s[0], __fmul_rn(g.s[1], g.s[1])));
  g.y = rsqrtf(S);
  g.R0 = __fmul_rn(S, g.y);
  g.R1 = 0.0f;
}

// the z part of d = a - p that every antenna of a flat array (one altitude)
// shares: d_z as float-float and the products of it that geo_refine and
// doppler_ff form, formed once per point as they form them (so the same values)
struct ZPart {
  float sh, sl;  // d_z = sh + sl (geo_lite's s[2], e[2])
  float qh, ql;  // sh^2, exact
  float se;      // fl(sh sl)
  float bh, bl;  // b_z sh, exact
  float be;      // fl(b_z sl)
};
__device__ __forceinline__ ZPart z_part(float sh, float sl, float bz) {
  ZPart z;
  z.sh = sh;
  z.sl = sl;
  two_prod(sh, sh, z.qh, z.ql);
  z.se = __fmul_rn(sh, sl);
  two_prod(bz, sh, z.bh, z.bl);
  z.be = __fmul_rn(bz, sl);
  return z;
}

// geo_lite of a float-float point whose z part comes from ZPart
__device__ __forceinline__ void geo_lite(const AntRec& A, float pxh, float pyh, float pxl, float pyl, const ZPart& z,
                                         GeoM& g) {
  two_sum(A.xh, -pxh, g.s[0], g.e[0]);
  two_sum(A.yh, -pyh, g.s[1], g.e[1]);
  g.s[2] = z.sh;
  g.e[2] = z.sl;
  g.e[0] = __fadd_rn(g.e[0], __fsub_rn(A.xl, pxl));
  g.e[1] = __fadd_rn(g.e[1], __fsub_rn(A.yl, pyl));
  const float S = __fmaf_rn(g.s[2], g.s[2], __fmaf_rn(g.s[0], g.s[0], __fmul_rn(g.s[1], g.s[1])));
  g.y = rsqrtf(S);
  g.R0 = __fmul_rn(S, g.y);
  g.R1 = 0.0f;
}

// R from the exact squares of d's components (p2 + q2 = s_z^2 and se =
// fl(s_z e_z) given)
__device__ __forceinline__ void geo_refine(GeoM& g, float p2, float q2, float se) {
  float p0, q0, p1, q1;
  two_prod(g.s[0], g.s[0], p0, q0);
  two_prod(g.s[1], g.s[1], p1, q1);
  float S1, E1, S2, E2;
  two_sum(p0, p1, S1, E1);
  two_sum(S1, p2, S2, E2);
  const float cross = __fmaf_rn(g.s[0], g.e[0], __fmaf_rn(g.s[1], g.e[1], se));
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, E1)), __fadd_rn(E2, __fmul_rn(2.0f, cross)));
  float rq, rqe;
  two_prod(g.R0, g.R0, rq, rqe);
  const float rho = __fadd_rn(__fsub_rn(__fsub_rn(S2, rq), rqe), lo);
  g.R1 = __fmul_rn(__fmul_rn(rho, 0.5f), g.y);
}
__device__ __forceinline__ void geo_refine(GeoM& g) {
  float p2, q2;
  two_prod(g.s[2], g.s[2], p2, q2);
  geo_refine(g, p2, q2, __fmul_rn(g.s[2], g.e[2]));
}
__device__ __forceinline__ void geo_refine(GeoM& g, const ZPart& z) { geo_refine(g, z.qh, z.ql, z.se); }

__device__ __forceinline__ void geo_mixed(const AntRec& A, float pxh, float pyh, float pzh, float pxl, float pyl,
                                          float pzl, GeoM& g) {
  geo_lite(A, pxh, pyh, pzh, pxl, pyl, pzl, g);
  geo_refine(g);
}

// (E_e - E_a)/dz in float-float, the quotient of the refractivity term of the
// exponential medium, dz = dzh + dzl the altitude difference a - e: the FP32
// quotient corrected once from the exact residual, or for |dz/H| <= 1e-3 the
// series (E_e/H)(1 + f), f = -x/2 + x^2/6 - x^3/24, x = dz/H
__device__ __forceinline__ void refr_quotient(const MedParams& M, float Eah, float Eal, float dzh, float dzl,
                                              float Eeh, float Eel, float& q0, float& q1) {
  const float x = __fmul_rn(dzh, M.invH_h);
  if (fabsf(x) > 1e-3f) {
    float Qh, Ql;
    two_sum(Eeh, -Eah, Qh, Ql);
    Ql = __fadd_rn(Ql, __fsub_rn(Eel, Eal));
    q0 = __fdividef(Qh, dzh);
    float ph, pl;
    two_prod(q0, dzh, ph, pl);
    const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(Qh, ph), pl), Ql), __fmul_rn(q0, dzl));
    q1 = __fdividef(r, dzh);
  } else {
    const float f = __fmul_rn(x, __fmaf_rn(x, __fmaf_rn(x, -1.0f / 24.0f, 1.0f / 6.0f), -0.5f));
    float eh, el;
    two_prod(Eeh, M.invH_h, eh, el);
    el = __fmaf_rn(Eeh, M.invH_l, __fmaf_rn(Eel, M.invH_h, el));
    // (eh + el)(1 + f)
    float g0, g1;
    two_sum(eh, __fmul_rn(eh, f), g0, g1);
    q0 = g0;
    q1 = __fadd_rn(g1, __fmaf_rn(el, f, el));
  }
}

// arrival position u = (t_e - t_ref)/dt + n_avg R / (c dt) in bins, float-float,
// with the refractivity quotient (q0, q1) given (exponential media; ignored in
// the uniform one).  tau_e = t_e/dt and the antenna's tau = t_ref/dt come in
// float-float.  KIND: the medium kind (a template argument, so each kernel
// carries only its own medium's arithmetic; it equals M.kind).  `dop` (curved
// rays only): the ray's optical path minus the straight line's, m
template <int KIND>
__device__ __forceinline__ ff arrival_mixed_q(const MedParams& M, const AntRec& A, const GeoM& g, float tauh,
                                              float taul, float q0, float q1, float dop = 0.0f) {
  float ts, te;
  two_sum(tauh, -A.tauh, ts, te);
  te = __fadd_rn(te, __fsub_rn(taul, A.taul));
  float sh = (KIND == C8R_UNIFORM) ? M.s_h : M.kc_h;
  float sl = (KIND == C8R_UNIFORM) ? M.s_l : M.kc_l;
  float p, pe;
  two_prod(g.R0, sh, p, pe);
  pe = __fmaf_rn(g.R0, sl, __fmaf_rn(g.R1, sh, pe));
  if constexpr (KIND != C8R_UNIFORM) {
    // refractivity term (n_avg - 1) R/(c dt) = N0 H/(c dt) * (E_e - E_a)/dz * R
    float w, we;
    two_prod(q0, g.R0, w, we);
    we = __fmaf_rn(q0, g.R1, __fmaf_rn(q1, g.R0, we));
    float v, ve;
    two_prod(w, M.cN_h, v, ve);
    ve = __fmaf_rn(w, M.cN_l, __fmaf_rn(we, M.cN_h, ve));
    float p2, pe2;
    fast_two_sum(p, v, p2, pe2);  // |v| = (n_avg - 1)|p| < |p|
    p = p2;
    pe = __fadd_rn(pe, __fadd_rn(pe2, ve));
    if constexpr (KIND == C8R_EXPONENTIAL_SPHERICAL) {
      // curvature correction (~1e-3 of the refractivity term, FP32 is enough)
      const float cs = __fmul_rn(
          sphere_path_correction<float>(A.xh, A.yh, A.zh, g.s[0], g.s[1], g.s[2], g.R0, M.N0f, M.invH_h, M.RE_f),
          M.kc_h);
      fast_two_sum(p, cs, p2, pe2);
      p = p2;
      pe = __fadd_rn(pe, pe2);
    }
    if constexpr (KIND == C8R_EXPONENTIAL_RAY) {
      // the ray's time saved against the straight line (<~1 bin; FP32 is enough)
      fast_two_sum(p, __fmul_rn(dop, M.kc_h), p2, pe2);
      p = p2;
      pe = __fadd_rn(pe, pe2);
    }
  }
  float uh, ue;
  two_sum(ts, p, uh, ue);
  ue = __fadd_rn(ue, __fadd_rn(te, pe));
  return ff{uh, ue};
}

// the same with the quotient formed here, from the emission point's E_e =
// exp(-z_e/H) and the altitude difference of g
template <int KIND>
__device__ __forceinline__ ff arrival_mixed(const MedParams& M, const AntRec& A, const GeoM& g, float tauh, float taul,
                                            float Eeh, float Eel, float dop = 0.0f) {
  float q0 = 0.0f, q1 = 0.0f;
  if constexpr (KIND != C8R_UNIFORM) refr_quotient(M, A.Eah, A.Eal, g.s[2], g.e[2], Eeh, Eel, q0, q1);
  return arrival_mixed_q<KIND>(M, A, g, tauh, taul, q0, q1, dop);
}

// bin index of a float-float arrival, clamped to [-1, n_bins]: -1 stands for
// "before the window" (or not a number), n_bins for "after it"; frac is the
// position inside the bin (meaningful only for an index inside the window)
__device__ __forceinline__ int bin_raw(ff u, int n_bins, float& frac) {
  frac = 0.0f;
  if (!(u.h > -1.0f)) return -1;
  // quick reject of arrivals well after the window (and of +inf).  The low part
  // is not renormalised: near 2^24 bins, where FP32 is spaced by 1 or 2, it can
  // reach a few units (u = 2^24 - 0.35, in the last bin of the largest window,
  // can come as u.h = 2^24 + 2, u.l = -2.35), so the bound leaves room for a low
  // part of up to 64 in magnitude (an arrival of ~1e9 bins)
  if (!(u.h < (float)n_bins + 64.0f)) return n_bins;
  float kf = floorf(u.h);
  float f = __fadd_rn(__fsub_rn(u.h, kf), u.l);
  // bring the fraction into [0, 1) by its own floor: the low part is not
  // renormalised, and for an arrival near 2^24 bins (FP32 spacing 1 or 2 there)
  // it can exceed 1 in magnitude, so a single step of +-1 would not do
  const float df = floorf(f);
  kf = __fadd_rn(kf, df);
  f = __fsub_rn(f, df);
  int k = (int)kf;
  frac = f;
  if (k < 0) return -1;
  if (k >= n_bins) return n_bins;
  return k;
}
// ---------------------------------------------------------------------------
// Bin of an arrival from plain FP32 arithmetic with a bound on its error, for
// the one-bin deposit (reading T: only the bin of an arrival matters there).
// The float-float arrival (arrival_mixed, ~1e-9 bin) costs about four times the
// FP32 one.  The FP32 arrival decides the bin whenever no bin edge (and neither
// end of the window) lies within its error bound; then it is the bin of the
// float-float arrival too, which is good to ~1e-7 bin at most, far inside the
// bound's 1e-6-bin floor.  Otherwise the caller evaluates the float-float
// arrival.
//
// Vertical split.  With w = z_e - z_a (the emission point's height above the
// antenna) and rho^2 = d_x^2 + d_y^2, the distance is R = w + x, where
// x = R - w = rho^2 / (R + w) since R^2 = w^2 + rho^2.  So
//   u = (tau_e - tau_a) + k R + v = (T_e - T_a) + k x + v,
//   T_e = tau_e + k z_e (per track endpoint), T_a = tau_a + k z_a (per antenna),
// with k = n/(c dt) in the uniform medium and 1/(c dt) in the exponential one
// (where v carries the refractivity).  T_e and T_a are formed once, in
// float-float, so no per-pair FP32 rounding acts on a term as large as k R
// (~1e5 bins): FP32 rounds T_e - T_a, about the arrival's own distance from
// the window start, and k x, which is small for emission points high above the
// antenna (x ~ R theta^2 / 2 at an angle theta off the vertical).  The split
// form x = rho^2 / (R + w) pays where x is small against R; elsewhere (an
// inclined line of sight, or a point below the antenna, w <= 0) the direct form
// x = R - w = fl(R + s_z) has the smaller error, and the caller picks the form
// (SPLIT below) for a whole warp: the split one when every lane's emission
// point lies within 45 degrees of the antenna's vertical (2 rho^2 < S, w > 0).
//
// The errors, with u = 2^-24 (the FP32 unit roundoff) and every step rounded
// once (intrinsics, no contraction):
//   s = fl(a_h - p): each component is off the exact d = a - p by at most
//     u |s_i| and the antenna's low part a_l.  x changes with s_z at the rate
//     x/R and with s_x, s_y at |s_{x,y}|/R, so the rounding moves x by at most
//     u (x + rho^2 / R) <= 3u x (also for w <= 0, where x >= R); a_l moves it by
//     at most 2 |a_l| (T_a holds the exact z_a);
//   rho^2 = fl(s_x^2 + s_y^2) (two roundings, 2u) and S = fl(s_z^2 + rho^2):
//     R' = S rsqrt(S) plus one Newton step with the residual fma(-R0, R0, S) is
//     sqrt(S) rounded once, within 2.5u R of |s|;
//   split form, w > 0: x = rho^2 / fl(R0 - s_z) with __fdividef (2 ulp: 4u),
//     from the unrefined R0 = fl(S rsqrtf(S)) (rsqrtf 2 ulp: R0 within 6u R of
//     |s|, so the denominator R + |s_z| >= R carries 7u); with rho^2, 13u x.
//     (w <= 0: x = fl(R0 + s_z) >= R, 7u x.)  Direct form: x = fl(R' + s_z),
//     2.5u R + u x;
//   q = fl(x k_h): u, and u more for the dropped k_l;
//   Td = fl(fl(T_e,h - T_a,h) + fl(T_e,l - T_a,l)): 2u |Td|, plus terms of
//     u^2 |T_e| and u^2 |T_a| from the float-float forms of T_e and T_a;
//   v (exponential medium) = N0 H/(c dt) (E_e - E_a)/dz R' (R0 in the split
//     form): the quotient (2 ulp) or its series for |dz/H| <= 1e-3, four more
//     roundings and R' give at most 14u |v| (17.5u with R0), plus
//     |v| |z_l|/|dz| from the antenna altitude's low part, |dz| > 1e-3 H in
//     the quotient's branch;
//   uf = fl(fl(Td + q) + v): u |Td + q| <= u (|uf| + |v|) (Td + q is uf - v
//     before the last rounding, small against Td and q once the arrival is
//     near the window) and u |uf|, and one more u |uf| in the window test
//     uf - bound >= n_bins.
// The bound used is u (2.25 |Td| + c_q q + c_v |v| + 3.25 |uf|) + fb_rel_v |v| +
// fb_abs, with c_q = 19 and c_v = 22 in the split form (18 and 17.5 derived)
// and c_q = 6.25, c_v = 17 plus 2.5u k_h R in the direct one (6, 14 and 2.5),
// each coefficient above its derivation; fb_abs holds 2 k |a_l|,
// 16 u^2 |T_a| (the share of T_e, |T_e| <= |Td| + |T_a|, beyond what the |Td|
// term covers) and a floor of 1e-6 bin for the float-float arrival's own error
// and the rounding of uf - floor(uf).  A CPU emulation of these steps (2-ulp
// reciprocal square root and quotient) against the FP64 oracle's arrivals
// stays below 0.6 of the bound on the benchmark showers; on a vertical shower
// 1-10 km above 0.2-ns traces the bound is ~6e-4 bin and ~0.1 % of the
// endpoints are left to the float-float arrival (8 % with k R rounded in FP32
// per pair).  On a shower inclined by 60 degrees x is about R/2 and the direct
// form holds the bound near that of an arrival rounded in FP32 throughout.
// ---------------------------------------------------------------------------
constexpr int kFastOut = -1;        // the arrival lies outside the window: no deposit
constexpr int kFastUndecided = -2;  // an edge lies within the bound: the float-float arrival decides

// d = a_h - p in FP32 (no low parts), rho^2 = d_x^2 + d_y^2, S = |d|^2 and
// R0 = |d| as geo_lite forms them (the same s, y and R0 bit for bit)
__device__ __forceinline__ void geo_fast(const AntRec& A, float px, float py, float pz, GeoM& g, float& S,
                                         float& rho2) {
  g.s[0] = __fadd_rn(A.xh, -px);
  g.s[1] = __fadd_rn(A.yh, -py);
  g.s[2] = __fadd_rn(A.zh, -pz);
  rho2 = __fmaf_rn(g.s[0], g.s[0], __fmul_rn(g.s[1], g.s[1]));
  S = __fmaf_rn(g.s[2], g.s[2], rho2);
  g.y = rsqrtf(S);
  g.R0 = __fmul_rn(S, g.y);
  g.R1 = 0.0f;
}

// T = tau + k z as float-float, the shifted time of arrival_fast, for a height
// z = zh + zl (zl = 0 for an FP32-exact endpoint)
__device__ __forceinline__ void shifted_time(float tauh, float taul, float zh, float zl, float kh, float kl,
                                             float& Th, float& Tl) {
  float p, e;
  two_prod(zh, kh, p, e);
  e = __fmaf_rn(zh, kl, __fmaf_rn(zl, kh, e));
  float s, e2;
  two_sum(tauh, p, s, e2);
  e2 = __fadd_rn(e2, __fadd_rn(taul, e));
  fast_two_sum(s, e2, Th, Tl);
}

// whether the split form of x pays for the emission point of g: within 45
// degrees of the antenna's vertical and above it
__device__ __forceinline__ bool split_pays(const GeoM& g, float S, float rho2) {
  return g.s[2] < 0.0f && __fadd_rn(rho2, rho2) < S;
}

// the FP32 quotient (E_e - E_a)/dz of the refractivity term for the FP32
// arrival (exponential medium): dz = s_z, the FP32 a_h - p of the emission
// point (the same for every antenna of a flat array); for |dz/H| <= 1e-3 its
// series (E_e/H)(1 + f)
__device__ __forceinline__ float fast_quotient(const MedParams& M, float Eah, float Eal, float sz, float Eeh,
                                               float Eel) {
  const float x = __fmul_rn(sz, M.invH_h);
  if (fabsf(x) > 1e-3f) return __fdividef(__fadd_rn(__fsub_rn(Eeh, Eah), __fsub_rn(Eel, Eal)), sz);
  const float f = __fmul_rn(x, __fmaf_rn(x, __fmaf_rn(x, -1.0f / 24.0f, 1.0f / 6.0f), -0.5f));
  return __fmul_rn(__fmul_rn(Eeh, M.invH_h), __fadd_rn(1.0f, f));
}

// The FP32 arrival uf of the emission point of g (S = |d|^2, rho2 = d_x^2 +
// d_y^2, T_e = Teh + Tel, qv the refractivity quotient of fast_quotient) and
// its error bound, returned; SPLIT picks the form of x; q_extra adds a term
// u * q_extra * k x for geometry whose d carries more than the one rounding of
// a_h - p (the midpoint)
template <int KIND, bool SPLIT>
__device__ __forceinline__ float arrival_fast(const MedParams& M, const AntRec& A, const GeoM& g, float S, float rho2,
                                              float Teh, float Tel, float qv, float q_extra, float& uf_out) {
  static_assert(KIND == C8R_UNIFORM || KIND == C8R_EXPONENTIAL, "plain straight-line media only");
  constexpr float u = 5.9604644775390625e-8f;  // 2^-24
  // R' = sqrt(S) rounded once (the direct form), or the unrefined R0 (the
  // split form, whose x is small: R enters it only through its denominator)
  float R;
  if constexpr (SPLIT) {
    R = g.R0;
  } else {
    const float r = __fmaf_rn(-g.R0, g.R0, S);
    R = __fmaf_rn(r, __fmul_rn(0.5f, g.y), g.R0);
  }
  // x = R - w, w = z_e - z_a = -s_z
  const float sz = g.s[2];
  float x;
  if constexpr (SPLIT) {
    x = sz < 0.0f ? __fdividef(rho2, __fsub_rn(R, sz)) : __fadd_rn(R, sz);
  } else {
    x = __fadd_rn(R, sz);
  }
  const float kh = KIND == C8R_UNIFORM ? M.s_h : M.kc_h;
  const float q = __fmul_rn(x, kh);
  const float Td = __fadd_rn(__fsub_rn(Teh, A.Tah), __fsub_rn(Tel, A.Tal));
  float v = 0.0f;
  if constexpr (KIND == C8R_EXPONENTIAL) v = __fmul_rn(__fmul_rn(qv, R), M.cN_h);
  const float uf = __fadd_rn(__fadd_rn(Td, q), v);
  uf_out = uf;
  const float tail = __fmaf_rn(2.25f * u, fabsf(Td),
                               __fmaf_rn(__fmaf_rn(SPLIT ? 22.0f : 17.0f, u, A.fb_rel_v), fabsf(v),
                                         __fmaf_rn(3.25f * u, fabsf(uf), A.fb_abs)));
  if constexpr (SPLIT) {
    return __fmaf_rn(__fmaf_rn(q_extra, u, 19.0f * u), q, tail);
  } else {
    return __fmaf_rn(__fmaf_rn(q_extra, u, 6.25f * u), q, __fmaf_rn(__fmul_rn(2.5f * u, kh), R, tail));
  }
}

template <int KIND, bool SPLIT>
__device__ __forceinline__ int arrival_bin_fast(const MedParams& M, const AntRec& A, const GeoM& g, float S,
                                                float rho2, float Teh, float Tel, float qv) {
  float uf;
  const float eps = arrival_fast<KIND, SPLIT>(M, A, g, S, rho2, Teh, Tel, qv, 0.0f, uf);
  if (uf < -eps || __fsub_rn(uf, eps) >= (float)M.n_bins) return kFastOut;
  const float k = floorf(uf);
  const float fr = __fsub_rn(uf, k);
  if (!(fr > eps && fr < __fsub_rn(1.0f, eps))) return kFastUndecided;  // also NaN
  return (int)k;
}

// distance k + 1 - u from a float-float arrival u in bin k to the bin's upper
// edge, formed from the arrival rather than as 1 - frac: just below an edge the
// fraction is close to 1, where FP32 is spaced by 6e-8, while the distance is
// small and keeps its relative precision ((k + 1) - u_h is exact there).  The
// first bin of a narrow ZHS interval straddling an edge takes this share.
__device__ __forceinline__ float gap_to_next_edge(ff u, int k) {
  return __fsub_rn(__fsub_rn((float)(k + 1), u.h), u.l);
}

__device__ __forceinline__ bool bin_of(ff u, int n_bins, int& k, float& frac) {
  k = bin_raw(u, n_bins, frac);
  return k >= 0 && k < n_bins;
}

// field part at one emission point (FP32): w = d x beta, V = (d x w)/R^2 =
// rhat x (rhat x beta), D = 1 - n beta.rhat in a cancellation-free form:
//   D = (1 - n|beta|) + n |w|^2 / (R (|beta| R + beta.d))   when beta.d >= 0
// (the second term is n|beta|(1 - cos theta)); the direct form otherwise.
struct FieldM {
  float V[3];  // rhat x (rhat x beta) times R^2  (i.e. d x w)
  float D;
  float invR;
  float bd;    // beta . d
  float w[3];  // d x beta
};
// Every step uses explicit-rounding intrinsics so the forward and the adjoint
// kernels, which inline this in different contexts, take identical branch
// decisions.
__device__ __forceinline__ void field_mixed(const GeoM& g, float bx, float by, float bz, float bmag, float om_nb,
                                            float n, FieldM& f) {
  const float sx = g.s[0], sy = g.s[1], sz = g.s[2];
  // w = d x beta from the FP32 part of d (the low parts, ~2^-24 |d|, change D by
  // ~1e-7 relative even near the Cherenkov angle, below the FP32 field arithmetic)
  const float wx = __fmaf_rn(sy, bz, -__fmul_rn(sz, by));
  const float wy = __fmaf_rn(sz, bx, -__fmul_rn(sx, bz));
  const float wz = __fmaf_rn(sx, by, -__fmul_rn(sy, bx));
  const float bd = __fmaf_rn(bx, sx, __fmaf_rn(by, sy, __fmul_rn(bz, sz)));
  const float R = g.R0;
  const float invR = g.y;
  if (bd >= 0.0f) {
    const float w2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
    const float den = __fmul_rn(R, __fmaf_rn(bmag, R, bd));
    f.D = __fadd_rn(om_nb, __fdividef(__fmul_rn(n, w2), den));
  } else {
    f.D = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(n, bd), invR));
  }
  // d x w = d (d.beta) - beta R^2  ->  V R^2
  f.V[0] = __fmaf_rn(sy, wz, -__fmul_rn(sz, wy));
  f.V[1] = __fmaf_rn(sz, wx, -__fmul_rn(sx, wz));
  f.V[2] = __fmaf_rn(sx, wy, -__fmul_rn(sy, wx));
  f.invR = invR;
  f.bd = bd;
  f.w[0] = wx;
  f.w[1] = wy;
  f.w[2] = wz;
}

// D = 1 - n (beta . d)/R in float-float, for a refined geometry (R = R0 + R1)
// and n - 1 given directly.  Its absolute error (~1e-10, set by n - 1 in FP32)
// is what the arrival interval ends u_m -/+ |D| (t1 - t0)/(2 dt) need: the
// half-width reaches ~10^2 bins, so D must be good to ~1e-9 absolute, which the
// FP32 form of field_mixed (good to ~1e-7 relative) is not for |D| of order 1.
// (p2 + q2 = b_z s_z exactly and bze = fl(b_z e_z) given)
__device__ __forceinline__ ff doppler_ff(const GeoM& g, float bx, float by, float p2, float q2, float bze,
                                         float nm1) {
  // beta . d with d = s + e exact: exact products of the high parts, summed
  // with TwoSum; the low parts and the rounding errors in FP32
  float p0, q0, p1, q1;
  two_prod(bx, g.s[0], p0, q0);
  two_prod(by, g.s[1], p1, q1);
  float S1, E1, S2, E2;
  two_sum(p0, p1, S1, E1);
  two_sum(S1, p2, S2, E2);
  const float be = __fmaf_rn(bx, g.e[0], __fmaf_rn(by, g.e[1], bze));
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, E1)), __fadd_rn(E2, be));
  // q = (beta . d)/R: FP32 quotient, then one correction from the exact residual
  const float qh = __fmul_rn(S2, g.y);
  float ph, pl;
  two_prod(qh, g.R0, ph, pl);
  const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(S2, ph), pl), lo), __fmul_rn(qh, g.R1));
  const float ql = __fmul_rn(r, g.y);
  // n q = q + (n - 1) q, then D = 1 - n q
  float nh, nl;
  two_sum(qh, __fmul_rn(nm1, qh), nh, nl);
  nl = __fadd_rn(nl, ql);
  float dh, dl;
  two_sum(1.0f, -nh, dh, dl);
  dl = __fsub_rn(dl, nl);
  // renormalise, so that the sign of D is the sign of D.h (near D = 0 the high
  // part alone can be 0 or of the other sign)
  ff D;
  D.h = __fadd_rn(dh, dl);
  D.l = __fsub_rn(dl, __fsub_rn(D.h, dh));
  return D;
}
__device__ __forceinline__ ff doppler_ff(const GeoM& g, float bx, float by, float bz, float nm1) {
  float p2, q2;
  two_prod(bz, g.s[2], p2, q2);
  return doppler_ff(g, bx, by, p2, q2, __fmul_rn(bz, g.e[2]), nm1);
}
__device__ __forceinline__ ff doppler_ff(const GeoM& g, float bx, float by, const ZPart& z, float nm1) {
  return doppler_ff(g, bx, by, z.bh, z.bl, z.be, nm1);
}

// the same field quantities at the midpoint of a track, from those of its two
// endpoints: d_m = (d0 + d1)/2 exactly (float-float), and w = d x beta and
// beta.d are linear in d, so w_m = (w0 + w1)/2, (beta.d)_m = (bd0 + bd1)/2
__device__ __forceinline__ void midpoint_from_endpoints(const GeoM& g0, const GeoM& g1, const FieldM& f0,
                                                        const FieldM& f1, float bmag, float om_nb, float n, GeoM& gm,
                                                        FieldM& fmid) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float S, E;
    two_sum(g0.s[c], g1.s[c], S, E);
    gm.s[c] = 0.5f * S;
    gm.e[c] = 0.5f * __fadd_rn(E, __fadd_rn(g0.e[c], g1.e[c]));
    fmid.w[c] = 0.5f * __fadd_rn(f0.w[c], f1.w[c]);
  }
  const float S2 = __fmaf_rn(gm.s[0], gm.s[0], __fmaf_rn(gm.s[1], gm.s[1], __fmul_rn(gm.s[2], gm.s[2])));
  gm.y = rsqrtf(S2);
  gm.R0 = __fmul_rn(S2, gm.y);
  gm.R1 = 0.0f;
  const float bd = 0.5f * __fadd_rn(f0.bd, f1.bd);
  const float wx = fmid.w[0], wy = fmid.w[1], wz = fmid.w[2];
  const float sx = gm.s[0], sy = gm.s[1], sz = gm.s[2];
  if (bd >= 0.0f) {
    const float w2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
    const float den = __fmul_rn(gm.R0, __fmaf_rn(bmag, gm.R0, bd));
    fmid.D = __fadd_rn(om_nb, __fdividef(__fmul_rn(n, w2), den));
  } else {
    fmid.D = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(n, bd), gm.y));
  }
  fmid.V[0] = __fmaf_rn(sy, wz, -__fmul_rn(sz, wy));
  fmid.V[1] = __fmaf_rn(sz, wx, -__fmul_rn(sx, wz));
  fmid.V[2] = __fmaf_rn(sx, wy, -__fmul_rn(sy, wx));
  fmid.invR = gm.y;
  fmid.bd = bd;
}

}  // namespace c8r
