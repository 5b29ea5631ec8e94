// generate.cu -- synthetic shower tracks generated on the device, so that a
// large shower can be streamed through the radio step chunk by chunk without a
// host-to-device copy of its tracks (the paper's full-shower workload, §5, is a
// stream of tracks from the simulation).  Counter-based: track g of shower
// `seed` is drawn from its own Philox4x32-10 blocks (Salmon, Moraes, Dror & Shaw,
// SC'11), so any range of tracks can be generated on its own.  The
// distributions are those of the synthetic shower the tests and the benchmark
// use; every FP64 operation rounds as written (this unit is compiled without
// FMA contraction) in the order of the host twin of this generator.
#include <cmath>
#include <cstdint>

#include "c8r_internal.h"

namespace c8r {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kPhiloxTag = 0x63387237u;  // fourth counter word of every block
constexpr int kHeightAttempts = 16;
constexpr double kLn10 = 2.302585092994046;         // ln 10
constexpr double kLnRange = 6.907755278982138;      // ln 1e4 - ln 10
constexpr double kTwoPi = 6.283185307179586;
constexpr double kSigmaAngle = 0.08726646259971647;  // 5 degrees in rad
constexpr double kCmPerNs = 0.29979245800000004;     // m/ns
constexpr double kInv2p32 = 2.3283064365386963e-10;  // 2^-32

struct U4 {
  uint32_t w[4];
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return U4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ double u01(uint32_t w) { return ((double)w + 0.5) * kInv2p32; }

struct GenArgs {
  uint64_t seed;
  int64_t first, n;
  double cz, sz;  // cos and sin of the zenith angle (rotation about y)
  float *x0, *y0, *z0, *x1, *y1, *z1, *t0, *t1, *bx, *by, *bz, *q;
};

__global__ void __launch_bounds__(256) k_generate(const GenArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const uint64_t g = (uint64_t)(a.first + i);
  const uint32_t lo = (uint32_t)g, hi = (uint32_t)(g >> 32);
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  U4 w = philox(lo, hi, 0u, kPhiloxTag, k0, k1);
  const double r = -30.0 * log(u01(w.w[0]));
  const double phi = kTwoPi * u01(w.w[1]);
  const double L = 0.5 + 4.5 * u01(w.w[2]);
  const double gamma = exp(kLn10 + kLnRange * u01(w.w[3]));
  w = philox(lo, hi, 1u, kPhiloxTag, k0, k1);
  const float q = u01(w.w[0]) < 0.55 ? -1.0f : 1.0f;
  const double rad = sqrt(-2.0 * log(u01(w.w[1])));
  const double ang = kTwoPi * u01(w.w[2]);
  const double ax = kSigmaAngle * (rad * cos(ang));
  const double ay = kSigmaAngle * (rad * sin(ang));
  double h = 4000.0;
  for (int j = 0; j < kHeightAttempts; ++j) {
    w = philox(lo, hi, 2u + (uint32_t)j, kPhiloxTag, k0, k1);
    const double z = sqrt(-2.0 * log(u01(w.w[0]))) * cos(kTwoPi * u01(w.w[1]));
    const double hj = 4000.0 + 1500.0 * z;
    if (hj >= 500.0 && hj <= 10000.0) {
      h = hj;
      break;
    }
  }
  double ux = -(cos(ax) * sin(ay)), uy = sin(ax), uz = -(cos(ax) * cos(ay));
  const double un = sqrt((ux * ux + uy * uy) + uz * uz);
  ux = ux / un;
  uy = uy / un;
  uz = uz / un;
  double x = r * cos(phi), y = r * sin(phi), zz = h;
  if (a.sz != 0.0) {
    const double xr = a.cz * x + a.sz * zz, zr = a.cz * zz - a.sz * x;
    const double uxr = a.cz * ux + a.sz * uz, uzr = a.cz * uz - a.sz * ux;
    x = xr;
    zz = zr;
    ux = uxr;
    uz = uzr;
  }
  const double bmag = sqrt(1.0 - 1.0 / (gamma * gamma));
  float b[3] = {(float)(ux * bmag), (float)(uy * bmag), (float)(uz * bmag)};
  double b2 = 0.0;
  for (int it = 0; it < 64; ++it) {
    b2 = ((double)b[0] * b[0] + (double)b[1] * b[1]) + (double)b[2] * b[2];
    if (!(b2 >= 1.0)) break;
    for (int k = 0; k < 3; ++k) b[k] = (float)((double)b[k] * (1.0 - 2e-7));
  }
  b2 = ((double)b[0] * b[0] + (double)b[1] * b[1]) + (double)b[2] * b[2];
  const double t0 = (10000.0 - h) / kCmPerNs;
  const double t1 = t0 + L / (sqrt(b2) * kCmPerNs);
  a.x0[i] = (float)x;
  a.y0[i] = (float)y;
  a.z0[i] = (float)zz;
  a.x1[i] = (float)(x + ux * L);
  a.y1[i] = (float)(y + uy * L);
  a.z1[i] = (float)(zz + uz * L);
  a.t0[i] = (float)t0;
  a.t1[i] = (float)t1;
  a.bx[i] = b[0];
  a.by[i] = b[1];
  a.bz[i] = b[2];
  a.q[i] = q;
}

}  // namespace
}  // namespace c8r

extern "C" int c8r_generate_tracks(uint64_t seed, int64_t first, int64_t n, double zenith_deg,
                                   const c8r_tracks_out* out, void* cuda_stream) {
  using namespace c8r;
  if (!out || n < 0 || first < 0 || !std::isfinite(zenith_deg)) return C8R_EINVAL;
  if (out->dtype != C8R_F32) return C8R_EINVAL;
  void* f[12] = {out->x0, out->y0, out->z0, out->x1, out->y1, out->z1, out->t0, out->t1, out->bx, out->by, out->bz,
                 out->q};
  for (void* p : f)
    if (!p) return C8R_EINVAL;
  if (n == 0) return C8R_OK;
  const double th = zenith_deg * (3.14159265358979323846 / 180.0);
  GenArgs a{seed, first, n, std::cos(th), std::sin(th),
            (float*)f[0], (float*)f[1], (float*)f[2], (float*)f[3], (float*)f[4],  (float*)f[5],
            (float*)f[6], (float*)f[7], (float*)f[8], (float*)f[9], (float*)f[10], (float*)f[11]};
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_generate<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? C8R_OK : C8R_ECUDA;
}
