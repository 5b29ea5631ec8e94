// ingest.cuh -- track ingest and the track filter (§2: "the track is checked
// according to the track filter ... relevant for the radio calculation or not").
//
// One thread per track slot reads the caller's SoA arrays (coalesced), applies
// the filter and writes the per-track quantities every later pair evaluation
// needs into field-major tiles of kTileT tracks.  Everything per track that
// costs FP64 (exp of the altitude, t/dt, 1 - |beta|) is done here once, so the
// pair kernels, which run once per track AND antenna, stay on the FP32 pipe.
// Padding slots and filtered tracks get a zero amplitude and are skipped later.
#pragma once

#include <cmath>

#include "c8r_internal.h"

namespace c8r {
namespace ingest_detail {


template <typename T>
__device__ __forceinline__ double ld(const void* p, int64_t i) {
  return (double)static_cast<const T*>(p)[i];
}

template <typename Tin>
__device__ __forceinline__ void load_track(const TrackPtrs& t, int64_t i, double v[12], bool round_to_f32) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double x = ld<Tin>(t.f[k], i);
    v[k] = round_to_f32 ? (double)(float)x : x;
  }
}

// track filter: q != 0, all fields finite, t1 > t0, |x1 - x0| > 0, 0 < |beta| < 1
// (in FP64, as the definition reads); b = |beta| when kept
__device__ __forceinline__ bool track_kept(const double v[12], double& b) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 12; ++k) ok = ok && isfinite(v[k]);
  if (!ok) return false;
  if (v[11] == 0.0) return false;
  if (!(v[7] > v[6])) return false;
  double lx = v[3] - v[0], ly = v[4] - v[1], lz = v[5] - v[2];
  if (!(lx * lx + ly * ly + lz * lz > 0.0)) return false;
  b = sqrt(v[8] * v[8] + v[9] * v[9] + v[10] * v[10]);
  return b > 0.0 && b < 1.0;
}

// float x float-float -> float-float, renormalised (relative error ~2^-47)
__device__ __forceinline__ void mul_f_ff(float a, float bh, float bl, float& h, float& l) {
  float p, e;
  two_prod(a, bh, p, e);
  e = __fmaf_rn(a, bl, e);
  h = __fadd_rn(p, e);
  l = __fsub_rn(e, __fsub_rn(h, p));
}

__device__ __forceinline__ void split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// track filter of the mixed path on FP32 values (the inputs rounded to FP32),
// taking the same decisions as the FP64 form above: for FP32 values, |x1 - x0|
// > 0 in FP64 iff some coordinate differs, and sqrt(S) < 1 iff S < 1 for the
// FP64 sum S = (bx^2 + by^2) + bz^2, evaluated in the same order and rounding
__device__ __forceinline__ bool track_kept_f32(const float f[12], double& S) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 12; ++k) ok = ok && isfinite(f[k]);
  if (!ok) return false;
  if (f[11] == 0.0f) return false;
  if (!(f[7] > f[6])) return false;
  if (f[3] == f[0] && f[4] == f[1] && f[5] == f[2]) return false;
  const double bx = f[8], by = f[9], bz = f[10];
  S = __dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz));
  return S > 0.0 && S < 1.0;
}

__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  float p, e;
  two_prod(ah, bh, p, e);
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  fast_two_sum(p, e, h, l);
}
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, h, l);
}

// e^x in float-float for x = xh + xl, |x| <= 60, from FP32 arithmetic.
// Cody-Waite reduction x = k ln2 + r, with ln2 split in three parts of which
// the first has 16 significant bits (k times it is exact for |k| < 2^8), then
// the Taylor series of e^r, |r| <= ln2/2, to r^12/12! (truncation below
// 2^-47): the terms from r^7 on in FP32, which is enough for their size, the
// others in float-float by Horner's rule; finally the exact scaling by 2^k.
__device__ __forceinline__ void exp_ff(float xh, float xl, float& eh, float& el) {
  constexpr float L1 = 0.693145751953125f, L2 = 1.428606765330187e-06f, L3 = 5.4956039718945e-14f;
  const float k = rintf(__fmul_rn(xh, 1.44269504088896341f));
  const float t = __fsub_rn(xh, __fmul_rn(k, L1));  // exact (Sterbenz)
  float ph, pl;
  two_prod(k, L2, ph, pl);
  float rh, rl;
  two_sum(t, -ph, rh, rl);
  rl = __fadd_rn(rl, __fsub_rn(__fsub_rn(xl, pl), __fmul_rn(k, L3)));
  fast_two_sum(rh, rl, rh, rl);
  // sum_{n=7..12} r^(n-7)/n!
  float q = 1.0f / 479001600.0f;
  q = __fmaf_rn(q, rh, 1.0f / 39916800.0f);
  q = __fmaf_rn(q, rh, 1.0f / 3628800.0f);
  q = __fmaf_rn(q, rh, 1.0f / 362880.0f);
  q = __fmaf_rn(q, rh, 1.0f / 40320.0f);
  q = __fmaf_rn(q, rh, 1.0f / 5040.0f);
  // 1/n! for n = 6 .. 0 as float-float (high part, low part)
  constexpr float ch[7] = {1.0f / 720.0f, 1.0f / 120.0f, 1.0f / 24.0f, 1.0f / 6.0f, 0.5f, 1.0f, 1.0f};
  constexpr double cd[7] = {1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0};
  float h = q, l = 0.0f;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    ff_mul(h, l, rh, rl, h, l);
    ff_add(h, l, ch[j], (float)(cd[j] - (double)ch[j]), h, l);
  }
  const float s = __int_as_float(((int)k + 127) << 23);  // 2^k, |k| <= 87
  eh = __fmul_rn(h, s);
  el = __fmul_rn(l, s);
}

// E = exp(-z/H) as float-float for an FP32 altitude given as zh + zl (m)
__device__ __forceinline__ void exp_alt(float zh, float zl, const MedParams& M, float& eh, float& el) {
  float xh, xl;
  ff_mul(-zh, -zl, M.invH_h, M.invH_l, xh, xl);
  if (fabsf(xh) <= 60.0f) {
    exp_ff(xh, xl, eh, el);
  } else {  // far outside the atmosphere model's range: FP64
    split(exp((double)xh + (double)xl), eh, el);
  }
}


// Map: padded slot g -> index of the caller's track in that slot, or -1 for a
// padding slot (identity for one shower; a per-shower table for a batch)
template <typename Tin, class Map>
__global__ void __launch_bounds__(256) k_ingest_mixed(TrackPtrs t, Map map, int64_t n_pad, float* tiles,
                                                      MedParams M, unsigned long long* kept,
                                                      unsigned long long* form) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false, from_above = false;
  if (i < n_pad) {
    float* tile = tiles + (i / kTileT) * (int64_t)(fm::NFIELDS * kTileT);
    const int l = (int)(i % kTileT);
    float out[fm::NFIELDS];
#pragma unroll
    for (int k = 0; k < fm::NFIELDS; ++k) out[k] = 0.0f;
    const int64_t src = map(i);
    if (src >= 0) {
      // the mixed path takes its inputs as FP32 values; the per-track quantities
      // are formed in float-float on the FP32 pipe, FP64 (slow on this part)
      // only for |beta|^2
      float f[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) f[k] = (float)static_cast<const Tin*>(t.f[k])[src];
      double S = 0.0;
      keep = track_kept_f32(f, S);
      if (keep) {
        out[fm::X0] = f[0]; out[fm::Y0] = f[1]; out[fm::Z0] = f[2];
        // the start point sees the antenna array's centroid from above, within
        // 45 degrees of the vertical (the vote for the split arrival form)
        const float sx = M.cen_x - f[0], sy = M.cen_y - f[1], sz = M.cen_z - f[2];
        const float P = sx * sx + sy * sy;
        from_above = sz < 0.0f && P < sz * sz;
        out[fm::X1] = f[3]; out[fm::Y1] = f[4]; out[fm::Z1] = f[5];
        out[fm::BX] = f[8]; out[fm::BY] = f[9]; out[fm::BZ] = f[10];
        // tau = t/dt, (t1 - t0)/dt = (exact difference) x 1/dt
        mul_f_ff(f[6], M.idt_h, M.idt_l, out[fm::TAU0H], out[fm::TAU0L]);
        mul_f_ff(f[7], M.idt_h, M.idt_l, out[fm::TAU1H], out[fm::TAU1L]);
        float dh, dl;
        two_sum(f[7], -f[6], dh, dl);
        float ph, pl;
        mul_f_ff(dh, M.idt_h, M.idt_l, ph, pl);
        pl = __fmaf_rn(dl, M.idt_h, pl);
        out[fm::DTAUH] = __fadd_rn(ph, pl);
        out[fm::DTAUL] = __fsub_rn(pl, __fsub_rn(out[fm::DTAUH], ph));
        out[fm::AMPE] = __fmul_rn(f[11], M.ampE);
        out[fm::AMPZ] = __fmul_rn(__fmul_rn(f[11], M.kzhs), out[fm::DTAUH]);
        // |beta| = sqrt(S); 1 - |beta| = (1 - S)/(1 + |beta|), 1 - S exact in FP64
        const float bmag = sqrtf((float)S);
        out[fm::BMAG] = bmag;
        out[fm::OMB] = __fdiv_rn((float)__dsub_rn(1.0, S), __fadd_rn(1.0f, bmag));
        if (M.kind != C8R_UNIFORM) {  // flat exp(-z/H); the sphere's part comes per pair
          exp_alt(f[2], 0.0f, M, out[fm::E0H], out[fm::E0L]);
          exp_alt(f[5], 0.0f, M, out[fm::E1H], out[fm::E1L]);
          float zmh, zml;  // (z0 + z1)/2, exact
          two_sum(f[2], f[5], zmh, zml);
          exp_alt(0.5f * zmh, 0.5f * zml, M, out[fm::EMH], out[fm::EML]);
        } else {
          out[fm::E0H] = out[fm::E1H] = out[fm::EMH] = 1.0f;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < fm::NFIELDS; ++k) tile[k * kTileT + l] = out[k];
  }
  // counts summed over the block first: one reduction per block and counter
  // (from every warp, these same-address reductions cost more than the ingest)
  const int nk = __syncthreads_count(keep);
  const int nv = form ? __syncthreads_count(from_above) : 0;  // form: uniform over the grid
  if (threadIdx.x == 0 && nk) {
    if (kept) atomicAdd(kept, (unsigned long long)nk);
    if (form) {
      atomicAdd(form, (unsigned long long)nk);  // kept tracks, and those seen from above
      if (nv) atomicAdd(form + 1, (unsigned long long)nv);
    }
  }
}

template <typename Tin, class Map>
__global__ void __launch_bounds__(256) k_ingest_f64(TrackPtrs t, Map map, int64_t n_pad, double* tiles,
                                                    MedParams M, unsigned long long* kept) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (i < n_pad) {
    double* tile = tiles + (i / kTileT) * (int64_t)(fd::NFIELDS * kTileT);
    const int l = (int)(i % kTileT);
    double out[fd::NFIELDS];
#pragma unroll
    for (int k = 0; k < fd::NFIELDS; ++k) out[k] = 0.0;
    const int64_t src = map(i);
    if (src >= 0) {
      double v[12];
      load_track<Tin>(t, src, v, false);
      double b;
      keep = track_kept(v, b);
      if (keep) {
#pragma unroll
        for (int k = 0; k < 6; ++k) out[fd::X0 + k] = v[k];
        out[fd::BX] = v[8]; out[fd::BY] = v[9]; out[fd::BZ] = v[10];
        out[fd::Q] = v[11];
        out[fd::T0] = v[6];
        out[fd::T1] = v[7];
        if (M.kind != C8R_UNIFORM) {
          out[fd::E0] = exp(-v[2] * M.invH);
          out[fd::E1] = exp(-v[5] * M.invH);
          out[fd::EM] = exp(-(0.5 * (v[2] + v[5])) * M.invH);
        } else {
          out[fd::E0] = out[fd::E1] = out[fd::EM] = 1.0;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < fd::NFIELDS; ++k) tile[k * kTileT + l] = out[k];
  }
  const int nk = __syncthreads_count(keep);
  if (kept && threadIdx.x == 0 && nk) atomicAdd(kept, (unsigned long long)nk);
}


struct IdentityMap {
  int64_t n;
  __device__ __forceinline__ int64_t operator()(int64_t g) const { return g < n ? g : -1; }
};

}  // namespace ingest_detail

template <class Map>
cudaError_t launch_ingest_map(int precision, const TrackPtrs& t, const Map& map, int64_t n_pad, void* tiles,
                              const MedParams& M, unsigned long long* kept, cudaStream_t st,
                              unsigned long long* form = nullptr) {
  using namespace ingest_detail;
  if (n_pad <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_pad + threads - 1) / threads;
  if (precision == C8R_FP64) {
    if (t.dtype == C8R_F64)
      k_ingest_f64<double, Map><<<(unsigned)blocks, threads, 0, st>>>(t, map, n_pad, (double*)tiles, M, kept);
    else
      k_ingest_f64<float, Map><<<(unsigned)blocks, threads, 0, st>>>(t, map, n_pad, (double*)tiles, M, kept);
  } else {
    if (t.dtype == C8R_F64)
      k_ingest_mixed<double, Map><<<(unsigned)blocks, threads, 0, st>>>(t, map, n_pad, (float*)tiles, M, kept, form);
    else
      k_ingest_mixed<float, Map><<<(unsigned)blocks, threads, 0, st>>>(t, map, n_pad, (float*)tiles, M, kept, form);
  }
  return cudaGetLastError();
}

}  // namespace c8r
