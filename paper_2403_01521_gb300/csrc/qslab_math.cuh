// Device arithmetic shared by the qslab kernels: phases from fixed-point
// positions, complex decays, Philox4x64-10.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab_internal.h"

namespace qslab {

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// --------------------------------------------------------------- phases
// A position is stored as the fraction x/Lx in fixed point (2^32 or 2^64
// units of one turn), so the phase k.rho = 2 pi (mx x/Lx + my y/Ly) reduces
// modulo one turn exactly in integer arithmetic.

__device__ __forceinline__ uint32_t phase_turns(int32_t mx, int32_t my,
                                                uint32_t xh, uint32_t yh) {
  return (uint32_t)mx * xh + (uint32_t)my * yh;
}
__device__ __forceinline__ uint64_t phase_turns(int32_t mx, int32_t my,
                                                uint64_t xh, uint64_t yh) {
  return (uint64_t)(int64_t)mx * xh + (uint64_t)(int64_t)my * yh;
}

// cos and sin of 2 pi ph / 2^32. The phase is rounded to the nearest quarter
// turn in integer arithmetic (exact); the remainder |x| <= pi/4 goes through
// the Taylor series of sin (to x^11) and cos (to x^10), whose truncation
// errors there are below 1e-10.
__device__ __forceinline__ void sincos_turns(uint32_t ph, float& c, float& s) {
  const uint32_t qd = (ph + 0x20000000u) >> 30;
  const int32_t r = (int32_t)(ph - (qd << 30));
  const float x = (float)r * 1.4629180792671596e-9f;  // 2 pi / 2^32
  const float x2 = x * x;
  float sp = fmaf(x2, -2.505210838544172e-8f, 2.7557319223985893e-6f);
  sp = fmaf(x2, sp, -1.984126984126984e-4f);
  sp = fmaf(x2, sp, 8.333333333333333e-3f);
  sp = fmaf(x2, sp, -0.16666666666666666f);
  const float sn = fmaf(x * x2, sp, x);
  float cp = fmaf(x2, -2.755731922398589e-7f, 2.48015873015873e-5f);
  cp = fmaf(x2, cp, -1.388888888888889e-3f);
  cp = fmaf(x2, cp, 0.041666666666666664f);
  cp = fmaf(x2, cp, -0.5f);
  const float cs = fmaf(x2, cp, 1.0f);
  // rotate by qd quarter turns
  const bool swap = qd & 1u;
  const float c0 = swap ? sn : cs;
  const float s0 = swap ? cs : sn;
  c = ((qd + 1u) & 2u) ? -c0 : c0;   // qd = 1, 2 negate cos
  s = (qd & 2u) ? -s0 : s0;          // qd = 2, 3 negate sin
}

// cos and sin of 2 pi ph / 2^32 from a table of the 256 turns j/256 (in
// shared memory, tab[j] = (cos, sin)(2 pi j/256), rounded from FP64 on the
// host) and the remainder x, |x| <= pi/256: sin x = x - x^3/6 (truncation
// below 3e-12), cos x = 1 - x^2/2 (below 1e-9), combined by the angle-sum
// formulas. About half the instructions of the series above; the error is
// about one unit in the last place.
__device__ __forceinline__ void sincos_table(uint32_t ph, const float2* tab, float& c, float& s) {
  const uint32_t j = (ph + 0x800000u) >> 24;            // nearest 1/256 turn
  const int32_t r = (int32_t)(ph << 8) >> 8;            // ph - j 2^24, in [-2^23, 2^23)
  const float x = (float)r * 1.4629180792671596e-9f;    // 2 pi / 2^32
  const float x2 = x * x;
  const float sx = fmaf(x * x2, -0.16666666666666666f, x);
  const float2 t = tab[j & 255u];
  c = fmaf(-t.y, sx, fmaf(t.x * x2, -0.5f, t.x));
  s = fmaf(t.x, sx, fmaf(t.y * x2, -0.5f, t.y));
}

// cos and sin of 2 pi ph / 2^64 in FP64.
__device__ __forceinline__ void sincos_turns(uint64_t ph, double& c, double& s) {
  const double t = (double)(int64_t)ph * 1.0842021724855044e-19;  // 2^-63
  sincospi(t, &s, &c);
}

// phase factors of a mode: FP32 from the shared-memory table, FP64 exact
__device__ __forceinline__ void phase_cs(uint32_t ph, const float2* tab, float& c, float& s) {
  sincos_table(ph, tab, c, s);
}
__device__ __forceinline__ void phase_cs(uint64_t ph, const float2*, double& c, double& s) {
  sincos_turns(ph, c, s);
}

// --------------------------------------------------------------- decays
__device__ __forceinline__ float exp_neg(float x) { return expf(-x); }
__device__ __forceinline__ double exp_neg(double x) { return exp(-x); }
// e^{-x} for terms that enter a sum once (not a product along a scan): the
// fast FP32 exponential (a few ulp) is enough there
__device__ __forceinline__ float exp_neg_term(float x) { return __expf(-x); }
__device__ __forceinline__ double exp_neg_term(double x) { return exp(-x); }

// 1 - e^{-x} for x >= 0, accurate relative to itself. A decay e^{-x} close
// to 1 cannot be stored in FP32 to better than about 6e-8 absolute, which for
// the x ~ 1e-6 of neighbouring particles is a relative error of several
// percent in 1 - e^{-x}; carrying e = 1 - e^{-x} instead keeps it exact to
// rounding. Taylor series to x^5 below 1/16 (truncation < 2e-9 relative).
__device__ __forceinline__ float one_minus_exp_neg(float x) {
  // branch-free: for x >= 1/16, 1 - e^{-x} >= 0.06 and the plain form is exact enough
  const float big = 1.0f - __expf(-x);
  float r = fmaf(x, 1.0f / 120.0f, -1.0f / 24.0f);
  r = fmaf(x, r, 1.0f / 6.0f);
  r = fmaf(x, r, -0.5f);
  r = fmaf(x, r, 1.0f);
  return x < 0.0625f ? x * r : big;
}
__device__ __forceinline__ double one_minus_exp_neg(double x) { return -expm1(-x); }

// e^{-a x} for complex a and real x >= 0.
// The FP32 recurrences multiply by such a decay at every step, and between
// neighbouring particles it lies within 1e-3 of 1: a systematic error of a
// fraction of an ulp in it (as library exp/sincos may have there) adds up
// linearly over a chunk. So for |a x| small the distance from 1 is formed
// from Taylor series (e^{-u} - 1 to u^6, cos v - 1 to v^6, sin v to v^7:
// truncation below 4e-11 relative for u, |v| < 1/16) and added to 1 with a
// single rounding; larger arguments use the library functions.
__device__ __forceinline__ Cplx<float> cexp_neg(float ar, float ai, float x) {
  const float u = ar * x, v = ai * x;
  // small-argument forms (the usual case: neighbouring particles)
  float em = fmaf(u, 1.0f / 720.0f, -1.0f / 120.0f);   // e^{-u} - 1 = -u + u^2/2 - ...
  em = fmaf(u, em, 1.0f / 24.0f);
  em = fmaf(u, em, -1.0f / 6.0f);
  em = fmaf(u, em, 0.5f);
  em = fmaf(u, em, -1.0f);
  em *= u;
  const float v2 = v * v;
  float cm = fmaf(v2, -1.0f / 720.0f, 1.0f / 24.0f);   // cos v - 1
  cm = fmaf(v2, cm, -0.5f);
  cm *= v2;
  float sv = fmaf(v2, -1.0f / 5040.0f, 1.0f / 120.0f);  // sin v
  sv = fmaf(v2, sv, -1.0f / 6.0f);
  sv = fmaf(v * v2, sv, v);
  const float re_small = 1.0f + fmaf(em, cm, em + cm);
  const float im_small = -fmaf(em, sv, sv);
  if (u < 0.0625f && fabsf(v) < 0.0625f) return {re_small, im_small};
  float s, c;
  sincosf(v, &s, &c);
  const float m = expf(-u);
  return {m * c, -m * s};
}
__device__ __forceinline__ Cplx<double> cexp_neg(double ar, double ai, double x) {
  double s, c;
  sincos(ai * x, &s, &c);
  const double m = exp(-ar * x);
  return {m * c, -m * s};
}

// --------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 64x64->128 multiplications with the round keys
// bumped by the Weyl constants.
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c.v[0]), lo0 = M0 * c.v[0];
    const uint64_t hi1 = __umul64hi(M1, c.v[2]), lo1 = M1 * c.v[2];
    U64x4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// --------------------------------------------------------------- warp sums
// Sum of 16 values per lane over the 32 lanes of a warp by recursive halving:
// afterwards every even lane l holds the total of value index l/2.
template <typename T>
__device__ __forceinline__ T warp_reduce16(T (&v)[16], int lane) {
#pragma unroll
  for (int lvl = 0; lvl < 4; ++lvl) {
    const int half = 8 >> lvl;         // 8, 4, 2, 1 values exchanged
    const int mask = 16 >> lvl;        // xor 16, 8, 4, 2
    const bool up = lane & mask;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const T send = up ? v[j] : v[j + half];
      const T keep = up ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// The same over each half-warp apart (lanes 0-15 and 16-31): afterwards lane
// l holds its half's total of value index l % 16.
template <typename T>
__device__ __forceinline__ T half_warp_reduce16(T (&v)[16], int lane) {
#pragma unroll
  for (int lvl = 0; lvl < 4; ++lvl) {
    const int half = 8 >> lvl;         // 8, 4, 2, 1 values exchanged
    const int mask = 8 >> lvl;         // xor 8, 4, 2, 1
    const bool up = lane & mask;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const T send = up ? v[j] : v[j + half];
      const T keep = up ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
  return v[0];
}

}  // namespace qslab
