// trig.cuh -- branch-free sin / cos and log for the rollout step, host- and
// device-callable (the host build serves the accuracy test).  A branch in
// the step (such as the large-argument path of sincosf) splits it into
// separate scheduling regions; these have none.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace brmppi {

// sin and cos of the turn within one path segment, |e| <= pi/4 (rows
// farther apart are rejected when the path is staged): Taylor series of sin
// to e^9 and of cos to e^10, truncation below 2e-9, no branch.
__host__ __device__ __forceinline__ void turn_sincos(float e, float* s, float* c) {
  const float e2 = e * e, e4 = e2 * e2;
  // sin e = e + e^3 (-1/3! + e^2/5! + e^4 (-1/7! + e^2/9!))
  *s = fmaf(e * e2,
            fmaf(e4, fmaf(e2, 2.7557318844628753e-06f, -1.9841270113829523e-04f),
                 fmaf(e2, 8.333333767950535e-03f, -0.1666666716337204f)),
            e);
  // cos e = 1 + e^2 (-1/2! + e^2/4! + e^4 (-1/6! + e^2/8!) - e^8/10!)
  *c = fmaf(e2,
            fmaf(e4 * e4, -2.755731998149713e-07f,
                 fmaf(e4, fmaf(e2, 2.4801587642286904e-05f, -1.3888889225199819e-03f),
                      fmaf(e2, 0.0416666679084301f, -0.5f))),
            1.0f);
}

// sin and cos of a state angle, without branches.  Cody-Waite reduction by
// pi/2 (Cody and Waite, 1980): pi/2 split into the float nearest it and the
// float nearest the remainder; x - k hi is exact for |x| < 2^24 pi/2, so r
// carries one rounding; then turn_sincos on |r| <= pi/4 and the quadrant.
// k = round(x 2/pi) by the shifter 1.5 * 2^23: adding it rounds the product
// to an integer exactly as rintf does (ties to even) for |x 2/pi| < 2^22,
// and the sum's low mantissa bits are k mod 4 -- no rounding or conversion
// instruction on the steer angle's dependency chain.  Within 1.5 ulp of the
// exact values for |x| <= 2^16 (host test against FP64); up to |x| = 2^24
// the outputs stay within 4e-6 of [-1, 1] (beyond 2^22 pi/2 the shifted sum
// loses integer resolution and |r| reaches pi/2, where the Taylor pair is
// still within 3.6e-6); NaN for NaN or infinite x.  Beyond 2^24 rad the
// outputs grow: only a rollout whose steering came within ~1e-7 rad of
// +-pi/2 gets there, and the huge or non-finite cost it then accrues carries
// zero weight in the softmin.
__host__ __device__ __forceinline__ void state_sincos(float x, float* s, float* c) {
  const float t = x * 0.636619746685028f + 12582912.0f;  // 2 / pi; 1.5 * 2^23
  const float kf = t - 12582912.0f;
  uint32_t tb;
#ifdef __CUDA_ARCH__
  tb = __float_as_uint(t);
#else
  std::memcpy(&tb, &t, sizeof(tb));
#endif
  const uint32_t q = tb;  // k mod 4 in the low bits (the shifter is 0 mod 4)
  float r = fmaf(-kf, 1.5707963705062866f, x);
  r = fmaf(-kf, -4.371138828673793e-08f, r);
  float sr, cr;
  turn_sincos(r, &sr, &cr);
  const bool odd = q & 1u;  // x = r + k pi/2
  const float ss = odd ? cr : sr, cc = odd ? sr : cr;
  *s = (q & 2u) ? -ss : ss;
  *c = ((q + 1u) & 2u) ? -cc : cc;
}

// sin and cos of 2 pi u for the Box-Muller uniforms u = (k + 1/2) 2^-23,
// k < 2^23 (the top 23 bits of a Philox word), from k's bits: no
// conversion, no branch.  4u = m + f with m = round(4u) = (k + 2^20) >> 21
// the quadrant and f = (k' + 1/2) 2^-21 - 1/2, k' = (k + 2^20) mod 2^21;
// f is the float 1 + k' 2^-21 (exponent 0, mantissa k' << 2) minus
// 3/2 - 2^-22, exact (Sterbenz).  Then 2 pi u = m pi/2 + r with r = f pi/2,
// |r| <= pi/4: the Taylor pair and the quadrant as in state_sincos.
__host__ __device__ __forceinline__ void unit_turn_sincos(uint32_t k, float* s, float* c) {
  const uint32_t kk = k + (1u << 20);
  const uint32_t m = kk >> 21;
  const uint32_t bits = 0x3f800000u | ((kk & 0x1fffffu) << 2);
  float one_f;
#ifdef __CUDA_ARCH__
  one_f = __uint_as_float(bits);
#else
  std::memcpy(&one_f, &bits, sizeof(one_f));
#endif
  const float r = (one_f - 1.49999976158142089844f) * 1.57079632679489661923f;
  float sr, cr;
  turn_sincos(r, &sr, &cr);
  const bool odd = m & 1u;
  const float ss = odd ? cr : sr, cc = odd ? sr : cr;
  *s = (m & 2u) ? -ss : ss;
  *c = ((m + 1u) & 2u) ? -cc : cc;
}

// -2 ln u for the Box-Muller uniforms u in [2^-24, 1), without branches.
// Cody and Waite's reduction (1980): u = 2^e m with m in [sqrt(1/2),
// sqrt(2)), so ln u = e ln 2 + ln m, and ln m = 2 atanh(s) with
// s = (m - 1) / (m + 1), |s| <= 0.1716, whose odd series to s^9 truncates
// below 2e-9 relative.  ln 2 is split into a 16-bit high part (e times it is
// exact for |e| <= 24) and the float nearest the remainder.  The device
// divides with the MUFU reciprocal (about 2 ulp).
__host__ __device__ __forceinline__ float neg2_log_unit(float u) {
  uint32_t b;
#ifdef __CUDA_ARCH__
  b = __float_as_uint(u);
#else
  std::memcpy(&b, &u, sizeof(b));
#endif
  // e = floor(log2(u / sqrt(1/2))): 0x3f800000 - 0x3f3504f3 (the bits of 1
  // and of sqrt(1/2)) carries into the exponent field when the mantissa
  // reaches sqrt(2); the sum stays positive for positive u
  const int e = static_cast<int>((b + 0x004afb0du) >> 23) - 127;
  const uint32_t mb = b - (static_cast<uint32_t>(e) << 23);  // m = u 2^-e
  float m;
#ifdef __CUDA_ARCH__
  m = __uint_as_float(mb);
#else
  std::memcpy(&m, &mb, sizeof(m));
#endif
  const float f = m - 1.0f;
#ifdef __CUDA_ARCH__
  const float s = __fdividef(f, f + 2.0f);
#else
  const float s = f / (f + 2.0f);
#endif
  const float z = s * s;
  // atanh s / s - 1 = z / 3 + z^2 / 5 + z^3 / 7 + z^4 / 9 + ...
  const float q = z * fmaf(z, fmaf(z, fmaf(z, 0.1111111111111111f, 0.14285714285714285f), 0.2f),
                           0.3333333333333333f);
  const float t = -4.0f * s;
  const float lm = fmaf(t, q, t);  // -2 ln m
  const float ef = static_cast<float>(e);
  // -2 ln 2 = -1.38629150390625 (high part, exact) - 2.8572136e-06
  return fmaf(ef, -1.38629150390625f, fmaf(ef, -2.8572136406188344e-06f, lm));
}

}  // namespace brmppi
