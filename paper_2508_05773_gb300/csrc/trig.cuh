// trig.cuh -- branch-free sin / cos for the rollout step, host- and
// device-callable (the host build serves the accuracy test).  A branch in
// the step (such as the large-argument path of sincosf) splits it into
// separate scheduling regions; these have none.
#pragma once

#include <cmath>
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
// Within 1.5 ulp of the exact values for |x| <= 2^16 (host test against
// FP64), within [-1, 1] up to |x| = 2^24, NaN for NaN or infinite x.
// Beyond 2^24 rad the rounding of x 2/pi leaves r unbounded: only a rollout
// whose steering came within ~1e-7 rad of +-pi/2 gets there, and the huge
// or non-finite cost it then accrues carries zero weight in the softmin.
__host__ __device__ __forceinline__ void state_sincos(float x, float* s, float* c) {
  const float kf = rintf(x * 0.636619746685028f);  // 2 / pi
#ifdef __CUDA_ARCH__
  const int q = static_cast<int>(kf);  // cvt.rzi: saturates, NaN -> 0
#else
  // the same in host C++, where the conversion of NaN or of |kf| >= 2^31 is
  // undefined: clamp first (only q mod 4 is used), NaN -> 0
  const int q = (kf == kf) ? static_cast<int>(fminf(fmaxf(kf, -1073741824.0f), 1073741824.0f)) : 0;
#endif
  float r = fmaf(-kf, 1.5707963705062866f, x);
  r = fmaf(-kf, -4.371138828673793e-08f, r);
  float sr, cr;
  turn_sincos(r, &sr, &cr);
  const bool odd = q & 1;  // x = r + q pi/2
  const float ss = odd ? cr : sr, cc = odd ? sr : cr;
  *s = (q & 2) ? -ss : ss;
  *c = ((q + 1) & 2) ? -cc : cc;
}

}  // namespace brmppi
