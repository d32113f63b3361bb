// Host build of the rollout step's branch-free sin / cos and of the
// Box-Muller logarithm and angle (csrc/trig.cuh), compared against the C library's
// double-precision sin / cos / log.  Prints one
// JSON line of maximum errors; tests/test_trig.py runs and judges it.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "trig.cuh"

int main() {
  const double ulp1 = std::ldexp(1.0, -23);  // one ulp of 1.0f
  double turn_s = 0, turn_c = 0, state_s = 0, state_c = 0, state_rel = 0, far_abs = 0;
  // turn_sincos on [-pi/4, pi/4]: every 64th float of a fine grid
  for (int i = -4000000; i <= 4000000; ++i) {
    const float e = static_cast<float>(i * (0.78539816339744831 / 4000000.0));
    float s, c;
    brmppi::turn_sincos(e, &s, &c);
    turn_s = std::fmax(turn_s, std::fabs(s - std::sin(static_cast<double>(e))));
    turn_c = std::fmax(turn_c, std::fabs(c - std::cos(static_cast<double>(e))));
  }
  // state_sincos on [-2^16, 2^16], including points next to multiples of pi/2
  for (int64_t i = -2000000000LL; i <= 2000000000LL; i += 997) {
    const float x = static_cast<float>(i * 3.2768e-5);
    float s, c;
    brmppi::state_sincos(x, &s, &c);
    state_s = std::fmax(state_s, std::fabs(s - std::sin(static_cast<double>(x))));
    state_c = std::fmax(state_c, std::fabs(c - std::cos(static_cast<double>(x))));
  }
  for (int k = -1000; k <= 1000; ++k) {
    float x = static_cast<float>(k * 1.5707963267948966);
    for (int n = 0; n < 5; ++n, x = std::nextafter(x, 1e30f)) {
      float s, c;
      brmppi::state_sincos(x, &s, &c);
      state_s = std::fmax(state_s, std::fabs(s - std::sin(static_cast<double>(x))));
      state_c = std::fmax(state_c, std::fabs(c - std::cos(static_cast<double>(x))));
    }
  }
  // relative error of sin near zero
  for (int i = 1; i <= 2000000; ++i) {
    const float x = static_cast<float>(i * 1e-6);
    float s, c;
    brmppi::state_sincos(x, &s, &c);
    state_rel = std::fmax(state_rel, std::fabs(s / std::sin(static_cast<double>(x)) - 1.0));
  }
  // 2^16 .. 2^24: within [-1, 1] (accuracy not claimed)
  for (int i = 16; i < 24; ++i)
    for (int j = 0; j < 100000; ++j) {
      float s, c;
      brmppi::state_sincos(std::ldexp(1.0f + j * 9.5e-6f, i), &s, &c);
      far_abs = std::fmax(far_abs, std::fmax(std::fabs(s), std::fabs(c)));
    }
  // -2 ln u on every Box-Muller uniform u = (k + 1/2) 2^-23, in ulp of the
  // exact value
  double log_ulp = 0;
  for (uint32_t k = 0; k < (1u << 23); ++k) {
    const float u = (static_cast<float>(k) + 0.5f) * 1.1920928955078125e-07f;
    const double ex = -2.0 * std::log(static_cast<double>(u));
    int ee;
    std::frexp(ex, &ee);
    log_ulp = std::fmax(log_ulp, std::fabs(brmppi::neg2_log_unit(u) - ex) / std::ldexp(1.0, ee - 24));
  }
  // sin / cos of 2 pi u on every Box-Muller uniform, from the bits of k
  double unit_s = 0, unit_c = 0;
  for (uint32_t k = 0; k < (1u << 23); ++k) {
    const double a = 6.283185307179586477 * ((k + 0.5) * std::ldexp(1.0, -23));
    float s, c;
    brmppi::unit_turn_sincos(k, &s, &c);
    unit_s = std::fmax(unit_s, std::fabs(s - std::sin(a)));
    unit_c = std::fmax(unit_c, std::fabs(c - std::cos(a)));
  }
  float sn, cn;
  brmppi::state_sincos(NAN, &sn, &cn);
  std::printf(
      "{\"turn_sin_ulp\": %.4f, \"turn_cos_ulp\": %.4f, \"state_sin_ulp\": %.4f, \"state_cos_ulp\": %.4f, "
      "\"state_sin_rel\": %.3e, \"far_max_abs\": %.4f, \"nan_propagates\": %d, \"neg2_log_ulp\": %.4f, \"unit_sin_ulp\": %.4f, \"unit_cos_ulp\": %.4f}\n",
      turn_s / ulp1, turn_c / ulp1, state_s / ulp1, state_c / ulp1, state_rel, far_abs,
      (std::isnan(sn) && std::isnan(cn)) ? 1 : 0, log_ulp, unit_s / ulp1, unit_c / ulp1);
  return 0;
}
