// rollout.cuh -- device code of BR-MPPI solves for sm_103a.
//
// Paper: "GPU-Accelerated Barrier-Rate Guided MPPI Control for
// Tractor-Trailer Systems" (arXiv 2508.05773).  One solve (Sec. II-B MPPI
// with the BR-MPPI rollout of Sec. IV-A):
//
//   for each sample s, step tau:
//     noise        Philox4x32-10 + Box-Muller, recomputed (never stored in
//                  HBM): in registers a step ahead (one lane per sample) or
//                  by noise warps into shared memory (wider teams)
//     sample       z_des = clip(U_nom + sigma n), u^alpha_des = clip(sigma_a n)
//     rows         barrier-rate equality per constraint (Eq. cbf_equality):
//                  hitch (Eq. hitch_angle_barrier) and obstacles
//                  (Eq. barrier_function) through the second-order expansion
//                  of Eq. barrier_function_approx (optionally third order for
//                  obstacles; moving and e = 4 obstacles, footprint discs, the
//                  jerk-input model: the extended instantiations)
//     projection   Eq. closed-form_projection in Woodbury form (below)
//     apply        u = clip(z*_u), alpha += z*_alpha
//     dynamics     explicit Euler (Eq. tt_discrete_kinematics)
//     cost         Eq. cost_function_contour at the new state
//   softmin + update (Eq. MPPI_update_rule) as per-tile partials of a
//   max-subtracted log-sum-exp, merged in tile order by the CTA that
//   finishes an instance's last tile.
//
// Launch model.  A work item is (instance, sample tile); a tile is the
// samples one CTA rolls out together.  A plain solve runs one CTA per tile;
// a batch runs a persistent grid that pulls items from a longest-first list
// with an atomic counter.  Partials are per tile and merged in tile order,
// so a solve gives the same bits alone or inside any batch with the same
// launch shape.
//
// Team decomposition: TPS consecutive lanes own one sample.  Every lane of
// a team computes the hitch row (its terms enter the team sums once); the
// obstacle rows are spread round-robin over the team (row j on lane
// j % TPS), each with its noise normal 4 + j.  The rank-2 structure of the
// projection makes the cross-lane exchange five floats per step.
//
// Projection in Woodbury form.  A = [A_u | diag(h~)] where only the a and
// omega columns of A_u are non-zero, M = diag(m_u, m_alpha):
//   K = A M^-1 A^T = D + A_u M_u^-1 A_u^T,  D = diag(h~^2 / m_alpha),
//   S2 = M_u + A_u^T D^-1 A_u (2x2),  g = A_u^T D^-1 r,  y = S2^-1 g,
//   r  = A M^-1 p - b,  lambda = D^-1 (r - A_u y),
//   z*_u = M_u^-1 p_u - y,  z*_alpha_i = p_alpha_i/m_alpha - (r_i - a_i.y)/h~_i,
// algebraically identical to M^-1 [p - A^T K^-1 (A M^-1 p - b)].  With
// u_i = a_i / h~_i and rho_i = r_i / h~_i (one reciprocal per row):
//   S2 = M_u + m_alpha sum u_i u_i^T,  g = m_alpha sum u_i rho_i,
// so the rows accumulate the sums and m_alpha is applied once.
//
// Numerics: states are carried relative to the initial pose (position
// relative to (px0, py0), angles relative to theta1_0, progress relative to
// psi0) so that binary32 rounding is relative to the few metres a rollout
// travels; position, speed, progress and the cost sum are compensated pairs
// (TwoSum); the softmin works on pair differences.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "trig.cuh"

namespace brmppi {

// ------------------------------------------------------------ descriptors
// Method constants shared by every instance of a launch.
struct KConst {
  int proj;
  int coll, obs8, abuf;  // collision cost, moving / e = 4 obstacle rows, buffer cost
  float Ts, hTs2, Ts2, inv_lambda;  // Ts, Ts^2 / 2, Ts^2
  float inv_l1, inv_l2, k_hitch, dtheta_max, kappa, r_inflate;
  float Qc, Ql, Qth, R0, R1, R2, mu, nu_bar;
  float zlo0, zlo1, zlo2, zhi0, zhi1, zhi2, sig0, sig1, sig2;
  float alpha0, sigma_alpha, ua_lo, ua_hi;
  float w_u0, w_u1, w_u2, pc_u0, pc_u1, pc_u2;  // W_u and rho/2 (hi + lo)
  float m_u0, m_u1, inv_m_u0, inv_m_u1, inv_m_u2;
  float w_am, pc_am, m_a;  // W_alpha / m_alpha, rho (hi + lo) / (2 m_alpha), m_alpha = W_alpha + rho
  float h_floor;
  float q_coll, q_abuf, inv_hbuf;
  float alpha_stab, inv_qs0, inv_qs1;  // hitch stabilizer: CBF rate, Q_h^-1
  int nd, discs;                       // footprint discs; non-default footprint
  int third;                           // obstacle rows to third order (rear-axle point only)
  int jerk;                            // jerk-input model: a is a state (x0[7]), input 0 the jerk
  float Ts3_6;                         // Ts^3 / 6
  float inv_nd;
  float disc_e1[8], disc_e2[8];        // disc m at p + disc_e1[m] e1 + disc_e2[m] e2
};

// One solve of a launch (all pointers device memory).
struct Inst {
  const double* x0;
  const float* U_nom;
  const float* obs;
  const float* path;
  float* U_out;
  float* traj_out;   // may be null
  float* J_out;      // may be null
  float* U_next;     // may be null
  int32_t* status;   // may be null
  float* states_out;  // may be null: every sample's states, S x (H+1) x 7
  float* u_safe;      // may be null: stabilized U*[0] (a, omega, nu, slack), written
                      // by the stabilizer launch that follows the solve
  float* inputs_out;  // may be null: every sample's applied inputs, S x H x 3
  float* J_lo_out;    // may be null: low parts of the compensated costs (J_out the high parts)
  float* part;       // tiles * part_stride floats
  unsigned int* sync;  // [0] finished tiles, [1] error bits
  int S, H, n_obs, n_pts, tiles, part_stride;
  float ds, inv_ds;
  double inv_ds_d;   // 1 / ds in FP64 (path cell of psi0)
  uint32_t key0, key1, ctr;
  int P;             // Philox blocks per step, ceil((4 + n_obs) / 4)
  int tile_base;     // single launches: tile index of the first CTA (a rank's share of the tiles)
  int no_merge;      // 1: write the tile partials (at part + (tile - tile_base) * part_stride) and
                     // stop; the instance's tiles are merged by merge_tiles_kernel
};

// Shared-memory capacities of a launch (floats).
// Every region is a multiple of 4 floats (16 bytes): float4 accesses stay
// aligned.
struct SmemCaps {
  int obs, path, phead, unom, ustar;
  int noise_per_team;  // teams wider than one lane: staged normals, 2 steps x P blocks x 4
  int uh_per_team;     // 3 H when the applied-input history stays in shared memory, else 0
  int merge;           // > 0: room for an instance's tile partials (merged in shared memory)
  __host__ __device__ static int pad4(int n) { return (n + 3) & ~3; }
  __host__ __device__ int total(int spb) const {
    const int tail = noise_per_team * spb + pad4(uh_per_team * spb);  // noise, history; then the partials
    return obs + path + phead + unom + ustar + pad4(3 * spb) + 256 + 16 + (tail > merge ? tail : merge);
  }
};

struct LaunchDesc {
  Inst single;          // used when work == nullptr (tile = blockIdx.x)
  const Inst* inst;     // batch: instance table
  const int2* work;     // batch: (instance, tile) items, longest first
  int n_work;
  unsigned int* work_ctr;  // [0] next item, [1] CTAs that ran out of work
  float* uh;            // per-CTA applied-input history: gridDim.x * uh_stride floats
                        // (unused by the exact-rows variants: their history is in shared memory)
  int uh_stride;        // 3 * H_max * samples per CTA
  int noise_warps;      // teams wider than one lane: warps that produce the noise
  int rows;             // > 0: the instantiation with exactly this many rows a lane
  SmemCaps caps;
};

enum : unsigned { ERR_EXPONENT = 1u, ERR_NONFINITE_X0 = 2u, ERR_PATH_TURN = 4u };

// Largest heading change between consecutive path rows (rad): the stage
// cost's interpolated heading turns a row's direction by at most this.
constexpr float kMaxPathTurn = 0.78539816339744831f;  // pi / 4

// ------------------------------------------------------------------- noise
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies; the key advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Two words -> two standard normals (Box-Muller). Uniform map
// u = ((w >> 9) + 1/2) 2^-23 in (0, 1), exact in binary32.  It is formed
// from bits, without an integer-to-float conversion: the float with
// exponent 0 and mantissa w >> 9 is 1 + (w >> 9) 2^-23, and subtracting
// 1 - 2^-24 from it is exact (Sterbenz: the operands are within a factor of
// two).  The angle 2 pi u_b is reduced from the bits of w_b >> 9 too
// (unit_turn_sincos).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const float ua = __uint_as_float(0x3f800000u | (wa >> 9)) - 0.999999940395355224609375f;
  // -2 ln ua lies in [1.2e-7, 33.3] (normal floats), taken without a
  // branch (neg2_log_unit); the radius as x rsqrt(x), no slow path
  const float r2 = neg2_log_unit(ua);
  const float radius = r2 * rsqrtf(r2);
  float sn, cs;
  unit_turn_sincos(wb >> 9, &sn, &cs);
  n0 = radius * cs;
  n1 = radius * sn;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }


// into [-pi, pi]; only the square of the result is used.  The turn count
// is rounded by the 1.5 * 2^23 shifter (as rintf for |a| < 2^22 2 pi; no
// rounding instruction)
__device__ __forceinline__ float wrap_pi(float a) {
  const float n = (a * 0.15915494309189533577f + 12582912.0f) - 12582912.0f;
  return a - 6.28318530717958647692f * n;
}

template <int TPS>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
  for (int m = 1; m < TPS; m <<= 1) v += __shfl_xor_sync(0xffffffffu, v, m, TPS);
  return v;
}

template <int TPS>
__device__ __forceinline__ float team_bcast0(float v) {
  if constexpr (TPS == 1) return v;
  return __shfl_sync(0xffffffffu, v, 0, TPS);
}

// (h, l) pairs: lexicographic order of normalised pairs
__device__ __forceinline__ bool pair_less(float ah, float al, float bh, float bl) {
  return ah < bh || (ah == bh && al < bl);
}

// x = hi + lo with hi = fl(x)
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  hi = static_cast<float>(x);
  lo = static_cast<float>(x - static_cast<double>(hi));
}

// Compensated accumulation (TwoSum): (h, l) += inc with the rounding error
// of the float sum carried in l.
__device__ __forceinline__ void acc2(float& h, float& l, float inc) {
  const float sum = h + inc;
  const float bp = sum - h;
  l += (h - (sum - bp)) + (inc - bp);
  h = sum;
}

// Barrier-rate row of the hitch barrier h = dtheta_max - kappa v - |Delta|,
// Delta = theta2 - theta1 (Eq. hitch_angle_barrier), through the
// second-order expansion of Eq. barrier_function_approx: the increment
// Ts hdot + Ts^2/2 hddot along the field with the input held is
// Aa a + Aw omega + c0 (progress never enters).  sp, cp = sin, cos of
// phi = -Delta; tn = tan(delta).
struct HitchRow {
  float h, Aa, Aw, c0;
};
__device__ __forceinline__ HitchRow hitch_row(const KConst& k, float Delta, float sp, float cp, float tn,
                                              float vv, float th1dot) {
  const float sg = Delta >= 0.f ? 1.f : -1.f;
  const float G = sp - k.k_hitch * cp * tn;
  const float th2dot = vv * G * k.inv_l2;
  const float phidot = th1dot - th2dot;
  const float sec2 = 1.f + tn * tn;
  HitchRow r;
  r.h = k.dtheta_max - k.kappa * vv - sg * Delta;
  r.Aa = -k.Ts * k.kappa - k.hTs2 * sg * (G * k.inv_l2 - tn * k.inv_l1);
  r.Aw = k.hTs2 * sg * vv * sec2 * (k.k_hitch * cp * k.inv_l2 + k.inv_l1);
  r.c0 = -k.Ts * sg * (th2dot - th1dot) - k.hTs2 * sg * vv * k.inv_l2 * (cp + k.k_hitch * tn * sp) * phidot;
  return r;
}

// Hitch-angle stabilizer (Sec. IV-D, Eq. hitch_angle_qp): the (a, omega)
// (jerk-input model: (jerk, omega)) nearest the reference in the diag(q_stab) norm, inside the input box,
// whose hitch increment g.u + c0 meets the discrete CBF condition
// (Eq. barrier_constraint_prelim, sign of Eq. cbf_equality)
//   g.u >= rhs = -alpha_stab h - c0.
// KKT with a diagonal weight and a box: the box projection of the reference
// if it meets the condition; else u(mu) = clip(u_ref + mu Q^-1 g) at the
// mu > 0 where g.u(mu) = rhs.  g.u(mu) is piecewise linear and
// non-decreasing with breaks where a coordinate meets a bound, so the root is
// found exactly on the segment that crosses rhs.  No crossing: the box
// corner that maximises the increment.  out = (a, omega, nu, slack).
__device__ __forceinline__ void hitch_stabilize(const KConst& k, float Delta, float vv, float dl, float acc, float ua,
                                                float uw, float un, float* out) {
  float sp, cp;
  sincosf(-Delta, &sp, &cp);
  const float tn = tanf(dl);
  HitchRow r = hitch_row(k, Delta, sp, cp, tn, vv, vv * tn * k.inv_l1);
  if (k.jerk) {  // jerk-input model: (jerk, omega), the acceleration acc a state
    r.c0 += acc * r.Aa;
    r.Aa = -k.hTs2 * k.kappa;
  }
  const float g0 = r.Aa, g1 = r.Aw;
  const float rhs = -k.alpha_stab * r.h - r.c0;
  float a = clampf(ua, k.zlo0, k.zhi0), w = clampf(uw, k.zlo1, k.zhi1);
  const float f0 = g0 * a + g1 * w;
  if (f0 < rhs) {
    const float d0 = g0 * k.inv_qs0, d1 = g1 * k.inv_qs1;
    // breakpoints: the mu > 0 where a coordinate meets a bound (+inf: none)
    auto brk = [](float ref, float d, float bound) {
      const float m = (bound - ref) / d;
      return (d != 0.f && m > 0.f) ? m : CUDART_INF_F;
    };
    float b0 = brk(ua, d0, k.zlo0), b1 = brk(ua, d0, k.zhi0);
    float b2 = brk(uw, d1, k.zlo1), b3 = brk(uw, d1, k.zhi1);
    auto cswap = [](float& x, float& y) {
      const float lo = fminf(x, y), hi = fmaxf(x, y);
      x = lo;
      y = hi;
    };
    cswap(b0, b1);  // sorting network for four keys
    cswap(b2, b3);
    cswap(b0, b2);
    cswap(b1, b3);
    cswap(b1, b2);
    float m_prev = 0.f, f_prev = f0;
    bool crossed = false;
    const float bs[4] = {b0, b1, b2, b3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float m = bs[i];
      if (crossed || !(m < CUDART_INF_F)) continue;
      const float f = g0 * clampf(ua + m * d0, k.zlo0, k.zhi0) + g1 * clampf(uw + m * d1, k.zlo1, k.zhi1);
      if (f >= rhs) {
        const float mu = m_prev + (rhs - f_prev) * (m - m_prev) / (f - f_prev);
        a = clampf(ua + mu * d0, k.zlo0, k.zhi0);
        w = clampf(uw + mu * d1, k.zlo1, k.zhi1);
        crossed = true;
      }
      m_prev = m;
      f_prev = f;
    }
    if (!crossed) {
      if (d0 != 0.f) a = d0 > 0.f ? k.zhi0 : k.zlo0;
      if (d1 != 0.f) w = d1 > 0.f ? k.zhi1 : k.zlo1;
    }
  }
  out[0] = a;
  out[1] = w;
  out[2] = un;
  out[3] = (g0 * a + g1 * w) - rhs;
}

// Frame of one solve (relative coordinates).  Doubles of x0 enter as
// unevaluated float pairs (hi + lo), so the staging needs no FP64 trig.
struct Frame {
  float ox_h, ox_l, oy_h, oy_l, oth_h, oth_l;  // origin (px0, py0, theta1_0)
  float c0, s0;                                // cos / sin of theta1_0
  float t2, v_h, v_l, dl;                      // theta2 - theta1_0, speed, steer angle
  float a0;                                    // acceleration (jerk-input model)
  float qf0;                                   // fractional path cell of psi0
  int i0;                                      // integer path cell of psi0
  float psi_h, psi_l;                          // psi0
  double psi0;
};

// The frame of x0, built by warp 0: lane j takes state component j, so the
// FP64 work runs side by side; the path cell of psi0 uses the host's FP64
// reciprocal of ds (no device division).
__device__ __forceinline__ void make_frame_warp(const double* x0, double inv_ds, unsigned int* err, Frame& fr,
                                                bool jerk) {
  const int lane = threadIdx.x & 31;
  if (lane >= (jerk ? 8 : 7)) {
    if (lane == 7) fr.a0 = 0.f;
    return;
  }
  const double x = x0[lane];
  if (!isfinite(x)) atomicOr(err, ERR_NONFINITE_X0);
  float hi, lo;
  split_double(x, hi, lo);
  switch (lane) {
    case 0: fr.ox_h = hi; fr.ox_l = lo; break;
    case 1: fr.oy_h = hi; fr.oy_l = lo; break;
    case 2: {
      fr.oth_h = hi;
      fr.oth_l = lo;
      float sn, cs;
      sincosf(hi, &sn, &cs);
      fr.c0 = cs - sn * lo;  // cos(hi + lo), lo below one ulp of hi
      fr.s0 = sn + cs * lo;
      break;
    }
    case 3: fr.t2 = static_cast<float>(x - x0[2]); break;
    case 4: fr.v_h = hi; fr.v_l = lo; break;
    case 5: fr.dl = static_cast<float>(x); break;
    case 6: {
      fr.psi0 = x;
      fr.psi_h = hi;
      fr.psi_l = lo;
      const double q0 = x * inv_ds;
      const double fq = fmin(fmax(floor(q0), -1.0e9), 1.0e9);
      fr.i0 = static_cast<int>(fq);
      fr.qf0 = static_cast<float>(q0 - fq);
      break;
    }
    default: fr.a0 = static_cast<float>(x); break;  // lane 7: acceleration (jerk-input model)
  }
}

// Shared memory of a CTA (offsets into the dynamic buffer, floats).
struct Smem {
  float* obs;    // 8 per obstacle.  Plain family (parked ellipses): cx, cy,
                 // Qxx, Qxy, Qyy, 0, 0, 0 (the world-axis quadratic form of
                 // h).  Family with the optional terms: cx, cy, cos, sin, kx,
                 // ky, vx', vy' with k = 1/A^2 (e = 2) or 1/A^4 (e = 4, kx
                 // stored negated) and the velocity in the obstacle frame
                 // (zero unless moving)
  float* path;   // 3 per row: x, y, heading (relative frame)
  float* phead;  // 2 per row: cos, sin of the row's heading in world axes
  float* unom;   // 3H
  float* ustar;  // 3H + 1 (merge)
  float* jh;     // spb
  float* jl;     // spb
  float* w;      // spb
  float* chunk;  // 256
  float* disc;   // 16: lever arms (along e1, along e2) of the footprint discs
  float* noise;  // spb x noise_per_team, then (exact-rows variants) the
                 // applied-input history, 3H x spb
  int noise_per_team;
  __device__ Smem(float* base, const SmemCaps& c, int spb) {
    obs = base;
    path = obs + c.obs;
    phead = path + c.path;
    unom = phead + c.phead;
    ustar = unom + c.unom;
    jh = ustar + c.ustar;
    jl = jh + spb;
    w = jl + spb;
    chunk = jh + SmemCaps::pad4(3 * spb);
    disc = chunk + 256;
    noise = disc + 16;
    noise_per_team = c.noise_per_team;
  }
};

struct Shared {
  Frame fr;
  float red_h[2], red_l[2];
  float wred_h[16], wred_l[16];  // per-warp pair minima (merge)
  int item;
  int last;
  unsigned err;  // the instance's error bits (merge)
};

// Asynchronous 4-byte copy global -> shared (cp.async): the copies of a
// loop stay in flight together instead of one load-store round trip each.
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// L2 prefetch of a global address (no value; null-safe).  Issued early for
// the outputs that the last CTA writes at the very end, it takes their
// address translation and line allocation off the solve's tail.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  if (p) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// grad h . e1' in the obstacle frame.
__device__ __forceinline__ float gda3(float hx, float hy, float dirx, float diry) { return hx * dirx + hy * diry; }

// Threads of a CTA that roll out samples: all of them with one lane per
// sample; with wider teams the last noise_warps warps produce the noise.
template <int TPS>
__device__ __forceinline__ int compute_threads(int noise_warps) {
  return static_cast<int>(blockDim.x) - 32 * noise_warps;
}

// Variants whose noise comes from producer warps: wider teams with at most
// two Philox blocks per lane.
template <int TPS, int BPT>
constexpr bool kNoiseWarps = TPS > 1 && BPT <= 2;

// The per-step hand-over between the noise warp and the compute warps
// (named barrier 1, every thread of the CTA; whole warps take one role).
__device__ __forceinline__ void step_barrier() { asm volatile("bar.sync 1, %0;" ::"r"(blockDim.x) : "memory"); }

// ----------------------------------------------------------- one sample tile
template <int TPS, int BPT, bool EXT, int ROWS>
__device__ void run_tile(const KConst& k, const Inst& in, int tile, float* uh, const Smem& S,
                         Shared& sh, int noise_warps) {
  // Teams wider than one lane run with extra warps (the last ones) that
  // produce every team's normals a step ahead (warp specialisation: the
  // noise leaves the compute warps' dependency chain).
  const int nc = compute_threads<TPS>(noise_warps);
  const int spb = nc / TPS;
  const bool producer = kNoiseWarps<TPS, BPT> && static_cast<int>(threadIdx.x) >= nc;
  const int team = producer ? 0 : static_cast<int>(threadIdx.x) / TPS;
  const int lt = threadIdx.x % TPS;
  const int s = tile * spb + team;
  const int H = in.H;
  const int n_rows = EXT ? in.n_obs * k.nd : in.n_obs;  // obstacle rows (obstacle x disc)

  if (threadIdx.x == 32) {  // warm the outputs' translations (any CTA may merge)
    prefetch_l2(in.U_out);
    prefetch_l2(in.traj_out);
    prefetch_l2(in.U_next);
    prefetch_l2(in.status);
    prefetch_l2(in.part + static_cast<size_t>(tile - in.tile_base) * in.part_stride);
    if (in.J_out) prefetch_l2(in.J_out + static_cast<size_t>(tile) * spb);
  }
  // --- frame and staging (tables in shared memory, relative coordinates).
  // The raw path, the nominal inputs and each thread's first obstacle are
  // loaded first, so that their global loads overlap warp 0's frame; the
  // shift into the frame follows the barrier.
  const bool obs8 = EXT && k.obs8;
  const int ostride = obs8 ? 8 : 6;
  for (int j = threadIdx.x; j < 3 * in.n_pts; j += blockDim.x) cp_async4(S.path + j, in.path + j);
  for (int j = threadIdx.x; j < 3 * H; j += blockDim.x) cp_async4(S.unom + j, in.U_nom + j);
  float ob0[8];
  const bool has_ob0 = static_cast<int>(threadIdx.x) < in.n_obs;
#pragma unroll
  for (int q = 0; q < 8; ++q) ob0[q] = (has_ob0 && q < ostride) ? in.obs[ostride * threadIdx.x + q] : 0.f;
  if (threadIdx.x < 32) make_frame_warp(in.x0, in.inv_ds_d, in.sync + 1, sh.fr, EXT && k.jerk);
  cp_async_wait_all();
  __syncthreads();
  const Frame& fr = sh.fr;
  auto stage_obstacle = [&](int o, float cx, float cy, float ax, float ay, float th, float e, float vx, float vy) {
    float* d = S.obs + 8 * o;
    const bool e4 = obs8 && e == 4.0f;
    if (e != 2.0f && !e4) atomicOr(in.sync + 1, ERR_EXPONENT);
    const float Ax = ax + k.r_inflate, Ay = ay + k.r_inflate;
    d[0] = (cx - fr.ox_h) - fr.ox_l;
    d[1] = (cy - fr.oy_h) - fr.oy_l;
    float so, co;
    sincosf(th, &so, &co);
    const float ix = 1.0f / (Ax * Ax), iy = 1.0f / (Ay * Ay);
    if constexpr (!EXT) {
      // parked ellipses: h = d^T Q d - 1 with d the offset in world axes and
      // Q = R^T diag(ix, iy) R (R the rotation into the obstacle's axes):
      // (Qxx, Qxy) in place of (cos, sin), Qyy in slot 4
      const float c2 = co * co, s2 = so * so;
      d[2] = fmaf(c2, ix, s2 * iy);
      d[3] = (co * so) * (ix - iy);
      d[4] = fmaf(s2, ix, c2 * iy);
      d[5] = d[6] = d[7] = 0.f;
    } else {
      d[2] = co;
      d[3] = so;
      d[4] = e4 ? -(ix * ix) : ix;
      d[5] = e4 ? iy * iy : iy;
      d[6] = co * vx + so * vy;
      d[7] = co * vy - so * vx;
    }
  };
  if (has_ob0) stage_obstacle(threadIdx.x, ob0[0], ob0[1], ob0[2], ob0[3], ob0[4], ob0[5], ob0[6], ob0[7]);
  for (int o = threadIdx.x + blockDim.x; o < in.n_obs; o += blockDim.x) {
    const float* ob = in.obs + ostride * o;
    stage_obstacle(o, ob[0], ob[1], ob[2], ob[3], ob[4], ob[5], obs8 ? ob[6] : 0.f, obs8 ? ob[7] : 0.f);
  }
  for (int j = threadIdx.x; j < in.n_pts; j += blockDim.x) {
    float* d = S.path + 3 * j;
    d[0] = (d[0] - fr.ox_h) - fr.ox_l;
    d[1] = (d[1] - fr.oy_h) - fr.oy_l;
    const float th = (d[2] - fr.oth_h) - fr.oth_l;
    d[2] = th;
    // the row's heading direction in world axes, once per solve: the stage
    // cost turns it by the interpolation angle instead of a sincos per step
    float st, ct;
    sincosf(th, &st, &ct);
    *reinterpret_cast<float2*>(S.phead + 2 * j) = make_float2(fr.c0 * ct - fr.s0 * st, fr.s0 * ct + fr.c0 * st);
  }
  if constexpr (EXT) {
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (static_cast<int>(threadIdx.x) == m) {
        S.disc[2 * m] = k.disc_e1[m];
        S.disc[2 * m + 1] = k.disc_e2[m];
      }
  }
  __syncthreads();

  // --- per-sample state (relative frame)
  const float c0 = fr.c0, s0 = fr.s0;
  float acc = fr.a0;  // acceleration state of the jerk-input model
  float px = 0.f, pxl = 0.f, py = 0.f, pyl = 0.f, t1 = 0.f, t2 = fr.t2, v = fr.v_h, vl = fr.v_l,
        dl = fr.dl, ps = 0.f, psl = 0.f;
  // obstacle slots per lane: one lane per sample holds every obstacle of
  // its Philox blocks 1.. ; wider teams hold obstacles lt, lt + TPS, ...;
  // ROWS > 0 (latency variants with noise warps): exactly ROWS slots a lane
  static_assert(ROWS == 0 || kNoiseWarps<TPS, BPT>, "exact row slots need the noise-warp variants");
  constexpr int OBS_SLOTS = ROWS > 0 ? ROWS : ((TPS == 1) ? (BPT > 1 ? 4 * (BPT - 1) : 1) : 4 * BPT);
  float alpha_h = k.alpha0;  // the hitch's barrier rate (same on every lane)
  float alpha[OBS_SLOTS];
#pragma unroll
  for (int q = 0; q < OBS_SLOTS; ++q) alpha[q] = k.alpha0;
  float Jh = 0.f, Jl = 0.f;
  float ua = 0.f, uw = 0.f, un = 0.f;  // applied input of the previous step
  const uint32_t sid = static_cast<uint32_t>(s);
  const int n_pts = in.n_pts;
  const float qf0 = fr.qf0;
  const int i0 = fr.i0;

  // the four normals of Philox block b at step tau
  auto draw_block = [&](int b, int tau, float* out) {
    const uint4 w = philox4x32_10(
        make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(tau), sid, in.ctr), in.key0, in.key1);
    box_muller(w.x, w.y, out[0], out[1]);
    box_muller(w.z, w.w, out[2], out[3]);
  };
  // block 0 of this lane (lane 0: the input normals and the hitch), drawn a
  // step ahead; further blocks are drawn where their rows are built
  auto draw_first = [&](int tau, float* out) {
    if (lt < in.P) {
      draw_block(lt, tau, out);
    } else {
      out[0] = out[1] = out[2] = out[3] = 0.f;
    }
  };

  // barrier of constraint row j (obstacle o seen from footprint disc m) at
  // the current state and time t (Eq. barrier_function; moving centres at
  // c + t v); (ce1, se1) and (ce2, se2) the unit headings of the state
  auto row_h = [&](int j, float t, float ce1, float se1, float ce2, float se2) -> float {
    const int o = (k.nd == 1) ? j : __float2int_rz((static_cast<float>(j) + 0.5f) * k.inv_nd);
    const int m = j - o * k.nd;
    const float4 o0 = *reinterpret_cast<const float4*>(S.obs + 8 * o);
    const float4 o1 = *reinterpret_cast<const float4*>(S.obs + 8 * o + 4);
    const float2 lv = *reinterpret_cast<const float2*>(S.disc + 2 * m);
    const float dx = (px - o0.x) + pxl + lv.x * ce1 + lv.y * ce2;
    const float dy = (py - o0.y) + pyl + lv.x * se1 + lv.y * se2;
    const float xp = o0.z * dx + o0.w * dy - t * o1.z;
    const float yp = o0.z * dy - o0.w * dx - t * o1.w;
    const bool e4 = o1.x < 0.f;
    const float kx = fabsf(o1.x), ky = o1.y;
    const float X = e4 ? xp * xp * kx : kx, Y = e4 ? yp * yp * ky : ky;
    return xp * xp * X + yp * yp * Y - 1.f;
  };

  // stage cost of the current state (time t) reached with input (ua, uw, un);
  // add = false computes it and adds zero (no branch in the step)
  auto stage_cost = [&](float t, float ce1, float se1, float ce2, float se2, bool add) {
    const float qf = qf0 + (ps * in.inv_ds + psl * in.inv_ds);
    const float fl = floorf(qf);
    int ii = i0 + static_cast<int>(fl);
    float ff = qf - fl;
    if (ii < 0) {
      ii = 0;
      ff = 0.f;
    } else if (ii > n_pts - 2) {
      ii = n_pts - 2;
      ff = 1.f;
    }
    const float* r0 = S.path + 3 * ii;
    const float xr = r0[0] + ff * (r0[3] - r0[0]);
    const float yr = r0[1] + ff * (r0[4] - r0[1]);
    const float eps = ff * (r0[5] - r0[2]);  // turn from row ii to the interpolated heading
    const float thr = r0[2] + eps;
    const float2 hd = *reinterpret_cast<const float2*>(S.phead + 2 * ii);
    float se, ce;
    turn_sincos(eps, &se, &ce);
    const float cth = hd.x * ce - hd.y * se;  // cos / sin of the heading in world axes
    const float sth = hd.y * ce + hd.x * se;
    const float dxr = (px - xr) + pxl, dyr = (py - yr) + pyl;
    const float ec = sth * dxr - cth * dyr;
    const float el = -cth * dxr - sth * dyr;
    const float e1 = wrap_pi(t1 - thr), e2 = wrap_pi(t2 - thr);
    const float dn = k.nu_bar - un;
    float rc = k.Qc * ec * ec + k.Ql * el * el + k.Qth * (e1 * e1 + e2 * e2) + k.R0 * ua * ua +
               k.R1 * uw * uw + k.R2 * un * un + k.mu * dn * dn;
    if (EXT && k.coll) {
      // the comparison method's collision penalty: depth of every
      // obstacle the state is inside (obstacles spread over the team)
      float c = 0.f;
      for (int j = lt; j < n_rows; j += TPS) c += fmaxf(-row_h(j, t, ce1, se1, ce2, se2), 0.f);
      rc += k.q_coll * team_sum<TPS>(c);
    }
    acc2(Jh, Jl, add ? rc : 0.f);
  };

  // stored-trajectory variant: the state of this sample after step tau, in
  // world coordinates (written by the team's first lane)
  float* st_out = (!producer && in.states_out && lt == 0 && s < in.S)
                      ? in.states_out + static_cast<size_t>(s) * static_cast<size_t>(H + 1) * 7
                      : nullptr;
  auto store_state = [&](int tau) {
    float* o = st_out + 7 * tau;
    o[0] = (fr.ox_h + px) + (fr.ox_l + pxl);
    o[1] = (fr.oy_h + py) + (fr.oy_l + pyl);
    o[2] = (fr.oth_h + t1) + fr.oth_l;
    o[3] = (fr.oth_h + t2) + fr.oth_l;
    o[4] = v + vl;
    o[5] = dl;
    o[6] = (fr.psi_h + ps) + (fr.psi_l + psl);
  };
  if (st_out) store_state(0);
  float* in_out = (!producer && in.inputs_out && lt == 0 && s < in.S)
                      ? in.inputs_out + static_cast<size_t>(s) * static_cast<size_t>(H) * 3
                      : nullptr;

  // Noise.  One lane per sample: the lane draws Philox block 0 a step ahead
  // and the further blocks where their rows are built.  Wider teams: the
  // producer warp writes the P blocks of every team's step tau + 1 into a
  // per-team double buffer in shared memory while the compute warps run step
  // tau; one CTA barrier per step hands the buffers over (at barrier tau the
  // producer has written step tau and the compute warps have finished step
  // tau - 1, whose buffer it fills next).  Constraint i is built by lane
  // i % TPS, so rows spread evenly over the team.
  float* nz = S.noise + team * S.noise_per_team;  // [2][P][4] (wide teams)
  const int P_drawn = k.proj ? in.P : 1;  // standard MPPI needs the input normals only
  // Variants with more than two blocks per lane (many constraints) stage
  // them on the team's own lanes instead (blocks b = lt, lt + TPS, ...): a
  // producer would need more warps than the CTA can hold.
  constexpr bool lane_staged = TPS > 1 && !kNoiseWarps<TPS, BPT>;
  auto stage_step = [&](int tau_d, float* buf) {
    for (int b = lt; b < P_drawn; b += TPS) {
      float t4[4];
      draw_block(b, tau_d, t4);
      *reinterpret_cast<float4*>(buf + 4 * b) = make_float4(t4[0], t4[1], t4[2], t4[3]);
    }
  };
  if constexpr (lane_staged) stage_step(0, nz);
  if constexpr (kNoiseWarps<TPS, BPT>) {
    if (producer) {
      const int pl = static_cast<int>(threadIdx.x) - nc;
      const int n_blocks = spb * P_drawn;
      auto produce = [&](int tau_d) {
        for (int i = pl; i < n_blocks; i += 32 * noise_warps) {
          const int tm = i / P_drawn, b = i - tm * P_drawn;
          const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(tau_d),
                                                   static_cast<uint32_t>(tile * spb + tm), in.ctr),
                                        in.key0, in.key1);
          float4 g;
          box_muller(w.x, w.y, g.x, g.y);
          box_muller(w.z, w.w, g.z, g.w);
          *reinterpret_cast<float4*>(S.noise + tm * S.noise_per_team + (tau_d & 1) * 4 * in.P + 4 * b) = g;
        }
      };
      produce(0);
      for (int tau = 0; tau < H; ++tau) {
        step_barrier();
        if (tau + 1 < H) produce(tau + 1);
      }
    }
  }
  float nrm[4];
  if constexpr (TPS == 1) draw_first(0, nrm);
  // trigonometry of the current state, carried from step to step: the state
  // angles theta1 and phi = theta1 - theta2 of step tau + 1 follow from step
  // tau's state alone (the input enters only the speed, steer angle and
  // progress), so their sin / cos are taken before step tau's projection
  // and stay off its dependency chain; only the steer angle's trigonometry
  // waits for the projection.
  float c1, s1, sp, cp;
  {
    float sr, cr;
    state_sincos(t1, &sr, &cr);
    c1 = c0 * cr - s0 * sr;
    s1 = s0 * cr + c0 * sr;
    state_sincos(t1 - t2, &sp, &cp);
  }
  // One step; PROJ is fixed for the whole loop (no branch on the flag
  // inside the step).
  auto step = [&](int tau, auto proj_c) {
    constexpr bool PROJ = decltype(proj_c)::value;
    float nxt[4];
    float* cur = nz;
    if constexpr (TPS == 1) {
      draw_first(tau + 1 < H ? tau + 1 : tau, nxt);  // off the state's critical path
    } else if constexpr (lane_staged) {
      __syncwarp();  // this step's normals are staged; last step's reads are done
      cur = nz + (tau & 1) * 4 * in.P;
      if (tau + 1 < H) stage_step(tau + 1, nz + ((tau + 1) & 1) * 4 * in.P);
    } else {
      step_barrier();  // this step's normals are staged
      cur = nz + (tau & 1) * 4 * in.P;
    }

    // trigonometry of the steer angle (the one state angle the previous
    // projection moved)
    float sd, cd;
    state_sincos(dl, &sd, &cd);
    const float tn = __fdividef(sd, cd);  // |cos| >= 4e-9 below 2^16: MUFU reciprocal (~2 ulp)
    const float vv = v + vl;
    const float th1dot = vv * tn * k.inv_l1;

    // cost of the previous step, at this state (independent of the rows);
    // at tau = 0 there is no previous step and the increment is zero
    // (adding zero to a compensated pair leaves it unchanged)
    stage_cost(static_cast<float>(tau) * k.Ts, c1, s1, c1 * cp + s1 * sp, s1 * cp - c1 * sp, tau > 0);

    // explicit Euler, the state-only part (right-hand sides at the current
    // state), and the next state's theta1 / phi trigonometry.  Latency
    // shapes (teams) form it before the projection, off its dependency
    // chain; one-lane shapes (issue-bound, many warps) after it, so that the
    // current and next values need not be live at once (no register copies
    // at the end of the step)
    const float Tv = k.Ts * vv;
    float px_n, pxl_n, py_n, pyl_n, t1_n, t2_n, c1_n, s1_n, sp_n, cp_n;
    auto state_part = [&]() {
      px_n = px;
      pxl_n = pxl;
      py_n = py;
      pyl_n = pyl;
      acc2(px_n, pxl_n, Tv * c1);
      acc2(py_n, pyl_n, Tv * s1);
      t1_n = t1 + k.Ts * th1dot;
      t2_n = t2 + Tv * k.inv_l2 * (sp - k.k_hitch * cp * tn);
      if constexpr (TPS > 1) {
        // even lanes take theta1, odd lanes phi, and each pair trades the
        // results: one sin / cos sequence in the warp's stream instead of two
        const bool odd = lt & 1;
        float sa, ca;
        state_sincos(odd ? t1_n - t2_n : t1_n, &sa, &ca);
        const float sb = __shfl_xor_sync(0xffffffffu, sa, 1);
        const float cb = __shfl_xor_sync(0xffffffffu, ca, 1);
        const float sr = odd ? sb : sa, cr = odd ? cb : ca;
        sp_n = odd ? sa : sb;
        cp_n = odd ? ca : cb;
        c1_n = c0 * cr - s0 * sr;
        s1_n = s0 * cr + c0 * sr;
      } else {
        float sr, cr;
        state_sincos(t1_n, &sr, &cr);
        c1_n = c0 * cr - s0 * sr;
        s1_n = s0 * cr + c0 * sr;
        state_sincos(t1_n - t2_n, &sp_n, &cp_n);
      }
    };
    if constexpr (TPS > 1) state_part();

    float na, nw, nn;
    if constexpr (TPS == 1) {
      na = nrm[0];
      nw = nrm[1];
      nn = nrm[2];
    } else {
      na = cur[0];
      nw = cur[1];
      nn = cur[2];
    }
    const float zd0 = clampf(S.unom[3 * tau + 0] + k.sig0 * na, k.zlo0, k.zhi0);
    const float zd1 = clampf(S.unom[3 * tau + 1] + k.sig1 * nw, k.zlo1, k.zhi1);
    const float zd2 = clampf(S.unom[3 * tau + 2] + k.sig2 * nn, k.zlo2, k.zhi2);

    float za, zw, zn;
    if constexpr (PROJ) {
      const float pu0 = k.w_u0 * zd0 + k.pc_u0;
      const float pu1 = k.w_u1 * zd1 + k.pc_u1;
      const float pu2 = k.w_u2 * zd2 + k.pc_u2;
      const float q0 = pu0 * k.inv_m_u0, q1 = pu1 * k.inv_m_u1;  // M_u^-1 p_u
      // hitch row: every lane of the team computes it (same state, same
      // normal); its terms enter the team sums once (lane 0)
      float Saa, Saw, Sww, ga, gw, ca_h, cw_h, cc_h;
      {
        const float n_h = (TPS == 1) ? nrm[3] : cur[3];
        HitchRow hr = hitch_row(k, t2 - t1, sp, cp, tn, vv, th1dot);
        if (EXT && k.jerk) {  // a is a state: its terms join the constant; the jerk enters via -kappa
          hr.c0 += acc * hr.Aa;
          hr.Aa = -k.hTs2 * k.kappa;
        }
        const float hm = fmaxf(fabsf(hr.h), k.h_floor);
        const float ht = copysignf(hm, hr.h);  // h's sign (h = -0 does not arise: an exact zero rounds to +0)
        const float zda = clampf(k.sigma_alpha * n_h, k.ua_lo, k.ua_hi);
        const float pam = k.w_am * zda + k.pc_am;  // p_alpha / m_alpha
        const float b = -alpha_h * hr.h - hr.c0;
        const float r = hr.Aa * q0 + hr.Aw * q1 + ht * pam - b;
        const float iht = __fdividef(1.f, ht);  // MUFU reciprocal (~1 ulp)
        const float rho = r * iht;
        ca_h = hr.Aa * iht;
        cw_h = hr.Aw * iht;
        cc_h = pam - rho;
        const float own = (lt == 0) ? 1.f : 0.f;  // the sums take the row once (lane 0)
        const float ua_ = own * ca_h;
        Saa = ua_ * ua_;
        ga = ua_ * rho;
        if constexpr (EXT) {
          const float uw_ = own * cw_h;
          Saw = ua_ * uw_;
          Sww = uw_ * uw_;
          gw = uw_ * rho;
        } else {
          // the plain family's ellipse rows have no steer-rate column: these
          // sums hold the hitch row's terms alone, the same on every lane of
          // the team (no team reduction; the values it would give)
          Saw = ca_h * cw_h;
          Sww = cw_h * cw_h;
          gw = cw_h * rho;
        }
      }

      // obstacle rows; the steer rate does not enter at second order.  Parked ellipses (e = 2): hdot shares dh/da's
      // direction term.  Moving or e = 4 rows (uniform branch): barrier of
      // the relative position at this step's time, relative velocity.
      // `live` = 0 turns a padding slot into a no-op without branching.
      float ca[OBS_SLOTS], cc[OBS_SLOTS];
      float cw[EXT ? OBS_SLOTS : 1];  // steer-rate column (footprint discs off the rear axle)
      // every slot that the alpha update reads is written below (padding
      // rows as zeros)
      const float tnow = static_cast<float>(tau) * k.Ts;
      float cbuf = 0.f;  // buffer cost of this lane's rows
      // heading rates and accelerations of the bodies (footprint discs):
      // th2 = th1 - phi; heading accelerations with the input held,
      // th1ddot = a1a a + a1w omega, th2ddot = a20 + a2a a + a2w omega
      float c2 = 0.f, s2 = 0.f, th2dot = 0.f, a1a = 0.f, a1w = 0.f, a20 = 0.f, a2a = 0.f, a2w = 0.f;
      if (EXT && k.discs) {
        c2 = c1 * cp + s1 * sp;
        s2 = s1 * cp - c1 * sp;
        const float G = sp - k.k_hitch * cp * tn;
        const float sec2 = 1.f + tn * tn;
        th2dot = vv * G * k.inv_l2;
        a1a = tn * k.inv_l1;
        a1w = vv * sec2 * k.inv_l1;
        a2a = G * k.inv_l2;
        a2w = -vv * k.k_hitch * cp * sec2 * k.inv_l2;
        a20 = vv * k.inv_l2 * (cp + k.k_hitch * tn * sp) * (th1dot - th2dot);
      }
      // per-step factors of the parked-ellipse rows (their rest term, below)
      const float cg_row = -2.f * k.Ts * vv, vth_row = -k.Ts2 * vv * th1dot, vq_row = -k.Ts2 * vv * vv;
      const float qxx_row = vq_row * c1 * c1, qyy_row = vq_row * s1 * s1, qxy_row = 2.f * vq_row * c1 * s1;
      auto obstacle_row = [&](int j, float n_alpha, int slot, float live) {
        float h, Aa, Aw = 0.f, brest;
        if constexpr (!EXT) {
          // staged as (cx, cy, Qxx, Qxy, Qyy): h = d^T Q d - 1 in world axes
          const float4 o0 = *reinterpret_cast<const float4*>(S.obs + 8 * j);
          const float qyy = S.obs[8 * j + 4];
          const float dx = (px - o0.x) + pxl, dy = (py - o0.y) + pyl;
          // with (gx, gy) = grad h / 2 = Q d and the heading e1 = (c1, s1):
          // h = d . (gx, gy) - 1; hdot = 2 v g, g = grad h . e1 / 2;
          // hddot (input part aside) = 2 v th1dot turn + 2 v^2 curv, turn =
          // grad h . n1 / 2, curv = e1^T (Hess h / 2) e1 = e1^T Q e1; so the
          // row's a-column Ts^2/2 dh/da = Ts^2 g and its rest
          // -(Ts hdot + Ts^2/2 hddot0) = -2 Ts v g - Ts^2 (v th1dot turn + v^2 curv)
          const float gx = fmaf(o0.z, dx, o0.w * dy), gy = fmaf(o0.w, dx, qyy * dy);
          h = fmaf(gx, dx, fmaf(gy, dy, -1.f));
          const float g = fmaf(gx, c1, gy * s1);
          const float turn = fmaf(gy, c1, -(gx * s1));
          Aa = k.Ts2 * g;
          brest = fmaf(cg_row, g, fmaf(vth_row, turn, fmaf(qxx_row, o0.z, fmaf(qxy_row, o0.w, qyy_row * qyy))));
        } else {
          // row j: obstacle o seen from footprint disc m (obstacle-major)
          const int o = (k.nd == 1) ? j : __float2int_rz((static_cast<float>(j) + 0.5f) * k.inv_nd);
          const int m = j - o * k.nd;
          const float4 o0 = *reinterpret_cast<const float4*>(S.obs + 8 * o);
          const float4 o1 = *reinterpret_cast<const float4*>(S.obs + 8 * o + 4);
          const float2 lv = *reinterpret_cast<const float2*>(S.disc + 2 * m);  // lever arms on e1, e2
          const float co = o0.z, so = o0.w;
          // unit headings in the obstacle frame: e1' = (dirx, diry),
          // n1' = (-diry, dirx), e2' = (d2x, d2y), n2' = (-d2y, d2x)
          const float dirx = co * c1 + so * s1, diry = co * s1 - so * c1;
          const float d2x = co * c2 + so * s2, d2y = co * s2 - so * c2;
          const float dx = (px - o0.x) + pxl, dy = (py - o0.y) + pyl;
          // disc centre relative to the (moving) obstacle centre at tnow;
          // e = 4 flagged by a negated kx; X = xp^(e-2) / Ax^e:
          // h = xp^2 X + ..., h_x = e xp X, h_xx = e (e-1) X
          const float xp = co * dx + so * dy + lv.x * dirx + lv.y * d2x - tnow * o1.z;
          const float yp = co * dy - so * dx + lv.x * diry + lv.y * d2y - tnow * o1.w;
          const bool e4 = o1.x < 0.f;
          const float kx = fabsf(o1.x), ky = o1.y;
          const float X = e4 ? xp * xp * kx : kx, Y = e4 ? yp * yp * ky : ky;
          const float ce = e4 ? 4.f : 2.f, cee = e4 ? 12.f : 2.f;
          h = xp * xp * X + yp * yp * Y - 1.f;
          const float hx = ce * xp * X, hy = ce * yp * Y;
          // disc velocity relative to the obstacle
          const float velx = vv * dirx - lv.x * th1dot * diry - lv.y * th2dot * d2y - o1.z;
          const float vely = vv * diry + lv.x * th1dot * dirx + lv.y * th2dot * d2x - o1.w;
          // disc acceleration = acc0 + a acc_a + omega acc_w
          const float aax = dirx - lv.x * a1a * diry - lv.y * a2a * d2y;
          const float aay = diry + lv.x * a1a * dirx + lv.y * a2a * d2x;
          const float awx = -lv.x * a1w * diry - lv.y * a2w * d2y;
          const float awy = lv.x * a1w * dirx + lv.y * a2w * d2x;
          const float t1q = th1dot * th1dot, t2q = th2dot * th2dot;
          const float a0x = -vv * th1dot * diry - lv.x * t1q * dirx - lv.y * (a20 * d2y + t2q * d2x);
          const float a0y = vv * th1dot * dirx - lv.x * t1q * diry + lv.y * (a20 * d2x - t2q * d2y);
          const float hdot = hx * velx + hy * vely;
          const float hdd0 = hx * a0x + hy * a0y + cee * (X * velx * velx + Y * vely * vely);
          Aa = k.hTs2 * (hx * aax + hy * aay);
          Aw = k.hTs2 * (hx * awx + hy * awy);
          brest = -k.Ts * hdot - k.hTs2 * hdd0;
          if (k.third) {
            // Ts^3/6 hdddot at the rear axle (lever arms zero), affine in
            // (a, omega): pdddot = 2 a th1dot n1 + v th1ddot n1 - v th1dot^2 e1,
            // hdddot = grad h . pdddot + 3 w^T Hess h pddot + D3 h [w, w, w]
            const float gn = hy * dirx - hx * diry;  // grad h . n1'
            const float hxxx = e4 ? 24.f * xp * kx : 0.f, hyyy = e4 ? 24.f * yp * ky : 0.f;
            const float wHx = cee * X * velx, wHy = cee * Y * vely;  // Hess h w
            const float ca3 = (2.f * th1dot + vv * tn * k.inv_l1) * gn + 3.f * (wHx * dirx + wHy * diry);
            const float cw3 = vv * vv * (1.f + tn * tn) * k.inv_l1 * gn;
            const float c03 = -vv * th1dot * th1dot * gda3(hx, hy, dirx, diry) +
                              3.f * vv * th1dot * (wHy * dirx - wHx * diry) +
                              hxxx * velx * velx * velx + hyyy * vely * vely * vely;
            Aa += k.Ts3_6 * ca3;
            Aw += k.Ts3_6 * cw3;
            brest -= k.Ts3_6 * c03;
          }
          if (k.jerk) {
            // a is a state (rear-axle point): its terms join the constant;
            // the jerk enters only at third order, through grad h . e1'
            brest -= acc * Aa;
            Aa = k.third ? k.Ts3_6 * gda3(hx, hy, dirx, diry) : 0.f;
          }
        }
        const float hm = fmaxf(fabsf(h), k.h_floor);
        const float ht = copysignf(hm, h);
        const float zda = clampf(k.sigma_alpha * n_alpha, k.ua_lo, k.ua_hi);
        const float pam = k.w_am * zda + k.pc_am;  // p_alpha / m_alpha
        const float b = -alpha[slot] * h + brest;
        float r = fmaf(Aa, q0, fmaf(ht, pam, -b));
        if constexpr (EXT) r = fmaf(Aw, q1, r);
        // MUFU reciprocal (~1 ulp); a padding slot (live = 0) gets 0: its
        // u, w and rho vanish, so it adds nothing to the sums (its own rate
        // drifts by p_alpha a step and is never read by a live row)
        const float iht = live * __fdividef(1.f, ht);
        const float u = Aa * iht;
        const float rho = r * iht;
        Saa += u * u;
        ga += u * rho;
        ca[slot] = u;
        cc[slot] = pam - rho;
        if constexpr (EXT) {
          const float w = Aw * iht;
          Saw += u * w;
          Sww += w * w;
          gw += w * rho;
          cw[slot] = w;
        }
        if (EXT && k.abuf) {
          // buffer zone: positive rates charged with weight clip(1 - h/h_buf)
          const float wz = clampf(1.f - h * k.inv_hbuf, 0.f, 1.f);
          const float ap = fmaxf(alpha[slot], 0.f);
          cbuf += live * (k.q_abuf * wz * ap * ap);
        }
      };

      if constexpr (TPS == 1) {
        // row j uses normal 4 + j: block 1 + j/4, drawn here
#pragma unroll
        for (int b8 = 1; b8 < BPT; ++b8) {
          if (b8 < in.P) {
            float nb[4];
            draw_block(b8, tau, nb);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int j = 4 * (b8 - 1) + m;
              ca[j] = 0.f;
              cc[j] = 0.f;
              if constexpr (EXT) cw[j] = 0.f;
              if (j < n_rows) obstacle_row(j, nb[m], j, 1.f);
            }
          }
        }
      } else if constexpr (ROWS > 0) {
        // exactly ROWS row slots a lane (row j on lane j % TPS): every slot
        // runs, padding rows masked by `live`; no branch in the step
#pragma unroll
        for (int slot = 0; slot < ROWS; ++slot) {
          const int j = lt + TPS * slot;
          const bool live = j < n_rows;
          const int jj = live ? j : 0;
          obstacle_row(jj, cur[4 + jj], slot, live ? 1.f : 0.f);
        }
      } else {
        // row j on lane j % TPS; every lane runs the team's slot count
        const int per_lane = (n_rows + TPS - 1) / TPS;
#pragma unroll
        for (int slot = 0; slot < OBS_SLOTS; ++slot) {
          ca[slot] = 0.f;
          cc[slot] = 0.f;
          if constexpr (EXT) cw[slot] = 0.f;
          if (slot < per_lane) {
            const int j = lt + TPS * slot;
            const bool live = j < n_rows;
            const int jj = live ? j : 0;
            obstacle_row(jj, cur[4 + jj], slot, live ? 1.f : 0.f);
          }
        }
      }
      if (EXT && k.abuf) acc2(Jh, Jl, team_sum<TPS>(cbuf));
      Saa = k.m_a * team_sum<TPS>(Saa) + k.m_u0;
      ga = k.m_a * team_sum<TPS>(ga);
      if constexpr (EXT) {
        Saw = k.m_a * team_sum<TPS>(Saw);
        Sww = k.m_a * team_sum<TPS>(Sww) + k.m_u1;
        gw = k.m_a * team_sum<TPS>(gw);
      } else {
        Saw = k.m_a * Saw;
        Sww = k.m_a * Sww + k.m_u1;
        gw = k.m_a * gw;
      }
      const float idet = __fdividef(1.f, Saa * Sww - Saw * Saw);  // SPD: det > 0
      const float ya = (Sww * ga - Saw * gw) * idet;
      const float yw = (Saa * gw - Saw * ga) * idet;
      za = q0 - ya;
      zw = q1 - yw;
      zn = pu2 * k.inv_m_u2;
      alpha_h += cc_h + ca_h * ya + cw_h * yw;
      auto alpha_update = [&](int slot) {
        if constexpr (EXT) {
          alpha[slot] += cc[slot] + ca[slot] * ya + cw[slot] * yw;
        } else {
          alpha[slot] += cc[slot] + ca[slot] * ya;
        }
      };
      if constexpr (TPS == 1) {
        // the blocks this instance draws (a uniform branch per block): rows
        // of the blocks beyond it are never read
#pragma unroll
        for (int b8 = 1; b8 < BPT; ++b8)
          if (b8 < in.P) {
#pragma unroll
            for (int m = 0; m < 4; ++m) alpha_update(4 * (b8 - 1) + m);
          }
      } else {
#pragma unroll
        for (int slot = 0; slot < OBS_SLOTS; ++slot) alpha_update(slot);
      }
    } else {
      za = zd0;
      zw = zd1;
      zn = zd2;
    }
    ua = clampf(za, k.zlo0, k.zhi0);
    uw = clampf(zw, k.zlo1, k.zhi1);
    un = clampf(zn, k.zlo2, k.zhi2);
    if constexpr (TPS == 1) state_part();

    // explicit Euler, the input-driven part; the state-only part was formed
    // from the same right-hand sides
    px = px_n;
    pxl = pxl_n;
    py = py_n;
    pyl = pyl_n;
    t1 = t1_n;
    t2 = t2_n;
    if (EXT && k.jerk) {  // input 0 is the jerk; the acceleration state drives the speed
      acc2(v, vl, k.Ts * acc);
      acc += k.Ts * ua;
    } else {
      acc2(v, vl, k.Ts * ua);
    }
    dl += k.Ts * uw;
    acc2(ps, psl, k.Ts * un);
    c1 = c1_n;
    s1 = s1_n;
    sp = sp_n;
    cp = cp_n;

    if (lt == 0) {
      uh[(3 * tau + 0) * spb + team] = ua;
      uh[(3 * tau + 1) * spb + team] = uw;
      uh[(3 * tau + 2) * spb + team] = un;
    }
    if (st_out) store_state(tau + 1);
    if (in_out) {
      in_out[3 * tau + 0] = ua;
      in_out[3 * tau + 1] = uw;
      in_out[3 * tau + 2] = un;
    }
    if constexpr (TPS == 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) nrm[q] = nxt[q];
    }
  };
  if (!producer) {
    if (k.proj) {
      for (int tau = 0; tau < H; ++tau) step(tau, std::true_type{});
    } else {
      for (int tau = 0; tau < H; ++tau) step(tau, std::false_type{});
    }
  }
  if (!producer) {  // cost of the last step
    float ce1 = 0.f, se1 = 0.f, ce2 = 0.f, se2 = 0.f;
    if (EXT && k.coll && k.discs) {
      float sr, cr, sq, cq;
      sincosf(t1, &sr, &cr);
      sincosf(t1 - t2, &sq, &cq);
      ce1 = c0 * cr - s0 * sr;
      se1 = s0 * cr + c0 * sr;
      ce2 = ce1 * cq + se1 * sq;
      se2 = se1 * cq - ce1 * sq;
    }
    stage_cost(static_cast<float>(H) * k.Ts, ce1, se1, ce2, se2, true);
  }

  // --- per-sample cost: normalise the pair
  {
    const float sum = Jh + Jl;
    Jl = Jl - (sum - Jh);
    Jh = sum;
  }
  const bool valid = s < in.S;
  if (!producer && lt == 0) {
    const bool fin = valid && isfinite(Jh) && isfinite(Jl);
    S.jh[team] = fin ? Jh : CUDART_INF_F;
    S.jl[team] = fin ? Jl : 0.f;
    if (valid && in.J_out) in.J_out[s] = Jh;  // the normalised pair's high part
    if (valid && in.J_lo_out) in.J_lo_out[s] = Jl;
  }
  __syncthreads();

  // --- tile softmin partial: min pair, weights, weight sum, weighted inputs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    float mh = CUDART_INF_F, ml = 0.f;
    for (int t = lane; t < spb; t += 32) {
      const float h = S.jh[t], l = S.jl[t];
      if (pair_less(h, l, mh, ml)) { mh = h; ml = l; }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
      const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
      if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
    }
    if (lane == 0) { sh.red_h[0] = mh; sh.red_l[0] = ml; }
  }
  __syncthreads();
  const float bmh = sh.red_h[0], bml = sh.red_l[0];
  const bool any_finite = bmh < CUDART_INF_F;
  for (int t = threadIdx.x; t < spb; t += blockDim.x) {
    const float h = S.jh[t];
    float w = 0.f;
    if (any_finite && h < CUDART_INF_F) w = expf(-((h - bmh) + (S.jl[t] - bml)) * k.inv_lambda);
    S.w[t] = w;
  }
  __syncthreads();
  float* part = in.part + static_cast<size_t>(tile - in.tile_base) * in.part_stride;
  const int nrows = 3 * H + 1;  // row 3H: the weight sum
  // one thread per row: its spb weighted inputs in sample order, four
  // chains (samples t mod 4) combined in a fixed order; the row's loads are
  // issued together (one L2 round trip per row instead of one per warp pass)
  const bool vec = (spb & 3) == 0 && (reinterpret_cast<uintptr_t>(uh) & 15) == 0;
  for (int row = threadIdx.x; row < nrows; row += blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float* src = uh + static_cast<size_t>(row) * spb;
    const bool wsum = row == 3 * H;
    int t = 0;
    if (vec) {
#pragma unroll 8
      for (; t < spb; t += 4) {
        const float4 w4 = *reinterpret_cast<const float4*>(S.w + t);
        const float4 v4 = wsum ? make_float4(1.f, 1.f, 1.f, 1.f) : *reinterpret_cast<const float4*>(src + t);
        a0 += w4.x * v4.x;
        a1 += w4.y * v4.y;
        a2 += w4.z * v4.z;
        a3 += w4.w * v4.w;
      }
    }
    for (; t < spb; ++t) a0 += S.w[t] * (wsum ? 1.f : src[t]);
    part[3 + row] = (a0 + a1) + (a2 + a3);
  }
  if (threadIdx.x == 0) {
    part[0] = bmh;
    part[1] = bml;
    part[2] = 0.f;
  }
}

// Exclusive prefix sum over the 32 lanes of a warp (lane order), offset by
// `carry`; `carry` advances by the warp's total (chunked scans).
static __device__ __forceinline__ float warp_exclusive_scan(float x, float& carry) {
  const int lane = threadIdx.x & 31;
  float s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  const float total = __shfl_sync(0xffffffffu, s, 31);
  float e = __shfl_up_sync(0xffffffffu, s, 1);
  if (lane == 0) e = 0.f;
  const float r = carry + e;
  carry += total;
  return r;
}

// --------------------------------------- merge of an instance's partials
// Run by the CTA that finished the instance's last tile: global minimum
// pair, rescaled sums in tile order, U*, warm start, status and the optimal
// trajectory (x0 integrated with U*).
// Optimal trajectory: x0 integrated with U* in the relative frame (explicit
// Euler, as the rollouts).  Speed, steer angle, progress, the acceleration
// of the jerk-input model and the tractor heading are prefix sums, scanned
// by warp 0 32 steps at a time; the trailer angle is the one nonlinear
// recurrence (thread 0, serial) while warp 1 scans the positions.  Per-step
// values go to `scratch` (8 (H+1) floats: the CTA's table regions when they
// can hold them, else the instance's consumed tile partials).  The
// elementary functions are the SFU approximations (absolute error ~2^-21
// per call, far inside the trajectory tolerance).
static __device__ void optimal_trajectory(const KConst& k, const Inst& in, const Smem& S, Shared& sh,
                                          float* __restrict__ scratch) {
  const int H = in.H, n = H + 1;
  const Frame& fr = sh.fr;
  float* V = scratch;          // speed
  float* D = scratch + n;      // steer angle
  float* Q = scratch + 2 * n;  // progress
  float* T = scratch + 3 * n;  // tan(steer angle)
  float* A = scratch + 4 * n;  // tractor heading
  float* B = scratch + 5 * n;  // trailer heading
  float* X = scratch + 6 * n;  // x
  float* Y = scratch + 7 * n;  // y
  const float* __restrict__ ustar = S.ustar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float Ts = k.Ts;
  __syncthreads();
  if (warp == 0) {
    float cv = fr.v_h + fr.v_l, cd = fr.dl, cq = 0.f, ca = fr.a0, c1 = 0.f;
    for (int base = 0; base < n; base += 32) {
      const int tau = base + lane;
      const bool step = tau < H;  // an input acts at tau < H; states run to H
      const float u0 = step ? ustar[3 * tau + 0] : 0.f;
      const float u1 = step ? ustar[3 * tau + 1] : 0.f;
      const float u2 = step ? ustar[3 * tau + 2] : 0.f;
      float iv = Ts * u0;
      if (k.jerk) {  // the speed integrates the acceleration state
        const float acc = warp_exclusive_scan(Ts * u0, ca);
        iv = step ? Ts * acc : 0.f;
      }
      const float v = warp_exclusive_scan(iv, cv);
      const float d = warp_exclusive_scan(Ts * u1, cd);
      const float q = warp_exclusive_scan(Ts * u2, cq);
      float sd, cs;
      __sincosf(d, &sd, &cs);
      const float t = __fdividef(sd, cs);
      const float a = warp_exclusive_scan(step ? (Ts * v) * t * k.inv_l1 : 0.f, c1);
      if (tau < n) {
        V[tau] = v;
        D[tau] = d;
        Q[tau] = q;
        T[tau] = t;
        A[tau] = a;
      }
    }
  }
  __syncthreads();
  const float c0 = fr.c0, s0 = fr.s0;
  auto positions = [&]() {  // one warp
    float cx = 0.f, cy = 0.f;
    for (int base = 0; base < n; base += 32) {
      const int tau = base + lane;
      float ix = 0.f, iy = 0.f;
      if (tau < H) {
        float a1, b1;
        __sincosf(A[tau], &a1, &b1);
        const float Tv = Ts * V[tau];
        ix = Tv * (c0 * b1 - s0 * a1);
        iy = Tv * (s0 * b1 + c0 * a1);
      }
      const float x = warp_exclusive_scan(ix, cx);
      const float y = warp_exclusive_scan(iy, cy);
      if (tau < n) {
        X[tau] = x;
        Y[tau] = y;
      }
    }
  };
  if (threadIdx.x == 0) {  // trailer angle
    // step tau + 1's coefficients are loaded before step tau's store, so
    // the loads overlap the chain (A, V, T and B share one scratch array)
    float q2 = fr.t2;
    float an = A[0], cn = (Ts * V[0]) * k.inv_l2, en = k.k_hitch * T[0];
    for (int tau = 0; tau < H; ++tau) {
      const float a = an, c = cn, e = en;
      if (tau + 1 < H) {
        an = A[tau + 1];
        cn = (Ts * V[tau + 1]) * k.inv_l2;
        en = k.k_hitch * T[tau + 1];
      }
      B[tau] = q2;
      float a2, b2;
      __sincosf(a - q2, &a2, &b2);
      q2 = fmaf(c, fmaf(-e, b2, a2), q2);
    }
    B[H] = q2;
  }
  if (warp == 1) positions();
  __syncthreads();
  if (blockDim.x < 64 && warp == 0) {  // no second warp: positions after the headings
    positions();
    __syncwarp();
  }
  float* tr = in.traj_out;
  for (int tau = threadIdx.x; tau <= H; tau += blockDim.x) {
    tr[7 * tau + 0] = (fr.ox_h + X[tau]) + fr.ox_l;
    tr[7 * tau + 1] = (fr.oy_h + Y[tau]) + fr.oy_l;
    tr[7 * tau + 2] = (fr.oth_h + A[tau]) + fr.oth_l;
    tr[7 * tau + 3] = (fr.oth_h + B[tau]) + fr.oth_l;
    tr[7 * tau + 4] = V[tau];
    tr[7 * tau + 5] = D[tau];
    tr[7 * tau + 6] = (fr.psi_h + Q[tau]) + fr.psi_l;
  }
}

// The same, one thread, no scratch (when neither scratch region can hold
// 8 (H+1) floats).
static __device__ void serial_trajectory(const KConst& k, const Inst& in, const Smem& S, Shared& sh) {
  const Frame& fr = sh.fr;
  const float c0 = fr.c0, s0 = fr.s0;
  const float* ustar = S.ustar;
  const int H = in.H;
  float qx = 0.f, qy = 0.f, q1 = 0.f, q2 = fr.t2, qv = fr.v_h + fr.v_l, qd = fr.dl, qp = 0.f, qa = fr.a0;
  float* tr = in.traj_out;
  for (int tau = 0; tau <= H; ++tau) {
    tr[7 * tau + 0] = (fr.ox_h + qx) + fr.ox_l;
    tr[7 * tau + 1] = (fr.oy_h + qy) + fr.oy_l;
    tr[7 * tau + 2] = (fr.oth_h + q1) + fr.oth_l;
    tr[7 * tau + 3] = (fr.oth_h + q2) + fr.oth_l;
    tr[7 * tau + 4] = qv;
    tr[7 * tau + 5] = qd;
    tr[7 * tau + 6] = (fr.psi_h + qp) + fr.psi_l;
    if (tau == H) break;
    float a1, b1, a2, b2, ad, bd;
    __sincosf(q1, &a1, &b1);
    __sincosf(q1 - q2, &a2, &b2);
    __sincosf(qd, &ad, &bd);
    const float tq = __fdividef(ad, bd);
    const float Tv = k.Ts * qv;
    qx += Tv * (c0 * b1 - s0 * a1);
    qy += Tv * (s0 * b1 + c0 * a1);
    q2 += Tv * k.inv_l2 * (a2 - k.k_hitch * b2 * tq);
    q1 += Tv * tq * k.inv_l1;
    if (k.jerk) {
      qv += k.Ts * qa;
      qa += k.Ts * ustar[3 * tau + 0];
    } else {
      qv += k.Ts * ustar[3 * tau + 0];
    }
    qd += k.Ts * ustar[3 * tau + 1];
    qp += k.Ts * ustar[3 * tau + 2];
  }
}

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg).
__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gmem_src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

// Minimum pair over the partials of an instance held in shared memory
// (tile b at mp + b * stride), into sh.red_h[1] / sh.red_l[1].
static __device__ void smem_pair_min(const float* mp, int nb, int stride, Shared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  float mh = CUDART_INF_F, ml = 0.f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const float h = mp[static_cast<size_t>(b) * stride + 0], l = mp[static_cast<size_t>(b) * stride + 1];
    if (pair_less(h, l, mh, ml)) { mh = h; ml = l; }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
    const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
    if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
  }
  if (lane == 0) { sh.wred_h[warp] = mh; sh.wred_l[warp] = ml; }
  __syncthreads();
  if (warp == 0) {
    mh = lane < nwarps ? sh.wred_h[lane] : CUDART_INF_F;
    ml = lane < nwarps ? sh.wred_l[lane] : 0.f;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
      const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
      if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
    }
    if (lane == 0) { sh.red_h[1] = mh; sh.red_l[1] = ml; }
  }
  __syncthreads();
}

// SMEM_PARTS: the instance's tile partials are copied into the CTA's shared
// memory at once (one L2 round trip; the launch reserved the room) and
// merged from there; else they are read from L2 in passes.  Both sum each
// row in the same order (four chains, tiles t mod 4, the tail on the first),
// so they give the same bits.
template <bool SMEM_PARTS>
static __device__ void merge_instance(const KConst& k, const Inst& in, const Smem& S, Shared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int nb = in.tiles;
  const int stride = in.part_stride;
  const int H = in.H;
  const int nrows = 3 * H + 1;
  float* ustar = S.ustar;
  bool ok;
  if constexpr (SMEM_PARTS) {
    // the partials region (nb * stride floats, a multiple of 4, 16-byte
    // aligned) into the regions after the disc table (noise, history: no
    // longer read); the error bits' atomic round trip overlaps the copy
    float* mp = S.noise;
    const int nf = nb * stride;
    for (int i = 4 * static_cast<int>(threadIdx.x); i < nf; i += 4 * static_cast<int>(blockDim.x))
      cp_async16(mp + i, in.part + i);
    if (threadIdx.x == 0) sh.err = atomicAdd(in.sync + 1, 0u);
    cp_async_wait_all();
    __syncthreads();
    smem_pair_min(mp, nb, stride, sh);
    const float gmh = sh.red_h[1], gml = sh.red_l[1];
    ok = gmh < CUDART_INF_F;
    for (int q = threadIdx.x; q < nrows; q += blockDim.x) ustar[q] = 0.f;
    for (int b0 = 0; b0 < nb; b0 += 256) {
      __syncthreads();
      for (int t = threadIdx.x; t < 256 && b0 + t < nb; t += blockDim.x) {
        const float* pt = mp + static_cast<size_t>(b0 + t) * stride;
        const float h = pt[0], l = pt[1];
        S.chunk[t] = (ok && h < CUDART_INF_F) ? expf(-((h - gmh) + (l - gml)) * k.inv_lambda) : 0.f;
      }
      __syncthreads();
      const int bend = min(256, nb - b0);
      for (int q = threadIdx.x; q < nrows; q += blockDim.x) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float* col = mp + static_cast<size_t>(b0) * stride + 3 + q;
        int t = 0;
        for (; t + 4 <= bend; t += 4) {
          a0 += S.chunk[t + 0] * col[static_cast<size_t>(t + 0) * stride];
          a1 += S.chunk[t + 1] * col[static_cast<size_t>(t + 1) * stride];
          a2 += S.chunk[t + 2] * col[static_cast<size_t>(t + 2) * stride];
          a3 += S.chunk[t + 3] * col[static_cast<size_t>(t + 3) * stride];
        }
        for (; t < bend; ++t) a0 += S.chunk[t] * col[static_cast<size_t>(t) * stride];
        ustar[q] += (a0 + a1) + (a2 + a3);
      }
    }
  } else {
    // global pair minimum: every thread its tiles (b = tid, tid + blockDim,
    // ...), then warps, then warp 0; the pair of tile tid stays in registers
    // for the weights below (one L2 round trip for both)
    float h0 = CUDART_INF_F, l0 = 0.f;
    // the solve's error bits, read now (an atomic round trip) and used after the sums
    if (threadIdx.x == 0) sh.err = atomicAdd(in.sync + 1, 0u);
    // the first 64 tiles' entries of this thread's first row, loaded now: their
    // round trip overlaps the minimum's (instances of at least 64 tiles)
    const bool pre_ok = static_cast<int>(threadIdx.x) < nrows && nb >= 64;
    float pre[64];
#pragma unroll
    for (int m = 0; m < 64; ++m)
      pre[m] = pre_ok ? __ldcg(in.part + static_cast<size_t>(m) * stride + 3 + threadIdx.x) : 0.f;
    {
      float mh = CUDART_INF_F, ml = 0.f;
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const float h = __ldcg(in.part + static_cast<size_t>(b) * stride + 0);
        const float l = __ldcg(in.part + static_cast<size_t>(b) * stride + 1);
        if (b == static_cast<int>(threadIdx.x)) {
          h0 = h;
          l0 = l;
        }
        if (pair_less(h, l, mh, ml)) { mh = h; ml = l; }
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
        const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
        if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
      }
      if (lane == 0) { sh.wred_h[warp] = mh; sh.wred_l[warp] = ml; }
      __syncthreads();
      if (warp == 0) {
        mh = lane < nwarps ? sh.wred_h[lane] : CUDART_INF_F;
        ml = lane < nwarps ? sh.wred_l[lane] : 0.f;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
          const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
          if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
        }
        if (lane == 0) { sh.red_h[1] = mh; sh.red_l[1] = ml; }
      }
    }
    __syncthreads();
    const float gmh = sh.red_h[1], gml = sh.red_l[1];
    ok = gmh < CUDART_INF_F;
    for (int q = threadIdx.x; q < nrows; q += blockDim.x) ustar[q] = 0.f;
    for (int b0 = 0; b0 < nb; b0 += 256) {
      __syncthreads();
      for (int t = threadIdx.x; t < 256 && b0 + t < nb; t += blockDim.x) {
        const size_t base = static_cast<size_t>(b0 + t) * stride;
        const bool held = b0 == 0 && t == static_cast<int>(threadIdx.x);
        const float h = held ? h0 : __ldcg(in.part + base + 0), l = held ? l0 : __ldcg(in.part + base + 1);
        S.chunk[t] = (ok && h < CUDART_INF_F) ? expf(-((h - gmh) + (l - gml)) * k.inv_lambda) : 0.f;
      }
      __syncthreads();
      const int bend = min(256, nb - b0);
      for (int q = threadIdx.x; q < nrows; q += blockDim.x) {
        // four independent chains (tiles t mod 4), combined in a fixed order;
        // 64 (then 16) L2 loads in flight per pass
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float* col = in.part + static_cast<size_t>(b0) * stride + 3 + q;
        int t = 0;
        for (; t + 64 <= bend; t += 64) {
          // `pre` is the pass buffer: it already holds the first pass of the
          // thread's first row
          if (!(pre_ok && b0 == 0 && t == 0 && q == static_cast<int>(threadIdx.x))) {
#pragma unroll
            for (int m = 0; m < 64; ++m) pre[m] = __ldcg(col + static_cast<size_t>(t + m) * stride);
          }
#pragma unroll
          for (int m = 0; m < 64; m += 4) {
            a0 += S.chunk[t + m + 0] * pre[m + 0];
            a1 += S.chunk[t + m + 1] * pre[m + 1];
            a2 += S.chunk[t + m + 2] * pre[m + 2];
            a3 += S.chunk[t + m + 3] * pre[m + 3];
          }
        }
        for (; t + 16 <= bend; t += 16) {
          float v[16];
#pragma unroll
          for (int m = 0; m < 16; ++m) v[m] = __ldcg(col + static_cast<size_t>(t + m) * stride);
#pragma unroll
          for (int m = 0; m < 16; m += 4) {
            a0 += S.chunk[t + m + 0] * v[m + 0];
            a1 += S.chunk[t + m + 1] * v[m + 1];
            a2 += S.chunk[t + m + 2] * v[m + 2];
            a3 += S.chunk[t + m + 3] * v[m + 3];
          }
        }
        for (; t + 4 <= bend; t += 4) {
          a0 += S.chunk[t + 0] * __ldcg(col + static_cast<size_t>(t + 0) * stride);
          a1 += S.chunk[t + 1] * __ldcg(col + static_cast<size_t>(t + 1) * stride);
          a2 += S.chunk[t + 2] * __ldcg(col + static_cast<size_t>(t + 2) * stride);
          a3 += S.chunk[t + 3] * __ldcg(col + static_cast<size_t>(t + 3) * stride);
        }
        for (; t < bend; ++t) a0 += S.chunk[t] * __ldcg(col + static_cast<size_t>(t) * stride);
        ustar[q] += (a0 + a1) + (a2 + a3);
      }
    }
  }
  // path turns between consecutive rows (this CTA's frame-shifted table;
  // 1e-4 rad over pi/4 covers the shift's rounding): an out-of-range turn
  // rejects the solve
  int turn_bad = 0;
  for (int j = threadIdx.x; j + 1 < in.n_pts; j += blockDim.x)
    turn_bad |= !(fabsf(S.path[3 * j + 5] - S.path[3 * j + 2]) <= kMaxPathTurn + 1e-4f);
  const bool turns_bad = __syncthreads_or(turn_bad);
  const float lsum = ustar[3 * H];
  const unsigned err = sh.err | (turns_bad ? ERR_PATH_TURN : 0u);
  for (int q = threadIdx.x; q < 3 * H; q += blockDim.x) {
    const float u = ok ? ustar[q] / lsum : S.unom[q];
    ustar[q] = u;
    in.U_out[q] = u;
  }
  __syncthreads();
  if (in.U_next) {
    for (int q = threadIdx.x; q < 3 * H; q += blockDim.x) {
      const int tau = q / 3, j = q % 3;
      in.U_next[q] = ustar[3 * min(tau + 1, H - 1) + j];
    }
  }
  if (threadIdx.x == 0) {
    if (in.status) {
      int32_t st = 0;
      if (err & (ERR_EXPONENT | ERR_PATH_TURN)) st = -1;
      else if ((err & ERR_NONFINITE_X0) || !ok) st = -5;
      *in.status = st;
    }
    in.sync[1] = 0u;
    in.sync[0] = 0u;
  }
  if (in.traj_out) {
    // scratch: the obstacle, path and nominal-input tables (contiguous, no
    // longer read by this CTA's merge), else the consumed partials
    if (static_cast<long long>(S.ustar - S.obs) >= 8LL * (H + 1)) {
      optimal_trajectory(k, in, S, sh, S.obs);
    } else if (static_cast<long long>(in.tiles) * in.part_stride >= 8LL * (H + 1)) {
      optimal_trajectory(k, in, S, sh, in.part);
    } else if (threadIdx.x == 0) {
      serial_trajectory(k, in, S, sh);
    }
  }
  __syncthreads();
}

// The tile's applied-input history in global memory is dead once the tile's
// weighted sums have read it: its L2 lines are dropped without being written
// back to DRAM (discard.global.L2, whole 128-byte lines only, so a line
// shared with the neighbouring CTA's slot is left alone).  Every read of the
// history must be complete (after a CTA barrier); the next tile writes
// before it reads.
__device__ __forceinline__ void discard_history(const float* uh, int n_floats) {
  const unsigned long long b0 = reinterpret_cast<unsigned long long>(uh);
  const unsigned long long b1 = b0 + 4ull * static_cast<unsigned long long>(n_floats);
  const unsigned long long first = (b0 + 127ull) & ~127ull, last = b1 & ~127ull;
  for (unsigned long long a = first + 128ull * threadIdx.x; a < last; a += 128ull * blockDim.x) {
    unsigned long long g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(a));
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(g) : "memory");
  }
}

// -------------------------------------------------------------- the kernel
// EXT: the instantiations that also carry the optional terms (moving and
// e = 4 obstacles, collision cost, buffer cost); the others compile them out.
template <int TPS, int BPT, bool EXT, int ROWS = 0>
// Launch bound: 512 threads (128 registers a thread); the exact-rows
// single-solve instantiations 384 (up to 170 registers: one CTA per SM on
// the latency shapes, where registers buy a longer schedule)
__global__ void __launch_bounds__(ROWS > 0 ? 384 : 512) solve_kernel(const KConst k, const LaunchDesc L) {
  extern __shared__ float dyn[];
  __shared__ Shared sh;
  const int spb = compute_threads<TPS>(L.noise_warps) / TPS;
  const Smem S(dyn, L.caps, spb);
  // applied-input history of the CTA's tile: shared memory in the exact-rows
  // variants (the launch reserved it), else the CTA's global slot
  float* uh;
  if constexpr (ROWS > 0) {
    uh = S.noise + L.caps.noise_per_team * spb;
  } else {
    uh = L.uh + static_cast<size_t>(blockIdx.x) * L.uh_stride;
  }

  for (int iter = 0;; ++iter) {
    int inst_id = 0, tile;
    if (L.work) {
      if (threadIdx.x == 0) sh.item = static_cast<int>(atomicAdd(L.work_ctr, 1u));
      __syncthreads();
      const int item = sh.item;
      __syncthreads();
      if (item >= L.n_work) break;
      const int2 w = L.work[item];
      inst_id = w.x;
      tile = w.y;
    } else {
      if (iter > 0) break;
      tile = L.single.tile_base + static_cast<int>(blockIdx.x);
    }
    Inst in;
    if (L.work) in = L.inst[inst_id];
    else in = L.single;
    run_tile<TPS, BPT, EXT, ROWS>(k, in, tile, uh, S, sh, L.noise_warps);

    // the CTA that completes an instance's last tile merges its partials
    __threadfence();
    __syncthreads();
    if constexpr (ROWS == 0) discard_history(uh, 3 * in.H * (compute_threads<TPS>(L.noise_warps) / TPS));
    if (in.no_merge) continue;  // a share of the tiles: merged elsewhere (single launches only)
    if (threadIdx.x == 0) sh.last = (atomicAdd(in.sync, 1u) == static_cast<unsigned>(in.tiles - 1));
    __syncthreads();
    if (sh.last) {
      __threadfence();
      merge_instance<(ROWS > 0)>(k, in, S, sh);
    }
    __syncthreads();
  }
  if (L.work) {
    // the last CTA to run out of work resets the work counters for the
    // next launch (no CTA reads them after its final fetch)
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(L.work_ctr + 1, 1u) == gridDim.x - 1) {
        L.work_ctr[0] = 0u;
        L.work_ctr[1] = 0u;
      }
    }
  }
}

// ------------------------------------------------ merge of gathered tiles
// One CTA merges an instance's complete set of tile partials, produced by
// no-merge launches (one per rank of a sample-partitioned solve) and
// gathered in tile order: the same frame, tables and merge as the CTA that
// finishes a single launch's last tile, so the results are the same bits.
template <bool EXT>
__global__ void __launch_bounds__(256) merge_tiles_kernel(const KConst k, const Inst in, const SmemCaps caps) {
  extern __shared__ float dyn[];
  __shared__ Shared sh;
  const Smem S(dyn, caps, 1);
  for (int j = threadIdx.x; j < 3 * in.n_pts; j += blockDim.x) cp_async4(S.path + j, in.path + j);
  for (int j = threadIdx.x; j < 3 * in.H; j += blockDim.x) cp_async4(S.unom + j, in.U_nom + j);
  if (threadIdx.x < 32) make_frame_warp(in.x0, in.inv_ds_d, in.sync + 1, sh.fr, EXT && k.jerk);
  const bool obs8 = EXT && k.obs8;
  for (int o = threadIdx.x; o < in.n_obs; o += blockDim.x) {
    const float e = in.obs[(obs8 ? 8 : 6) * o + 5];
    if (e != 2.0f && !(obs8 && e == 4.0f)) atomicOr(in.sync + 1, ERR_EXPONENT);
  }
  cp_async_wait_all();
  __syncthreads();
  const Frame& fr = sh.fr;
  for (int j = threadIdx.x; j < in.n_pts; j += blockDim.x) {  // the path in the frame, as the tiles stage it
    float* d = S.path + 3 * j;
    d[0] = (d[0] - fr.ox_h) - fr.ox_l;
    d[1] = (d[1] - fr.oy_h) - fr.oy_l;
    d[2] = (d[2] - fr.oth_h) - fr.oth_l;
  }
  __syncthreads();
  merge_instance<false>(k, in, S, sh);
}

}  // namespace brmppi
