// rollout.cuh -- device code of one BR-MPPI solve for sm_103a.
//
// Paper: "GPU-Accelerated Barrier-Rate Guided MPPI Control for
// Tractor-Trailer Systems" (arXiv 2508.05773).  One solve (Sec. II-B MPPI
// with the BR-MPPI rollout of Sec. IV-A):
//
//   for each sample s, step tau:
//     noise        Philox4x32-10 + Box-Muller, recomputed in registers
//     sample       z_des = clip(U_nom + sigma n), u^alpha_des = clip(sigma_a n)
//     rows         barrier-rate equality per constraint (Eq. cbf_equality):
//                  hitch (Eq. hitch_angle_barrier) and ellipses
//                  (Eq. barrier_function) through the second-order expansion
//                  of Eq. barrier_function_approx
//     projection   Eq. closed-form_projection in Woodbury form (below)
//     apply        u = clip(z*_u), alpha += z*_alpha
//     dynamics     explicit Euler (Eq. tt_discrete_kinematics)
//     cost         Eq. cost_function_contour at the new state
//   softmin + update (Eq. MPPI_update_rule) as block partials of a
//   max-subtracted log-sum-exp, merged in a fixed order by the last block.
//
// Work decomposition: a "team" of TPS consecutive lanes owns one sample.
// Lane j of a team owns Philox blocks b = j, j + TPS, ... (< ceil(d/4)),
// i.e. the normals q = 4b..4b+3 and with them the constraints i = q - 3.
// Block 0 (team lane 0) carries the three input normals and the hitch row.
// The rank-2 structure of the projection makes the cross-lane exchange five
// floats per step (a butterfly over the team).
//
// Projection in Woodbury form.  A = [A_u | diag(h~)] where only the a and
// omega columns of A_u are non-zero, M = diag(m_u, m_alpha):
//   K = A M^-1 A^T = D + A_u M_u^-1 A_u^T,  D = diag(h~^2 / m_alpha),
//   S2 = M_u + A_u^T D^-1 A_u (2x2),  g = A_u^T D^-1 r,  y = S2^-1 g,
//   r  = A M^-1 p - b,  lambda = D^-1 (r - A_u y),
//   z*_u = M_u^-1 p_u - y,  z*_alpha_i = p_alpha_i/m_alpha - (r_i - a_i.y)/h~_i,
// algebraically identical to M^-1 [p - A^T K^-1 (A M^-1 p - b)].
//
// Numerics: states are carried relative to the initial pose (position
// relative to (px0, py0), angles relative to theta1_0, progress relative to
// psi0), so that FP32 rounding is relative to the few metres a rollout
// travels rather than to the world coordinates; the cost sum is carried as
// an unevaluated pair (TwoSum), and the softmin works on pair differences.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace brmppi {

// ---------------------------------------------------------------- constants
struct KParams {
  int S, H, n_obs, n_pts, Nc, P, proj;
  float Ts, hTs2, inv_lambda;
  float inv_l1, inv_l2, k_hitch, dtheta_max, kappa, r_inflate;
  float Qc, Ql, Qth, R0, R1, R2, mu, nu_bar;
  float zlo0, zlo1, zlo2, zhi0, zhi1, zhi2, sig0, sig1, sig2;
  float alpha0, sigma_alpha, ua_lo, ua_hi;
  float w_u0, w_u1, w_u2, pc_u0, pc_u1, pc_u2;  // W_u and rho/2 (hi + lo)
  float m_u0, m_u1, inv_m_u0, inv_m_u1, inv_m_u2;
  float w_a, pc_a, m_a, inv_m_a;
  float h_floor, ds, inv_ds;
  uint32_t key0, key1, ctr;
  int part_stride;  // floats per block partial
};

struct KIO {
  const double* x0;
  const float* U_nom;
  const float* obs;
  const float* path;
  float* U_out;
  float* traj_out;
  float* J_out;
  float* U_next;
  int32_t* status;
  float* part;
  unsigned int* ticket;
  unsigned int* err;
};

enum : unsigned { ERR_EXPONENT = 1u, ERR_NONFINITE_X0 = 2u };

// Dynamic shared memory layout (floats), identical for every launch shape.
struct SmemLayout {
  int obs, path, unom, uh, jh, jl, w, chunk, total;
  __host__ __device__ SmemLayout(int n_obs, int n_pts, int H, int spb) {
    int o = 0;
    obs = o;   o += 8 * n_obs;
    path = o;  o += 3 * n_pts;
    unom = o;  o += 3 * H;
    uh = o;    o += 3 * H * spb;
    jh = o;    o += spb;
    jl = o;    o += spb;
    w = o;     o += spb;
    chunk = o; o += 256;
    total = o;
  }
};

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
// ((w >> 9) + 1/2) * 2^-23 lies in (0, 1) and is exact in binary32.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const float ua = (static_cast<float>(wa >> 9) + 0.5f) * 1.1920928955078125e-07f;
  const float ub = (static_cast<float>(wb >> 9) + 0.5f) * 1.1920928955078125e-07f;
  const float radius = sqrtf(-2.0f * logf(ua));
  float sn, cs;
  sincospif(2.0f * ub, &sn, &cs);
  n0 = radius * cs;
  n1 = radius * sn;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// into [-pi, pi]; only the square of the result is used
__device__ __forceinline__ float wrap_pi(float a) {
  return a - 6.28318530717958647692f * rintf(a * 0.15915494309189533577f);
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

// ------------------------------------------------------------ the rollout
// Frame of one solve (relative coordinates), computed per block from x0.
// Doubles of x0 enter as unevaluated float pairs (hi + lo), so that the
// per-block staging needs no FP64 arithmetic.
struct Frame {
  float ox_h, ox_l, oy_h, oy_l, oth_h, oth_l;  // origin (px0, py0, theta1_0)
  float c0, s0;                                // cos / sin of theta1_0
  float t2, v_h, v_l, dl;                      // theta2 - theta1_0, speed, steer angle
  float qf0;                                   // fractional path cell of psi0
  int i0;                                      // integer path cell of psi0
  double psi0;
};

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

template <int TPS, int BPT>
__global__ void __launch_bounds__(512)
rollout_solve_kernel(const KParams p, const KIO io) {
  extern __shared__ float sm[];
  __shared__ Frame fr;
  __shared__ float red_h[32], red_l[32];
  __shared__ int am_last;

  const int spb = blockDim.x / TPS;
  const SmemLayout L(p.n_obs, p.n_pts, p.H, spb);
  const int team = threadIdx.x / TPS;
  const int lt = threadIdx.x % TPS;
  const int s = blockIdx.x * spb + team;

  // --- frame and staging (tables in shared memory, relative coordinates)
  if (threadIdx.x == 0) {
    const double* x0 = io.x0;
    bool finite = true;
    for (int j = 0; j < 7; ++j) finite = finite && isfinite(x0[j]);
    if (!finite) atomicOr(io.err, ERR_NONFINITE_X0);
    split_double(x0[0], fr.ox_h, fr.ox_l);
    split_double(x0[1], fr.oy_h, fr.oy_l);
    split_double(x0[2], fr.oth_h, fr.oth_l);
    float sn, cs;
    sincosf(fr.oth_h, &sn, &cs);
    fr.c0 = cs - sn * fr.oth_l;  // cos(hi + lo), lo below one ulp of hi
    fr.s0 = sn + cs * fr.oth_l;
    fr.t2 = static_cast<float>(x0[3] - x0[2]);
    split_double(x0[4], fr.v_h, fr.v_l);
    fr.dl = static_cast<float>(x0[5]);
    fr.psi0 = x0[6];
    const double q0 = x0[6] / static_cast<double>(p.ds);
    const double fq = fmin(fmax(floor(q0), -1.0e9), 1.0e9);
    fr.i0 = static_cast<int>(fq);
    fr.qf0 = static_cast<float>(q0 - fq);
  }
  __syncthreads();
  for (int o = threadIdx.x; o < p.n_obs; o += blockDim.x) {
    const float* ob = io.obs + 6 * o;
    float* d = sm + L.obs + 8 * o;
    if (ob[5] != 2.0f) atomicOr(io.err, ERR_EXPONENT);
    const float Ax = ob[2] + p.r_inflate, Ay = ob[3] + p.r_inflate;
    d[0] = (ob[0] - fr.ox_h) - fr.ox_l;
    d[1] = (ob[1] - fr.oy_h) - fr.oy_l;
    sincosf(ob[4], &d[3], &d[2]);
    d[4] = 1.0f / (Ax * Ax);
    d[5] = 1.0f / (Ay * Ay);
    d[6] = 0.0f;
    d[7] = 0.0f;
  }
  for (int j = threadIdx.x; j < p.n_pts; j += blockDim.x) {
    const float* r = io.path + 3 * j;
    float* d = sm + L.path + 3 * j;
    d[0] = (r[0] - fr.ox_h) - fr.ox_l;
    d[1] = (r[1] - fr.oy_h) - fr.oy_l;
    d[2] = (r[2] - fr.oth_h) - fr.oth_l;
  }
  for (int j = threadIdx.x; j < 3 * p.H; j += blockDim.x) sm[L.unom + j] = io.U_nom[j];
  __syncthreads();

  const float* obs_s = sm + L.obs;
  const float* path_s = sm + L.path;
  const float* unom_s = sm + L.unom;
  float* uh_s = sm + L.uh;

  // --- per-sample state (relative frame); position, speed and progress
  // carried as compensated pairs
  const float c0 = fr.c0, s0 = fr.s0;
  float px = 0.f, pxl = 0.f, py = 0.f, pyl = 0.f, t1 = 0.f, t2 = fr.t2, v = fr.v_h, vl = fr.v_l,
        dl = fr.dl, ps = 0.f, psl = 0.f;
  float alpha[4 * BPT];
#pragma unroll
  for (int k = 0; k < 4 * BPT; ++k) alpha[k] = p.alpha0;
  float Jh = 0.f, Jl = 0.f;
  const uint32_t sid = static_cast<uint32_t>(s);

  // noise of step tau for this lane's Philox blocks (computed one step ahead)
  auto draw = [&](int tau, float* out) {
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const int b = lt + TPS * k;
      if (b < p.P) {
        const uint4 w = philox4x32_10(
            make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(tau), sid, p.ctr), p.key0, p.key1);
        box_muller(w.x, w.y, out[4 * k + 0], out[4 * k + 1]);
        box_muller(w.z, w.w, out[4 * k + 2], out[4 * k + 3]);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) out[4 * k + m] = 0.f;
      }
    }
  };
  float nrm[4 * BPT];
  draw(0, nrm);

  for (int tau = 0; tau < p.H; ++tau) {
    float nxt[4 * BPT];
    draw(tau + 1 < p.H ? tau + 1 : tau, nxt);
    const float na = team_bcast0<TPS>(nrm[0]);
    const float nw = team_bcast0<TPS>(nrm[1]);
    const float nn = team_bcast0<TPS>(nrm[2]);
    const float zd0 = clampf(unom_s[3 * tau + 0] + p.sig0 * na, p.zlo0, p.zhi0);
    const float zd1 = clampf(unom_s[3 * tau + 1] + p.sig1 * nw, p.zlo1, p.zhi1);
    const float zd2 = clampf(unom_s[3 * tau + 2] + p.sig2 * nn, p.zlo2, p.zhi2);

    // trigonometry of the current state
    float sr, cr;
    sincosf(t1, &sr, &cr);
    const float c1 = c0 * cr - s0 * sr;
    const float s1 = s0 * cr + c0 * sr;
    const float phi = t1 - t2;
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float tn = tanf(dl);
    const float vv = v + vl;
    const float th1dot = vv * tn * p.inv_l1;

    float za, zw, zn;
    if (p.proj) {
      const float pu0 = p.w_u0 * zd0 + p.pc_u0;
      const float pu1 = p.w_u1 * zd1 + p.pc_u1;
      const float pu2 = p.w_u2 * zd2 + p.pc_u2;
      const float q0 = pu0 * p.inv_m_u0, q1 = pu1 * p.inv_m_u1;  // M_u^-1 p_u
      float Saa = 0.f, Saw = 0.f, Sww = 0.f, ga = 0.f, gw = 0.f;
      float ca[4 * BPT], cw[4 * BPT], cc[4 * BPT];
#pragma unroll
      for (int k = 0; k < BPT; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int slot = 4 * k + m;
          const int i = 4 * (lt + TPS * k) + m - 3;  // constraint index
          ca[slot] = 0.f;
          cw[slot] = 0.f;
          cc[slot] = 0.f;
          if (i >= 0 && i < p.Nc) {
            float Aa, Aw, h, brest;
            if (i == 0) {
              // hitch row: Delta = th2 - th1, sigma = sgn(Delta), sgn(0) = +1
              const float Delta = t2 - t1;
              const float sg = Delta >= 0.f ? 1.f : -1.f;
              const float G = sp - p.k_hitch * cp * tn;
              const float th2dot = vv * G * p.inv_l2;
              const float phidot = th1dot - th2dot;
              const float sec2 = 1.f + tn * tn;
              h = p.dtheta_max - p.kappa * vv - sg * Delta;
              Aa = -p.Ts * p.kappa - p.hTs2 * sg * (G * p.inv_l2 - tn * p.inv_l1);
              Aw = p.hTs2 * sg * vv * sec2 * (p.k_hitch * cp * p.inv_l2 + p.inv_l1);
              const float c0h = -p.Ts * sg * (th2dot - th1dot) -
                                p.hTs2 * sg * vv * p.inv_l2 * (cp + p.k_hitch * tn * sp) * phidot;
              brest = -c0h;
            } else {
              // ellipse row (e = 2) in the obstacle frame
              const float* ob = obs_s + 8 * (i - 1);
              const float dx = (px - ob[0]) + pxl, dy = (py - ob[1]) + pyl;
              const float co = ob[2], so = ob[3], iax = ob[4], iay = ob[5];
              const float xp = co * dx + so * dy;
              const float yp = co * dy - so * dx;
              h = xp * xp * iax + yp * yp * iay - 1.f;
              const float hx = 2.f * xp * iax, hy = 2.f * yp * iay;
              const float dirx = co * c1 + so * s1, diry = co * s1 - so * c1;
              const float velx = vv * dirx, vely = vv * diry;
              const float vw = vv * th1dot;
              const float hdot = hx * velx + hy * vely;
              const float hdd0 = vw * (hy * dirx - hx * diry) +
                                 2.f * (iax * velx * velx + iay * vely * vely);
              Aa = p.hTs2 * (hx * dirx + hy * diry);
              Aw = 0.f;
              brest = -p.Ts * hdot - p.hTs2 * hdd0;
            }
            const float hm = fmaxf(fabsf(h), p.h_floor);
            const float ht = h >= 0.f ? hm : -hm;
            const float zda = clampf(p.sigma_alpha * nrm[slot], p.ua_lo, p.ua_hi);
            const float pa = p.w_a * zda + p.pc_a;
            const float b = -alpha[slot] * h + brest;
            const float r = Aa * q0 + Aw * q1 + ht * pa * p.inv_m_a - b;
            const float iht = 1.f / ht;
            const float invD = p.m_a * iht * iht;
            Saa += Aa * Aa * invD;
            Saw += Aa * Aw * invD;
            Sww += Aw * Aw * invD;
            ga += Aa * r * invD;
            gw += Aw * r * invD;
            ca[slot] = Aa * iht;
            cw[slot] = Aw * iht;
            cc[slot] = pa * p.inv_m_a - r * iht;
          }
        }
      }
      Saa = team_sum<TPS>(Saa) + p.m_u0;
      Saw = team_sum<TPS>(Saw);
      Sww = team_sum<TPS>(Sww) + p.m_u1;
      ga = team_sum<TPS>(ga);
      gw = team_sum<TPS>(gw);
      const float idet = 1.f / (Saa * Sww - Saw * Saw);
      const float ya = (Sww * ga - Saw * gw) * idet;
      const float yw = (Saa * gw - Saw * ga) * idet;
      za = q0 - ya;
      zw = q1 - yw;
      zn = pu2 * p.inv_m_u2;
#pragma unroll
      for (int slot = 0; slot < 4 * BPT; ++slot) alpha[slot] += cc[slot] + ca[slot] * ya + cw[slot] * yw;
    } else {
      za = zd0;
      zw = zd1;
      zn = zd2;
    }
    const float ua = clampf(za, p.zlo0, p.zhi0);
    const float uw = clampf(zw, p.zlo1, p.zhi1);
    const float un = clampf(zn, p.zlo2, p.zhi2);

    // explicit Euler step, right-hand sides at the current state
    const float Tv = p.Ts * vv;
    acc2(px, pxl, Tv * c1);
    acc2(py, pyl, Tv * s1);
    t1 += p.Ts * th1dot;
    t2 += Tv * p.inv_l2 * (sp - p.k_hitch * cp * tn);
    acc2(v, vl, p.Ts * ua);
    dl += p.Ts * uw;
    acc2(ps, psl, p.Ts * un);

    // stage cost at the new state
    const float qf = fr.qf0 + (ps * p.inv_ds + psl * p.inv_ds);
    const float fl = floorf(qf);
    int ii = fr.i0 + static_cast<int>(fl);
    float ff = qf - fl;
    if (ii < 0) {
      ii = 0;
      ff = 0.f;
    } else if (ii > p.n_pts - 2) {
      ii = p.n_pts - 2;
      ff = 1.f;
    }
    const float* r0 = path_s + 3 * ii;
    const float xr = r0[0] + ff * (r0[3] - r0[0]);
    const float yr = r0[1] + ff * (r0[4] - r0[1]);
    const float thr = r0[2] + ff * (r0[5] - r0[2]);
    float st, ct;
    sincosf(thr, &st, &ct);
    const float cth = c0 * ct - s0 * st;
    const float sth = s0 * ct + c0 * st;
    const float dxr = (px - xr) + pxl, dyr = (py - yr) + pyl;
    const float ec = sth * dxr - cth * dyr;
    const float el = -cth * dxr - sth * dyr;
    const float e1 = wrap_pi(t1 - thr), e2 = wrap_pi(t2 - thr);
    const float dn = p.nu_bar - un;
    const float rc = p.Qc * ec * ec + p.Ql * el * el + p.Qth * (e1 * e1 + e2 * e2) +
                     p.R0 * ua * ua + p.R1 * uw * uw + p.R2 * un * un + p.mu * dn * dn;
    // TwoSum accumulation
    const float sum = Jh + rc;
    const float bp = sum - Jh;
    Jl += (Jh - (sum - bp)) + (rc - bp);
    Jh = sum;

    if (lt == 0) {
      uh_s[(3 * tau + 0) * spb + team] = ua;
      uh_s[(3 * tau + 1) * spb + team] = uw;
      uh_s[(3 * tau + 2) * spb + team] = un;
    }
#pragma unroll
    for (int k = 0; k < 4 * BPT; ++k) nrm[k] = nxt[k];
  }

  // --- per-sample cost: normalise the pair
  {
    const float sum = Jh + Jl;
    Jl = Jl - (sum - Jh);
    Jh = sum;
  }
  const bool valid = s < p.S;
  if (lt == 0) {
    const bool fin = valid && isfinite(Jh) && isfinite(Jl);
    sm[L.jh + team] = fin ? Jh : CUDART_INF_F;
    sm[L.jl + team] = fin ? Jl : 0.f;
    if (valid && io.J_out) io.J_out[s] = Jh + Jl;
  }
  __syncthreads();

  // --- block softmin partial: min, weights, sum, weighted inputs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  if (warp == 0) {
    float mh = CUDART_INF_F, ml = 0.f;
    for (int t = lane; t < spb; t += 32) {
      const float h = sm[L.jh + t], l = sm[L.jl + t];
      if (pair_less(h, l, mh, ml)) { mh = h; ml = l; }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
      const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
      if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
    }
    if (lane == 0) { red_h[0] = mh; red_l[0] = ml; }
  }
  __syncthreads();
  const float bmh = red_h[0], bml = red_l[0];
  const bool any_finite = bmh < CUDART_INF_F;
  for (int t = threadIdx.x; t < spb; t += blockDim.x) {
    const float h = sm[L.jh + t];
    float w = 0.f;
    if (any_finite && h < CUDART_INF_F) w = expf(-((h - bmh) + (sm[L.jl + t] - bml)) * p.inv_lambda);
    sm[L.w + t] = w;
  }
  __syncthreads();
  float* part = io.part + static_cast<size_t>(blockIdx.x) * p.part_stride;
  const int nrows = 3 * p.H + 1;  // row 3H: the weight sum
  for (int row = warp; row < nrows; row += nwarps) {
    float acc = 0.f;
    if (row < 3 * p.H) {
      for (int t = lane; t < spb; t += 32) acc += sm[L.w + t] * uh_s[row * spb + t];
    } else {
      for (int t = lane; t < spb; t += 32) acc += sm[L.w + t];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (lane == 0) part[3 + row] = acc;
  }
  if (threadIdx.x == 0) {
    part[0] = bmh;
    part[1] = bml;
    part[2] = any_finite ? 1.f : 0.f;
  }

  // --- last block merges the partials in block order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(io.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();

  const int nb = gridDim.x;
  const int stride = p.part_stride;
  // global minimum pair
  if (warp == 0) {
    float mh = CUDART_INF_F, ml = 0.f;
    for (int b = lane; b < nb; b += 32) {
      const float h = __ldcg(io.part + static_cast<size_t>(b) * stride + 0);
      const float l = __ldcg(io.part + static_cast<size_t>(b) * stride + 1);
      if (pair_less(h, l, mh, ml)) { mh = h; ml = l; }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, mh, m);
      const float ol = __shfl_xor_sync(0xffffffffu, ml, m);
      if (pair_less(oh, ol, mh, ml)) { mh = oh; ml = ol; }
    }
    if (lane == 0) { red_h[1] = mh; red_l[1] = ml; }
  }
  __syncthreads();
  const float gmh = red_h[1], gml = red_l[1];
  const bool ok = gmh < CUDART_INF_F;
  float* chunk = sm + L.chunk;
  float* ustar = sm + L.uh;  // reuse: 3H + 1 accumulators
  for (int k = threadIdx.x; k < nrows; k += blockDim.x) ustar[k] = 0.f;
  for (int b0 = 0; b0 < nb; b0 += 256) {
    __syncthreads();
    for (int t = threadIdx.x; t < 256 && b0 + t < nb; t += blockDim.x) {
      const size_t base = static_cast<size_t>(b0 + t) * stride;
      const float h = __ldcg(io.part + base + 0), l = __ldcg(io.part + base + 1);
      chunk[t] = (ok && h < CUDART_INF_F) ? expf(-((h - gmh) + (l - gml)) * p.inv_lambda) : 0.f;
    }
    __syncthreads();
    const int bend = min(256, nb - b0);
    for (int k = threadIdx.x; k < nrows; k += blockDim.x) {
      float acc = ustar[k];
      for (int t = 0; t < bend; ++t) {
        const float sc = chunk[t];
        if (sc != 0.f) acc += sc * __ldcg(io.part + static_cast<size_t>(b0 + t) * stride + 3 + k);
      }
      ustar[k] = acc;
    }
  }
  __syncthreads();
  const float lsum = ustar[3 * p.H];
  const unsigned err = atomicAdd(io.err, 0u);
  for (int k = threadIdx.x; k < 3 * p.H; k += blockDim.x) {
    const float u = ok ? ustar[k] / lsum : unom_s[k];
    ustar[k] = u;
    io.U_out[k] = u;
  }
  __syncthreads();
  if (io.U_next) {
    for (int k = threadIdx.x; k < 3 * p.H; k += blockDim.x) {
      const int tau = k / 3, j = k % 3;
      io.U_next[k] = ustar[3 * min(tau + 1, p.H - 1) + j];
    }
  }
  if (threadIdx.x == 0) {
    if (io.status) {
      int32_t st = 0;
      if (err & ERR_EXPONENT) st = -1;
      else if ((err & ERR_NONFINITE_X0) || !ok) st = -5;
      *io.status = st;
    }
    // optimal trajectory: x0 integrated with U* (same relative frame)
    if (io.traj_out) {
      float qx = 0.f, qy = 0.f, q1 = 0.f, q2 = fr.t2, qv = fr.v_h + fr.v_l, qd = fr.dl, qp = 0.f;
      float* tr = io.traj_out;
      for (int tau = 0; tau <= p.H; ++tau) {
        tr[7 * tau + 0] = (fr.ox_h + qx) + fr.ox_l;
        tr[7 * tau + 1] = (fr.oy_h + qy) + fr.oy_l;
        tr[7 * tau + 2] = (fr.oth_h + q1) + fr.oth_l;
        tr[7 * tau + 3] = (fr.oth_h + q2) + fr.oth_l;
        tr[7 * tau + 4] = qv;
        tr[7 * tau + 5] = qd;
        tr[7 * tau + 6] = static_cast<float>(fr.psi0 + static_cast<double>(qp));
        if (tau == p.H) break;
        float a1, b1;
        sincosf(q1, &a1, &b1);
        const float cc1 = c0 * b1 - s0 * a1, ss1 = s0 * b1 + c0 * a1;
        float a2, b2;
        sincosf(q1 - q2, &a2, &b2);
        const float tq = tanf(qd);
        const float Tv = p.Ts * qv;
        qx += Tv * cc1;
        qy += Tv * ss1;
        const float d1 = Tv * tq * p.inv_l1;
        q2 += Tv * p.inv_l2 * (a2 - p.k_hitch * b2 * tq);
        q1 += d1;
        qv += p.Ts * ustar[3 * tau + 0];
        qd += p.Ts * ustar[3 * tau + 1];
        qp += p.Ts * ustar[3 * tau + 2];
      }
    }
    *io.err = 0u;
    *io.ticket = 0u;
  }
}

}  // namespace brmppi
