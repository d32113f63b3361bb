/*
 * brmppi_oracle.c -- plain FP64 CPU oracle for one BR-MPPI control solve.
 *
 * TEST INFRASTRUCTURE ONLY (see brmppi_oracle.h).  Slow on purpose: plain
 * loops, libm, a dense Cholesky solve for the projection, no blocking, no
 * fusion.  Each function names the passage of the paper it restates.
 *
 * Readings of the paper where it is silent or garbled (the same readings the
 * CUDA path takes):
 *   - model: accel a is an input, progress psi is a state driven by nu
 *     (psi' = nu, Sec. IV-B); explicit Euler with every right-hand side at
 *     step k (Sec. III-A); angles are never wrapped, delta is not clamped.
 *   - barrier-rate row: L_f h + L_g h u is the second-order Taylor increment
 *     Ts*hdot + Ts^2/2*hddot along the continuous vector field with the input
 *     held (Eq. barrier_function_approx, Sec. IV-C), for obstacles and hitch.
 *   - sign of the CBF equality as printed in Eq. cbf_equality.
 *   - alpha_i starts at alpha0 each rollout; its nominal input is 0; the
 *     sampled u^alpha is clipped to [ua_lo, ua_hi]; alpha itself is unclipped.
 *   - A's alpha column uses h_tilde = sgn(h) max(|h|, h_floor), sgn(0) = +1.
 *   - z_des is clipped to the box before projection; after projection only
 *     the physical input u is clipped (the applied input).
 *   - the applied input drives dynamics, cost and the weighted update.
 *   - J = sum_{tau=0}^{H-1} r(x_{tau+1}, u_tau), no terminal cost, no
 *     lambda u^T Sigma^-1 u term; heading errors wrapped into (-pi, pi];
 *     theta2r = theta1r (one heading column).
 */
#include "brmppi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10.  Salmon et al., SC'11: each round multiplies words 0 and 2
   by the two round constants, and the next counter is
   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
   the key is bumped by the two Weyl constants before every round but the
   first. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 32-bit word -> uniform in (0, 1): the top 23 bits plus one half, scaled by
   2^-23 (exact in binary32 and binary64). */
static double word_to_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Noise of the MPPI sampling step (Sec. II-B: w ~ N(0, Sigma)), drawn from
   the counter-based stream: normal q is lane q%4 of Philox block q/4 at
   counter (q/4, tau, s, counter_lo32), key (seed_lo32, seed_hi32); lanes
   (0,1) and (2,3) are Box-Muller pairs. */
void orc_normals(uint64_t seed, uint64_t counter, uint32_t s, uint32_t tau, int d, double *n) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int blk = 0; 4 * blk < d; ++blk) {
    const uint32_t ctr[4] = {(uint32_t)blk, tau, s, (uint32_t)counter};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double g[4];
    for (int pair = 0; pair < 2; ++pair) {
      double ua = word_to_uniform(w[2 * pair]);
      double ub = word_to_uniform(w[2 * pair + 1]);
      double radius = sqrt(-2.0 * log(ua));
      double angle = 2.0 * M_PI * ub;
      g[2 * pair] = radius * cos(angle);
      g[2 * pair + 1] = radius * sin(angle);
    }
    for (int lane = 0; lane < 4 && 4 * blk + lane < d; ++lane) n[4 * blk + lane] = g[lane];
  }
}

/* The noise stream as a table (for comparing generators block by block):
   for samples s < n_samples, steps tau < H, blocks b < n_blocks, the Philox
   words of counter (b, tau, s, counter lo) and the four normals of block b
   from orc_normals, at ((s*H + tau)*n_blocks + b)*4 + j.  Either output may
   be NULL. */
void orc_noise_table(uint64_t seed, uint64_t counter, int n_samples, int H, int n_blocks, uint32_t *words,
                     double *normals) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  double *n = normals ? (double *)malloc(sizeof(double) * 4 * (size_t)n_blocks) : NULL;
  for (int s = 0; s < n_samples; ++s)
    for (int tau = 0; tau < H; ++tau) {
      const size_t base = ((size_t)s * (size_t)H + (size_t)tau) * (size_t)n_blocks * 4;
      if (words)
        for (int b = 0; b < n_blocks; ++b) {
          const uint32_t ctr[4] = {(uint32_t)b, (uint32_t)tau, (uint32_t)s, (uint32_t)counter};
          orc_philox4x32_10(ctr, key, words + base + 4 * (size_t)b);
        }
      if (n) {
        orc_normals(seed, counter, (uint32_t)s, (uint32_t)tau, 4 * n_blocks, n);
        memcpy(normals + base, n, sizeof(double) * 4 * (size_t)n_blocks);
      }
    }
  free(n);
}

/* ------------------------------------------------------------------ */
/* Tractor-trailer kinematics, explicit Euler (Sec. III-A,
   Eq. tt_discrete_kinematics), with acceleration a as input and the path
   progress psi integrated from nu. */
void orc_dynamics_step(const orc_params *P, const double x[7], const double u[3], double xn[7]) {
  const double px = x[0], py = x[1], th1 = x[2], th2 = x[3], v = x[4], delta = x[5], psi = x[6];
  const double a = u[0], omega = u[1], nu = u[2];
  const double Ts = P->Ts;
  xn[0] = px + Ts * v * cos(th1);
  xn[1] = py + Ts * v * sin(th1);
  xn[2] = th1 + Ts * v / P->l1 * tan(delta);
  xn[3] = th2 + Ts * v / P->l2 *
                    (sin(th1 - th2) - (P->lh / P->l1) * cos(th1 - th2) * tan(delta));
  xn[4] = v + Ts * a;
  xn[5] = delta + Ts * omega;
  xn[6] = psi + Ts * nu;
}

void orc_integrate(const orc_params *P, const double x0[7], const double *U, int H, double *traj) {
  memcpy(traj, x0, 7 * sizeof(double));
  for (int k = 0; k < H; ++k) orc_dynamics_step(P, traj + 7 * k, U + 3 * k, traj + 7 * (k + 1));
}

static double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ */
/* Integer power for the super-ellipse exponent. */
static double ipow(double base, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= base;
  return r;
}

static int obstacle_exponent(const double *obs) {
  double e = obs[5];
  int ei = (int)e;
  if ((double)ei != e || ei < 2 || (ei % 2) != 0) return -1;
  return ei;
}

/* Velocity of an obstacle row: zero for rows of 6, (vx, vy) for rows of 8. */
static void obstacle_velocity(const double *obs, int stride, double *vx, double *vy) {
  *vx = (stride >= 8) ? obs[6] : 0.0;
  *vy = (stride >= 8) ? obs[7] : 0.0;
}

/* Super-ellipse barrier (Sec. IV-C, Eq. barrier_function): semi-axes
   inflated by the footprint disc radius, coordinates rotated into the
   obstacle frame; a moving obstacle (predicted pedestrian) has its centre at
   c + t v at time t. */
double orc_obstacle_h_at(const orc_params *P, const double *obs, int stride, double t,
                         const double x[7]) {
  const int e = obstacle_exponent(obs);
  if (e < 0) return NAN;
  double vx, vy;
  obstacle_velocity(obs, stride, &vx, &vy);
  const double cx = obs[0] + t * vx, cy = obs[1] + t * vy;
  const double Ax = obs[2] + P->r_inflate, Ay = obs[3] + P->r_inflate;
  const double th_o = obs[4];
  const double xp = cos(th_o) * (x[0] - cx) + sin(th_o) * (x[1] - cy);
  const double yp = -sin(th_o) * (x[0] - cx) + cos(th_o) * (x[1] - cy);
  return ipow(xp / Ax, e) + ipow(yp / Ay, e) - 1.0;
}

double orc_obstacle_h(const orc_params *P, const double obs[6], const double x[7]) {
  return orc_obstacle_h_at(P, obs, 6, 0.0, x);
}

/* Barrier-rate equality row for one obstacle (Eq. cbf_equality with the
   second-order expansion of Eq. barrier_function_approx).
   Along the continuous field with the input held, the rear-axle point
   moves with  pdot = v (cos th1, sin th1)  and
   pddot = a (cos th1, sin th1) + v * th1dot * (-sin th1, cos th1),
   th1dot = v tan(delta) / l1, while the obstacle centre moves at the
   constant velocity c_dot (zero for a parked vehicle).  With h = h(x', y')
   of the relative position p - c:
   hdot  = grad h . (pdot - c_dot)',
   hddot = grad h . pddot' + (pdot - c_dot)'^T Hess h (pdot - c_dot)'.
   hddot is affine in a; steer rate and progress rate do not enter at second
   order.  Row: A_u = (Ts^2/2 * dhddot/da, 0, 0) and
   b = -alpha h - Ts hdot - Ts^2/2 hddot|_{a=0}. */
void orc_obstacle_row_at(const orc_params *P, const double *obs, int stride, double t,
                         const double x[7], double A_u[3], double *h, double *b_rest) {
  const int e = obstacle_exponent(obs);
  double vx, vy;
  obstacle_velocity(obs, stride, &vx, &vy);
  const double cx = obs[0] + t * vx, cy = obs[1] + t * vy;
  const double Ax = obs[2] + P->r_inflate, Ay = obs[3] + P->r_inflate;
  const double th_o = obs[4];
  const double co = cos(th_o), so = sin(th_o);
  const double px = x[0], py = x[1], th1 = x[2], v = x[4], delta = x[5];
  const double Ts = P->Ts;

  /* rotate a world vector into the obstacle frame */
#define ROT_X(wx, wy) (co * (wx) + so * (wy))
#define ROT_Y(wx, wy) (-so * (wx) + co * (wy))
  const double xp = ROT_X(px - cx, py - cy);
  const double yp = ROT_Y(px - cx, py - cy);

  /* derivatives of h in obstacle-frame coordinates */
  const double Axe = ipow(Ax, e), Aye = ipow(Ay, e);
  const double hval = ipow(xp, e) / Axe + ipow(yp, e) / Aye - 1.0;
  const double hx = e * ipow(xp, e - 1) / Axe;
  const double hy = e * ipow(yp, e - 1) / Aye;
  const double hxx = e * (e - 1) * ipow(xp, e - 2) / Axe;
  const double hyy = e * (e - 1) * ipow(yp, e - 2) / Aye;

  const double c1 = cos(th1), s1 = sin(th1);
  const double th1dot = v * tan(delta) / P->l1;
  /* relative velocity, and the two parts of the acceleration */
  const double vel_x = ROT_X(v * c1 - vx, v * s1 - vy), vel_y = ROT_Y(v * c1 - vx, v * s1 - vy);
  const double dir_x = ROT_X(c1, s1), dir_y = ROT_Y(c1, s1); /* multiplies a */
  const double cen_x = ROT_X(-v * th1dot * s1, v * th1dot * c1);
  const double cen_y = ROT_Y(-v * th1dot * s1, v * th1dot * c1);
#undef ROT_X
#undef ROT_Y

  const double hdot = hx * vel_x + hy * vel_y;
  const double hddot_0 = hx * cen_x + hy * cen_y + hxx * vel_x * vel_x + hyy * vel_y * vel_y;
  const double dhddot_da = hx * dir_x + hy * dir_y;

  A_u[0] = 0.5 * Ts * Ts * dhddot_da;
  A_u[1] = 0.0;
  A_u[2] = 0.0;
  *h = hval;
  *b_rest = -Ts * hdot - 0.5 * Ts * Ts * hddot_0;
}

void orc_obstacle_row(const orc_params *P, const double obs[6], const double x[7],
                      double A_u[3], double *h, double *b_rest) {
  orc_obstacle_row_at(P, obs, 6, 0.0, x, A_u, h, b_rest);
}

/* Third-order row (the expansion of Eq. barrier_function_approx carried one
   order further, which brings the steer rate into obstacle rows).  With the
   input held, for the rear-axle point and w = pdot - c_dot:
     pddot  = a e1 + v th1dot n1,
     pdddot = 2 a th1dot n1 + v th1ddot n1 - v th1dot^2 e1,
     th1ddot = (a t + v (1 + t^2) omega) / l1,
     hdddot = grad h . pdddot + 3 w^T Hess h pddot + D3 h [w, w, w],
   D3 h [w, w, w] = h_xxx w_x^3 + h_yyy w_y^3 in the obstacle frame.  All
   three are affine in (a, omega); the coefficients are read off by
   evaluating the increment at unit inputs, as for the hitch row. */
static double point_increment3(const orc_params *P, const double *obs, int stride, double t,
                               const double x[7], double a, double omega) {
  const int e = obstacle_exponent(obs);
  double vx, vy;
  obstacle_velocity(obs, stride, &vx, &vy);
  const double cx = obs[0] + t * vx, cy = obs[1] + t * vy;
  const double Ax = obs[2] + P->r_inflate, Ay = obs[3] + P->r_inflate;
  const double co = cos(obs[4]), so = sin(obs[4]);
  const double th1 = x[2], v = x[4], tn = tan(x[5]);
  const double th1dot = v * tn / P->l1;
  const double th1ddot = (a * tn + v * (1.0 + tn * tn) * omega) / P->l1;
  const double e1[2] = {cos(th1), sin(th1)}, n1[2] = {-sin(th1), cos(th1)};
  double w[2], acc[2], jerk[2];
  for (int j = 0; j < 2; ++j) {
    w[j] = v * e1[j] - (j == 0 ? vx : vy);
    acc[j] = a * e1[j] + v * th1dot * n1[j];
    jerk[j] = 2.0 * a * th1dot * n1[j] + v * th1ddot * n1[j] - v * th1dot * th1dot * e1[j];
  }
  /* into the obstacle frame */
  const double rx = x[0] - cx, ry = x[1] - cy;
  const double xp = co * rx + so * ry, yp = -so * rx + co * ry;
  const double wx = co * w[0] + so * w[1], wy = -so * w[0] + co * w[1];
  const double ax_ = co * acc[0] + so * acc[1], ay_ = -so * acc[0] + co * acc[1];
  const double jx = co * jerk[0] + so * jerk[1], jy = -so * jerk[0] + co * jerk[1];
  const double Axe = ipow(Ax, e), Aye = ipow(Ay, e);
  const double hx = e * ipow(xp, e - 1) / Axe, hy = e * ipow(yp, e - 1) / Aye;
  const double hxx = e * (e - 1) * ipow(xp, e - 2) / Axe, hyy = e * (e - 1) * ipow(yp, e - 2) / Aye;
  const double hxxx = e * (e - 1) * (e - 2) * (e >= 3 ? ipow(xp, e - 3) : 0.0) / Axe;
  const double hyyy = e * (e - 1) * (e - 2) * (e >= 3 ? ipow(yp, e - 3) : 0.0) / Aye;
  const double hdot = hx * wx + hy * wy;
  const double hddot = hx * ax_ + hy * ay_ + hxx * wx * wx + hyy * wy * wy;
  const double hdddot = hx * jx + hy * jy + 3.0 * (hxx * wx * ax_ + hyy * wy * ay_) +
                        hxxx * wx * wx * wx + hyyy * wy * wy * wy;
  const double Ts = P->Ts;
  return Ts * hdot + 0.5 * Ts * Ts * hddot + Ts * Ts * Ts / 6.0 * hdddot;
}

void orc_obstacle_row3(const orc_params *P, const double *obs, int stride, double t,
                       const double x[7], double A_u[3], double *h, double *b_rest) {
  const double c0 = point_increment3(P, obs, stride, t, x, 0.0, 0.0);
  A_u[0] = point_increment3(P, obs, stride, t, x, 1.0, 0.0) - c0;
  A_u[1] = point_increment3(P, obs, stride, t, x, 0.0, 1.0) - c0;
  A_u[2] = 0.0;
  *h = orc_obstacle_h_at(P, obs, stride, t, x);
  *b_rest = -c0;
}

/* ------------------------------------------------------------------ */
/* Jerk-input model: the paper's own form of the kinematics, where the
   longitudinal acceleration a is a state integrated from the jerk.  Explicit
   Euler with every right-hand side at step k, as for the acceleration model;
   the extra state is x[7] = a. */
void orc_jerk_step(const orc_params *P, const double x[8], const double u[3], double xn[8]) {
  const double ua[3] = {x[7], u[1], u[2]}; /* the acceleration drives the speed */
  orc_dynamics_step(P, x, ua, xn);
  xn[7] = x[7] + P->Ts * u[0];
}

void orc_jerk_integrate(const orc_params *P, const double x0[8], const double *U, int H,
                        double *traj) {
  memcpy(traj, x0, 8 * sizeof(double));
  for (int k = 0; k < H; ++k) orc_jerk_step(P, traj + 8 * k, U + 3 * k, traj + 8 * (k + 1));
}

/* Hitch barrier along the jerk model with the input held: a is a state,
     hdot  = -kappa a - sigma (th2dot - th1dot),
     hddot = -kappa jerk - sigma (th2ddot - th1ddot),
   th1ddot, th2ddot as for the acceleration model with a the state value.
   Affine in (jerk, omega); read off at unit inputs. */
static double jerk_hitch_increment(const orc_params *P, const double x[8], double jerk, double omega) {
  const double th1 = x[2], th2 = x[3], v = x[4], delta = x[5], a = x[7];
  const double Delta = th2 - th1;
  const double sigma = (Delta >= 0.0) ? 1.0 : -1.0;
  const double phi = th1 - th2;
  const double t = tan(delta);
  const double k = P->lh / P->l1;
  const double G = sin(phi) - k * cos(phi) * t;
  const double th1dot = v * t / P->l1;
  const double th2dot = v * G / P->l2;
  const double phidot = th1dot - th2dot;
  const double th1ddot = (a * t + v * (1.0 + t * t) * omega) / P->l1;
  const double th2ddot =
      a * G / P->l2 +
      v / P->l2 * ((cos(phi) + k * t * sin(phi)) * phidot - k * cos(phi) * (1.0 + t * t) * omega);
  const double hdot = -P->kappa * a - sigma * (th2dot - th1dot);
  const double hddot = -P->kappa * jerk - sigma * (th2ddot - th1ddot);
  return P->Ts * hdot + 0.5 * P->Ts * P->Ts * hddot;
}

void orc_jerk_hitch_row(const orc_params *P, const double x[8], double A_u[3], double *h,
                        double *b_rest) {
  const double c0 = jerk_hitch_increment(P, x, 0.0, 0.0);
  A_u[0] = jerk_hitch_increment(P, x, 1.0, 0.0) - c0;
  A_u[1] = jerk_hitch_increment(P, x, 0.0, 1.0) - c0;
  A_u[2] = 0.0;
  *h = orc_hitch_h(P, x);
  *b_rest = -c0;
}

/* Obstacle at the rear axle along the jerk model, input held:
     pddot  = a e1 + v th1dot n1                           (no input),
     pdddot = jerk e1 + 2 a th1dot n1 + v th1ddot n1 - v th1dot^2 e1,
     th1ddot = (a t + v (1 + t^2) omega) / l1;
   second order carries no input (relative degree 3), third order brings
   the jerk and the steer rate in. */
static double jerk_point_increment(const orc_params *P, const double *obs, int stride, double t,
                                   const double x[8], double jerk, double omega) {
  const int e = obstacle_exponent(obs);
  double vx, vy;
  obstacle_velocity(obs, stride, &vx, &vy);
  const double cx = obs[0] + t * vx, cy = obs[1] + t * vy;
  const double Ax = obs[2] + P->r_inflate, Ay = obs[3] + P->r_inflate;
  const double co = cos(obs[4]), so = sin(obs[4]);
  const double th1 = x[2], v = x[4], tn = tan(x[5]), a = x[7];
  const double th1dot = v * tn / P->l1;
  const double th1ddot = (a * tn + v * (1.0 + tn * tn) * omega) / P->l1;
  const double e1[2] = {cos(th1), sin(th1)}, n1[2] = {-sin(th1), cos(th1)};
  double w[2], acc[2], jk[2];
  for (int j = 0; j < 2; ++j) {
    w[j] = v * e1[j] - (j == 0 ? vx : vy);
    acc[j] = a * e1[j] + v * th1dot * n1[j];
    jk[j] = jerk * e1[j] + 2.0 * a * th1dot * n1[j] + v * th1ddot * n1[j] - v * th1dot * th1dot * e1[j];
  }
  const double rx = x[0] - cx, ry = x[1] - cy;
  const double xp = co * rx + so * ry, yp = -so * rx + co * ry;
  const double wx = co * w[0] + so * w[1], wy = -so * w[0] + co * w[1];
  const double ax_ = co * acc[0] + so * acc[1], ay_ = -so * acc[0] + co * acc[1];
  const double jx = co * jk[0] + so * jk[1], jy = -so * jk[0] + co * jk[1];
  const double Axe = ipow(Ax, e), Aye = ipow(Ay, e);
  const double hx = e * ipow(xp, e - 1) / Axe, hy = e * ipow(yp, e - 1) / Aye;
  const double hxx = e * (e - 1) * ipow(xp, e - 2) / Axe, hyy = e * (e - 1) * ipow(yp, e - 2) / Aye;
  const double hxxx = e * (e - 1) * (e - 2) * (e >= 3 ? ipow(xp, e - 3) : 0.0) / Axe;
  const double hyyy = e * (e - 1) * (e - 2) * (e >= 3 ? ipow(yp, e - 3) : 0.0) / Aye;
  const double hdot = hx * wx + hy * wy;
  const double hddot = hx * ax_ + hy * ay_ + hxx * wx * wx + hyy * wy * wy;
  const double Ts = P->Ts;
  double inc = Ts * hdot + 0.5 * Ts * Ts * hddot;
  if (P->flags & ORC_THIRD_ORDER) {
    const double hdddot = hx * jx + hy * jy + 3.0 * (hxx * wx * ax_ + hyy * wy * ay_) +
                          hxxx * wx * wx * wx + hyyy * wy * wy * wy;
    inc += Ts * Ts * Ts / 6.0 * hdddot;
  }
  return inc;
}

void orc_jerk_obstacle_row(const orc_params *P, const double *obs, int stride, double t,
                           const double x[8], double A_u[3], double *h, double *b_rest) {
  const double c0 = jerk_point_increment(P, obs, stride, t, x, 0.0, 0.0);
  A_u[0] = jerk_point_increment(P, obs, stride, t, x, 1.0, 0.0) - c0;
  A_u[1] = jerk_point_increment(P, obs, stride, t, x, 0.0, 1.0) - c0;
  A_u[2] = 0.0;
  *h = orc_obstacle_h_at(P, obs, stride, t, x);
  *b_rest = -c0;
}

/* ------------------------------------------------------------------ */
/* Footprint discs.  Heading accelerations along the field with the input
   held (a, omega constant): with t = tan(delta), phi = th1 - th2,
   k = lh / l1, G = sin(phi) - k cos(phi) t,
     th1dot  = v t / l1,                 th1ddot = (a t + v (1 + t^2) omega) / l1,
     th2dot  = v G / l2,
     th2ddot = a G / l2 + v / l2 ((cos(phi) + k t sin(phi)) phidot
                                  - k cos(phi) (1 + t^2) omega).
   Tractor disc p_d = p + d e1:
     pdot  = v e1 + d th1dot n1,
     pddot = a e1 + v th1dot n1 + d th1ddot n1 - d th1dot^2 e1;
   trailer disc p_d = p - lh e1 - L e2, L = l2 - d:
     pdot  = v e1 - lh th1dot n1 - L th2dot n2,
     pddot = a e1 + v th1dot n1 - lh th1ddot n1 + lh th1dot^2 e1
             - L th2ddot n2 + L th2dot^2 e2,
   with n1, n2 the headings turned by +90 degrees. */
typedef struct {
  double pos[2], vel[2];
  double acc0[2], acc_a[2], acc_w[2]; /* pddot = acc0 + a acc_a + omega acc_w */
} disc_motion;

static void disc_kinematics(const orc_params *P, int m, const double x[7], disc_motion *dm) {
  const double th1 = x[2], th2 = x[3], v = x[4], delta = x[5];
  const double e1[2] = {cos(th1), sin(th1)}, n1[2] = {-sin(th1), cos(th1)};
  const double e2[2] = {cos(th2), sin(th2)}, n2[2] = {-sin(th2), cos(th2)};
  const double t = tan(delta), sec2 = 1.0 + t * t;
  const double phi = th1 - th2, k = P->lh / P->l1;
  const double G = sin(phi) - k * cos(phi) * t;
  const double th1dot = v * t / P->l1, th2dot = v * G / P->l2;
  const double phidot = th1dot - th2dot;
  /* heading accelerations: constant part, coefficient of a, of omega */
  const double a1_0 = 0.0, a1_a = t / P->l1, a1_w = v * sec2 / P->l1;
  const double a2_0 = v / P->l2 * (cos(phi) + k * t * sin(phi)) * phidot;
  const double a2_a = G / P->l2, a2_w = -v / P->l2 * k * cos(phi) * sec2;
  const double d = P->disc_off[m];
  const int on_trailer = (P->disc_trailer_mask >> m) & 1;
  for (int j = 0; j < 2; ++j) {
    if (!on_trailer) {
      dm->pos[j] = x[j] + d * e1[j];
      dm->vel[j] = v * e1[j] + d * th1dot * n1[j];
      dm->acc0[j] = v * th1dot * n1[j] + d * a1_0 * n1[j] - d * th1dot * th1dot * e1[j];
      dm->acc_a[j] = e1[j] + d * a1_a * n1[j];
      dm->acc_w[j] = d * a1_w * n1[j];
    } else {
      const double L = P->l2 - d;
      dm->pos[j] = x[j] - P->lh * e1[j] - L * e2[j];
      dm->vel[j] = v * e1[j] - P->lh * th1dot * n1[j] - L * th2dot * n2[j];
      dm->acc0[j] = v * th1dot * n1[j] - P->lh * a1_0 * n1[j] + P->lh * th1dot * th1dot * e1[j] -
                    L * a2_0 * n2[j] + L * th2dot * th2dot * e2[j];
      dm->acc_a[j] = e1[j] - P->lh * a1_a * n1[j] - L * a2_a * n2[j];
      dm->acc_w[j] = -P->lh * a1_w * n1[j] - L * a2_w * n2[j];
    }
  }
}

void orc_disc_position(const orc_params *P, int m, const double x[7], double pos[2]) {
  disc_motion dm;
  disc_kinematics(P, m, x, &dm);
  pos[0] = dm.pos[0];
  pos[1] = dm.pos[1];
}

double orc_disc_h(const orc_params *P, const double *obs, int stride, double t, int m,
                  const double x[7]) {
  double xd[7];
  memcpy(xd, x, sizeof(xd));
  orc_disc_position(P, m, x, xd);
  return orc_obstacle_h_at(P, obs, stride, t, xd);
}

/* Row of obstacle `obs` seen from disc m: the super-ellipse of the relative
   position p_d - c(t), hdot = grad h . (pdot - c_dot)',
   hddot = grad h . pddot' + (pdot - c_dot)'^T Hess h (pdot - c_dot)',
   affine in (a, omega). */
void orc_disc_row(const orc_params *P, const double *obs, int stride, double t, int m,
                  const double x[7], double A_u[3], double *h, double *b_rest) {
  const int e = obstacle_exponent(obs);
  double vx, vy;
  obstacle_velocity(obs, stride, &vx, &vy);
  disc_motion dm;
  disc_kinematics(P, m, x, &dm);
  const double cx = obs[0] + t * vx, cy = obs[1] + t * vy;
  const double Ax = obs[2] + P->r_inflate, Ay = obs[3] + P->r_inflate;
  const double co = cos(obs[4]), so = sin(obs[4]);
#define DROT_X(wx, wy) (co * (wx) + so * (wy))
#define DROT_Y(wx, wy) (-so * (wx) + co * (wy))
  const double xp = DROT_X(dm.pos[0] - cx, dm.pos[1] - cy);
  const double yp = DROT_Y(dm.pos[0] - cx, dm.pos[1] - cy);
  const double Axe = ipow(Ax, e), Aye = ipow(Ay, e);
  const double hx = e * ipow(xp, e - 1) / Axe, hy = e * ipow(yp, e - 1) / Aye;
  const double hxx = e * (e - 1) * ipow(xp, e - 2) / Axe, hyy = e * (e - 1) * ipow(yp, e - 2) / Aye;
  const double wx = DROT_X(dm.vel[0] - vx, dm.vel[1] - vy), wy = DROT_Y(dm.vel[0] - vx, dm.vel[1] - vy);
  const double c0x = DROT_X(dm.acc0[0], dm.acc0[1]), c0y = DROT_Y(dm.acc0[0], dm.acc0[1]);
  const double cax = DROT_X(dm.acc_a[0], dm.acc_a[1]), cay = DROT_Y(dm.acc_a[0], dm.acc_a[1]);
  const double cwx = DROT_X(dm.acc_w[0], dm.acc_w[1]), cwy = DROT_Y(dm.acc_w[0], dm.acc_w[1]);
#undef DROT_X
#undef DROT_Y
  const double hdot = hx * wx + hy * wy;
  const double hddot_0 = hx * c0x + hy * c0y + hxx * wx * wx + hyy * wy * wy;
  A_u[0] = 0.5 * P->Ts * P->Ts * (hx * cax + hy * cay);
  A_u[1] = 0.5 * P->Ts * P->Ts * (hx * cwx + hy * cwy);
  A_u[2] = 0.0;
  *h = ipow(xp / Ax, e) + ipow(yp / Ay, e) - 1.0;
  *b_rest = -P->Ts * hdot - 0.5 * P->Ts * P->Ts * hddot_0;
}

/* Standard MPPI with a collision cost (the comparison method of Sec. V):
   each obstacle the state penetrates adds q_coll times its depth -h_o (a
   hinge, zero outside). */
double orc_collision_cost(const orc_params *P, const double *obs, int stride, int n_obs, double t,
                          const double x[7]) {
  double c = 0.0;
  for (int o = 0; o < n_obs; ++o)
    for (int m = 0; m < P->n_discs; ++m) {
      const double h = orc_disc_h(P, obs + (size_t)stride * (size_t)o, stride, t, m, x);
      if (h < 0.0) c += -h;
    }
  return P->q_coll * c;
}

/* Buffer-zone cost of BR-MPPI (Sec. IV-A): positive barrier rates are
   charged near an obstacle, pushing the sampled rates negative there (hdot
   >= 0 close to the boundary).  The zone weight falls linearly from 1 at
   h = 0 to 0 at h = h_buf. */
double orc_alpha_buffer_cost(const orc_params *P, int n, const double *h, const double *alpha) {
  double c = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = 1.0 - h[i] / P->h_buf;
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    const double ap = alpha[i] > 0.0 ? alpha[i] : 0.0;
    c += w * ap * ap;
  }
  return P->q_abuf * c;
}

/* Hitch-angle barrier (Sec. IV-D, Eq. hitch_angle_barrier):
   h_h = dtheta_max - kappa v - |th2 - th1|. */
double orc_hitch_h(const orc_params *P, const double x[7]) {
  return P->dtheta_max - P->kappa * x[4] - fabs(x[3] - x[2]);
}

/* Barrier-rate row of the hitch barrier, second-order expansion as for the
   obstacles.  With Delta = th2 - th1, sigma = sgn(Delta) (sgn(0) = +1),
   phi = th1 - th2, t = tan(delta), k = lh/l1:
     th1dot = v t / l1,  G = sin(phi) - k cos(phi) t,  th2dot = v G / l2,
     hdot   = -kappa a - sigma (th2dot - th1dot),
     hddot  = -sigma (th2ddot - th1ddot)          (a held: vddot = 0)
     th1ddot = (a t + v (1 + t^2) omega) / l1
     th2ddot = a G / l2 + v / l2 * ((cos(phi) + k t sin(phi)) phidot
                                    - k cos(phi) (1 + t^2) omega)
   which is affine in (a, omega).  The row coefficients are read off by
   evaluating Ts hdot + Ts^2/2 hddot at unit inputs. */
static double hitch_increment(const orc_params *P, const double x[7], double a, double omega) {
  const double th1 = x[2], th2 = x[3], v = x[4], delta = x[5];
  const double Delta = th2 - th1;
  const double sigma = (Delta >= 0.0) ? 1.0 : -1.0;
  const double phi = th1 - th2;
  const double t = tan(delta);
  const double k = P->lh / P->l1;
  const double G = sin(phi) - k * cos(phi) * t;
  const double th1dot = v * t / P->l1;
  const double th2dot = v * G / P->l2;
  const double phidot = th1dot - th2dot;
  const double th1ddot = (a * t + v * (1.0 + t * t) * omega) / P->l1;
  const double th2ddot =
      a * G / P->l2 +
      v / P->l2 * ((cos(phi) + k * t * sin(phi)) * phidot - k * cos(phi) * (1.0 + t * t) * omega);
  const double hdot = -P->kappa * a - sigma * (th2dot - th1dot);
  const double hddot = -sigma * (th2ddot - th1ddot);
  return P->Ts * hdot + 0.5 * P->Ts * P->Ts * hddot;
}

void orc_hitch_row(const orc_params *P, const double x[7], double A_u[3], double *h, double *b_rest) {
  const double c0 = hitch_increment(P, x, 0.0, 0.0);
  const double ca = hitch_increment(P, x, 1.0, 0.0) - c0;
  const double cw = hitch_increment(P, x, 0.0, 1.0) - c0;
  A_u[0] = ca;
  A_u[1] = cw;
  A_u[2] = 0.0;
  *h = orc_hitch_h(P, x);
  *b_rest = -c0;
}

/* Hitch-angle stabilizer (Sec. IV-D, Eq. hitch_angle_qp): after BR-MPPI,
   the reference input u_ref = (a, omega, nu) is moved to
     argmin (u - u_ref)^T Q_h (u - u_ref)  over (a, omega) in the input box
     s.t.  Ts hdot + Ts^2/2 hddot >= -alpha_stab h_h(x),
   the discrete CBF condition (Eq. barrier_constraint_prelim, with the sign
   of Eq. cbf_equality and the same second-order increment as the rollout's
   hitch row, g . u + c0).  nu does not move the vehicle and passes through.
   KKT for a diagonal Q_h and a box: if the box projection of u_ref meets the
   condition it is the minimiser; otherwise the condition is active and
   u(mu) = clip(u_ref + mu Q_h^-1 g) with the smallest mu >= 0 that meets it.
   g . u(mu) is continuous and non-decreasing in mu, so mu is found by
   bisection. */
int orc_hitch_stabilize(const orc_params *P, const double *x, const double u_ref[3],
                        double u_out[3], double *slack) {
  double A_u[3], h, b_rest;
  if (P->flags & ORC_JERK) /* the paper's inputs: (jerk, omega); x holds the acceleration */
    orc_jerk_hitch_row(P, x, A_u, &h, &b_rest);
  else
    orc_hitch_row(P, x, A_u, &h, &b_rest);
  const double g[2] = {A_u[0], A_u[1]};
  const double c0 = -b_rest;
  const double rhs = -P->alpha_stab * h - c0; /* need g . u >= rhs */
  double u[2];
  int infeasible = 0;
  for (int j = 0; j < 2; ++j) u[j] = clip(u_ref[j], P->z_lo[j], P->z_hi[j]);
  if (g[0] * u[0] + g[1] * u[1] < rhs) {
    double lo = 0.0, hi = 1.0, cand[2];
#define U_OF_MU(mu, out)                                                             \
  for (int j = 0; j < 2; ++j)                                                        \
    (out)[j] = clip(u_ref[j] + (mu) * g[j] / P->q_stab[j], P->z_lo[j], P->z_hi[j]);
    for (;;) {
      U_OF_MU(hi, cand);
      if (g[0] * cand[0] + g[1] * cand[1] >= rhs) break;
      lo = hi;
      hi *= 2.0;
      if (hi > 1e300) {
        infeasible = 1;
        break;
      }
    }
    if (infeasible) {
      /* no input in the box meets the condition: the one that comes closest */
      for (int j = 0; j < 2; ++j)
        u[j] = g[j] > 0.0 ? P->z_hi[j] : (g[j] < 0.0 ? P->z_lo[j] : clip(u_ref[j], P->z_lo[j], P->z_hi[j]));
    } else {
      for (int it = 0; it < 2000 && hi - lo > 1e-17 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        U_OF_MU(mid, cand);
        if (g[0] * cand[0] + g[1] * cand[1] >= rhs)
          hi = mid;
        else
          lo = mid;
      }
      U_OF_MU(hi, u);
    }
#undef U_OF_MU
  }
  u_out[0] = u[0];
  u_out[1] = u[1];
  u_out[2] = u_ref[2];
  if (slack) *slack = g[0] * u[0] + g[1] * u[1] - rhs;
  return infeasible;
}

/* ------------------------------------------------------------------ */
/* Dense linear algebra for the projection: Cholesky, with Gaussian
   elimination (partial pivoting) as the fallback. */
static int cholesky_solve(int n, double *K, double *rhs) {
  for (int j = 0; j < n; ++j) {
    double s = K[j * n + j];
    for (int k = 0; k < j; ++k) s -= K[j * n + k] * K[j * n + k];
    if (!(s > 0.0)) return -1;
    const double Ljj = sqrt(s);
    K[j * n + j] = Ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = K[i * n + j];
      for (int k = 0; k < j; ++k) t -= K[i * n + k] * K[j * n + k];
      K[i * n + j] = t / Ljj;
    }
  }
  for (int i = 0; i < n; ++i) { /* L y = rhs */
    double t = rhs[i];
    for (int k = 0; k < i; ++k) t -= K[i * n + k] * rhs[k];
    rhs[i] = t / K[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
    double t = rhs[i];
    for (int k = i + 1; k < n; ++k) t -= K[k * n + i] * rhs[k];
    rhs[i] = t / K[i * n + i];
  }
  return 0;
}

static int gauss_solve(int n, double *K, double *rhs) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(K[r * n + c]) > fabs(K[piv * n + c])) piv = r;
    if (K[piv * n + c] == 0.0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        double t = K[c * n + k];
        K[c * n + k] = K[piv * n + k];
        K[piv * n + k] = t;
      }
      double t = rhs[c];
      rhs[c] = rhs[piv];
      rhs[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = K[r * n + c] / K[c * n + c];
      for (int k = c; k < n; ++k) K[r * n + k] -= f * K[c * n + k];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double t = rhs[r];
    for (int k = r + 1; k < n; ++k) t -= K[r * n + k] * rhs[k];
    rhs[r] = t / K[r * n + r];
  }
  return 0;
}

/* Soft-bound projection (Sec. IV-A, Eq. softproj), closed form
   (Eq. closed-form_projection):
     M = W + rho I,   p = W z_des + rho/2 (z_hi + z_lo),
     z* = M^-1 [ p - A^T (A M^-1 A^T)^-1 (A M^-1 p - b) ]. */
int orc_project(int d, int nc, const double *A, const double *b, const double *w, double rho,
                const double *z_lo, const double *z_hi, const double *z_des, double *z_star) {
  double *Minv = (double *)malloc(sizeof(double) * (size_t)d);
  double *p = (double *)malloc(sizeof(double) * (size_t)d);
  double *K = (double *)malloc(sizeof(double) * (size_t)(nc * nc + 1));
  double *K2 = (double *)malloc(sizeof(double) * (size_t)(nc * nc + 1));
  double *lam = (double *)malloc(sizeof(double) * (size_t)(nc + 1));
  double *lam2 = (double *)malloc(sizeof(double) * (size_t)(nc + 1));
  int status = ORC_OK;
  for (int j = 0; j < d; ++j) {
    Minv[j] = 1.0 / (w[j] + rho);
    p[j] = w[j] * z_des[j] + 0.5 * rho * (z_hi[j] + z_lo[j]);
  }
  for (int i = 0; i < nc; ++i) {
    double t = 0.0;
    for (int j = 0; j < d; ++j) t += A[i * d + j] * Minv[j] * p[j];
    lam[i] = t - b[i]; /* A M^-1 p - b */
    for (int r = 0; r < nc; ++r) {
      double kk = 0.0;
      for (int j = 0; j < d; ++j) kk += A[i * d + j] * Minv[j] * A[r * d + j];
      K[i * nc + r] = kk; /* A M^-1 A^T */
    }
  }
  memcpy(K2, K, sizeof(double) * (size_t)(nc * nc));
  memcpy(lam2, lam, sizeof(double) * (size_t)nc);
  if (nc > 0 && cholesky_solve(nc, K, lam) != 0) {
    memcpy(lam, lam2, sizeof(double) * (size_t)nc);
    if (gauss_solve(nc, K2, lam) != 0) status = ORC_EINVAL;
  }
  if (status == ORC_OK) {
    for (int j = 0; j < d; ++j) {
      double t = p[j];
      for (int i = 0; i < nc; ++i) t -= A[i * d + j] * lam[i];
      z_star[j] = Minv[j] * t;
    }
  }
  free(Minv);
  free(p);
  free(K);
  free(K2);
  free(lam);
  free(lam2);
  return status;
}

/* ------------------------------------------------------------------ */
/* Reference path zeta(psi) parameterised by arc length (Sec. IV-B), read
   from a table sampled every ds: psi clamped to the table, linear
   interpolation of (x, y, theta). */
void orc_path_lookup(const double *path, int n, double ds, double psi, double *xr, double *yr,
                     double *thr) {
  const double psi_max = (double)(n - 1) * ds;
  double q = psi;
  if (q < 0.0) q = 0.0;
  if (q > psi_max) q = psi_max;
  int i = (int)floor(q / ds);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  const double f = q / ds - (double)i;
  const double *r0 = path + 3 * i, *r1 = path + 3 * (i + 1);
  *xr = r0[0] + f * (r1[0] - r0[0]);
  *yr = r0[1] + f * (r1[1] - r0[1]);
  *thr = r0[2] + f * (r1[2] - r0[2]);
}

static double wrap_angle(double a) {
  /* into (-pi, pi] */
  double r = fmod(a + M_PI, 2.0 * M_PI);
  if (r < 0.0) r += 2.0 * M_PI;
  r -= M_PI;
  if (r == -M_PI) r = M_PI;
  return r;
}

/* Contouring stage cost (Sec. IV-B, Eq. cost_function_contour with the
   errors of Eq. contour_lag_errors):
   r = Qc e_c^2 + Ql e_l^2 + Qth |e_theta|^2 + u^T R u + mu (nu_bar - nu)^2. */
double orc_stage_cost(const orc_params *P, const double x[7], const double u[3], const double *path,
                      int n, double ds) {
  double xr, yr, thr;
  orc_path_lookup(path, n, ds, x[6], &xr, &yr, &thr);
  const double e_c = sin(thr) * (x[0] - xr) - cos(thr) * (x[1] - yr);
  const double e_l = -cos(thr) * (x[0] - xr) - sin(thr) * (x[1] - yr);
  const double e_th1 = wrap_angle(x[2] - thr);
  const double e_th2 = wrap_angle(x[3] - thr);
  double r = P->Qc * e_c * e_c + P->Ql * e_l * e_l + P->Qth * (e_th1 * e_th1 + e_th2 * e_th2);
  for (int j = 0; j < 3; ++j) r += P->R[j] * u[j] * u[j];
  r += P->mu * (P->nu_bar - u[2]) * (P->nu_bar - u[2]);
  return r;
}

/* Importance weights of MPPI (Sec. II-B):
   gamma_s = exp(-(J_s - min J)/lambda), gamma_bar = gamma / sum gamma. */
int orc_softmin(int S, const double *J, double lambda, double *gamma_bar) {
  double Jmin = INFINITY;
  for (int s = 0; s < S; ++s)
    if (isfinite(J[s]) && J[s] < Jmin) Jmin = J[s];
  if (!isfinite(Jmin)) {
    for (int s = 0; s < S; ++s) gamma_bar[s] = 0.0;
    return ORC_ENONFINITE;
  }
  double sum = 0.0;
  for (int s = 0; s < S; ++s) {
    gamma_bar[s] = isfinite(J[s]) ? exp(-(J[s] - Jmin) / lambda) : 0.0;
    sum += gamma_bar[s];
  }
  for (int s = 0; s < S; ++s) gamma_bar[s] /= sum;
  return ORC_OK;
}


/* ------------------------------------------------------------------ */
/* One BR-MPPI rollout (Sec. IV-A): at every step sample z_des, build the
   barrier-rate rows at the current state, project, apply the clipped input,
   update the barrier rates alpha_{tau+1} = alpha_tau + u^alpha, step the
   kinematics and accumulate the stage cost. */
int orc_rollout_sample(const orc_params *P, const double *x0, const double *U_nom,
                       const double *obs, int n_obs, const double *path, int n_pts, double ds,
                       uint64_t seed, uint64_t counter, uint32_t s, double *states, double *u_out,
                       double *alpha_out, double *z_des_out, double *z_star_out, double *J_out) {
  const int H = P->H;
  const int nd = P->n_discs;
  const int Nc = 1 + n_obs * nd;
  const int d = 3 + Nc;
  const int proj = !(P->flags & ORC_PROJ_NONE);
  const int stride = (P->flags & ORC_OBS8) ? 8 : 6;
  for (int o = 0; o < n_obs; ++o)
    if (obstacle_exponent(obs + (size_t)stride * (size_t)o) < 0) return ORC_EINVAL;
  if (n_pts < 2 || !(ds > 0.0) || nd < 1 || nd > 8) return ORC_EINVAL;
  const int jerk = (P->flags & ORC_JERK) != 0;
  const int nx = jerk ? 8 : 7;
  if ((P->flags & (ORC_THIRD_ORDER | ORC_JERK)) &&
      (nd != 1 || P->disc_trailer_mask != 0 || P->disc_off[0] != 0.0))
    return ORC_EINVAL; /* offset discs: the rows are not affine in the input */

  double *n = (double *)malloc(sizeof(double) * (size_t)d);
  double *alpha = (double *)malloc(sizeof(double) * (size_t)Nc);
  double *A = (double *)calloc((size_t)(Nc * d), sizeof(double));
  double *b = (double *)malloc(sizeof(double) * (size_t)Nc);
  double *w = (double *)malloc(sizeof(double) * (size_t)d);
  double *zlo = (double *)malloc(sizeof(double) * (size_t)d);
  double *zhi = (double *)malloc(sizeof(double) * (size_t)d);
  double *zdes = (double *)malloc(sizeof(double) * (size_t)d);
  double *zs = (double *)malloc(sizeof(double) * (size_t)d);
  double *hrow = (double *)malloc(sizeof(double) * (size_t)Nc);
  for (int j = 0; j < 3; ++j) {
    w[j] = P->w_u[j];
    zlo[j] = P->z_lo[j];
    zhi[j] = P->z_hi[j];
  }
  for (int i = 0; i < Nc; ++i) {
    w[3 + i] = P->w_alpha;
    zlo[3 + i] = P->ua_lo;
    zhi[3 + i] = P->ua_hi;
    alpha[i] = P->alpha0;
  }
  double x[8] = {0}, xn[8] = {0}, u[3];
  memcpy(x, x0, sizeof(double) * (size_t)nx);
  if (states) memcpy(states, x0, sizeof(double) * (size_t)nx);
  if (alpha_out)
    for (int i = 0; i < Nc; ++i) alpha_out[i] = alpha[i];
  double J = 0.0;
  int status = ORC_OK;

  for (int tau = 0; tau < H; ++tau) {
    /* 1. noise and the sampled augmented input (perturbed nominal) */
    orc_normals(seed, counter, s, (uint32_t)tau, proj ? d : 3, n);
    for (int j = 0; j < 3; ++j)
      zdes[j] = clip(U_nom[3 * tau + j] + P->sigma[j] * n[j], P->z_lo[j], P->z_hi[j]);
    for (int i = 0; i < Nc; ++i)
      zdes[3 + i] = proj ? clip(P->sigma_alpha * n[3 + i], P->ua_lo, P->ua_hi) : 0.0;

    if (proj) {
      /* 2. barrier-rate equality rows A z = b at the current state */
      for (int i = 0; i < Nc; ++i) {
        double Au[3], h, b_rest;
        if (i == 0 && jerk)
          orc_jerk_hitch_row(P, x, Au, &h, &b_rest);
        else if (i == 0)
          orc_hitch_row(P, x, Au, &h, &b_rest);
        else if (jerk)
          orc_jerk_obstacle_row(P, obs + (size_t)stride * (size_t)(i - 1), stride, tau * P->Ts, x, Au,
                                &h, &b_rest);
        else if (P->flags & ORC_THIRD_ORDER)
          orc_obstacle_row3(P, obs + (size_t)stride * (size_t)(i - 1), stride, tau * P->Ts, x, Au, &h,
                            &b_rest);
        else
          orc_disc_row(P, obs + (size_t)stride * (size_t)((i - 1) / nd), stride, tau * P->Ts,
                       (i - 1) % nd, x, Au, &h, &b_rest);
        hrow[i] = h;
        const double hmag = fabs(h) > P->h_floor ? fabs(h) : P->h_floor;
        const double h_tilde = (h >= 0.0) ? hmag : -hmag;
        for (int j = 0; j < d; ++j) A[i * d + j] = 0.0;
        A[i * d + 0] = Au[0];
        A[i * d + 1] = Au[1];
        A[i * d + 2] = Au[2];
        A[i * d + 3 + i] = h_tilde;
        b[i] = -alpha[i] * h + b_rest;
      }
      /* 3. soft-bound projection */
      if (orc_project(d, Nc, A, b, w, P->rho, zlo, zhi, zdes, zs) != ORC_OK) {
        status = ORC_EINVAL;
        break;
      }
    } else {
      for (int j = 0; j < d; ++j) zs[j] = zdes[j];
    }
    if (z_des_out) memcpy(z_des_out + (size_t)d * tau, zdes, sizeof(double) * (size_t)d);
    if (z_star_out) memcpy(z_star_out + (size_t)d * tau, zs, sizeof(double) * (size_t)d);

    /* buffer cost of the obstacle rows just built: their h at this state
       and the rates alpha_tau they were built with */
    if (proj && (P->flags & ORC_ALPHA_BUFFER))
      J += orc_alpha_buffer_cost(P, n_obs * nd, hrow + 1, alpha + 1);

    /* 4. applied input (clipped) and barrier-rate update */
    for (int j = 0; j < 3; ++j) u[j] = clip(zs[j], P->z_lo[j], P->z_hi[j]);
    if (proj)
      for (int i = 0; i < Nc; ++i) alpha[i] += zs[3 + i];

    /* 5. kinematics and stage cost at the new state, and the comparison
       method's collision cost there */
    if (jerk)
      orc_jerk_step(P, x, u, xn);
    else
      orc_dynamics_step(P, x, u, xn);
    memcpy(x, xn, sizeof(x));
    J += orc_stage_cost(P, x, u, path, n_pts, ds);
    if (P->flags & ORC_COLLISION_COST)
      J += orc_collision_cost(P, obs, stride, n_obs, (tau + 1) * P->Ts, x);

    if (states) memcpy(states + (size_t)nx * (size_t)(tau + 1), x, sizeof(double) * (size_t)nx);
    if (u_out) memcpy(u_out + 3 * tau, u, sizeof(u));
    if (alpha_out)
      for (int i = 0; i < Nc; ++i) alpha_out[(size_t)Nc * (tau + 1) + i] = alpha[i];
  }
  if (J_out) *J_out = J;
  free(n);
  free(alpha);
  free(A);
  free(b);
  free(w);
  free(zlo);
  free(zhi);
  free(zdes);
  free(zs);
  free(hrow);
  return status;
}

/* ------------------------------------------------------------------ */
/* The solve: S rollouts, softmin weights, and the update of
   Eq. MPPI_update_rule over the applied inputs; then the optimal
   trajectory, x0 integrated with U*. */
/* The MPPI update (Sec. II-B, Eq. MPPI_update_rule): softmin weights of the
   costs, then U*[k] = sum_s gamma_bar_s u_s[k] over the applied inputs, in
   sample order.  No finite cost: U_out = U_nom and ORC_ENONFINITE.
   gamma_bar: S doubles of workspace (the weights on return). */
int orc_update(int S, int H, const double *J, const double *u_hist, double lambda,
               const double *U_nom, double *gamma_bar, double *U_out) {
  const int status = orc_softmin(S, J, lambda, gamma_bar);
  if (status == ORC_OK) {
    for (int k = 0; k < 3 * H; ++k) {
      double acc = 0.0;
      for (int s = 0; s < S; ++s) acc += gamma_bar[s] * u_hist[(size_t)s * (size_t)H * 3 + (size_t)k];
      U_out[k] = acc;
    }
  } else {
    for (int k = 0; k < 3 * H; ++k) U_out[k] = U_nom[k];
  }
  return status;
}

/* Rollouts of samples s0 .. s1-1 (each exactly as orc_rollout_sample):
   J_out (s1 - s0), u_hist (s1 - s0)*H*3, states_out (s1 - s0)*(H+1)*NX;
   u_hist and states_out may be NULL.  Lets a caller spread one solve's
   samples over several processes. */
int orc_rollout_range(const orc_params *P, const double *x0, const double *U_nom, const double *obs,
                      int n_obs, const double *path, int n_pts, double ds, uint64_t seed,
                      uint64_t counter, uint32_t s0, uint32_t s1, double *J_out, double *u_hist,
                      double *states_out) {
  const int H = P->H;
  const int nx = (P->flags & ORC_JERK) ? 8 : 7;
  for (uint32_t s = s0; s < s1; ++s) {
    const size_t i = (size_t)(s - s0);
    const int st = orc_rollout_sample(P, x0, U_nom, obs, n_obs, path, n_pts, ds, seed, counter, s,
                                      states_out ? states_out + i * (size_t)(H + 1) * (size_t)nx : NULL,
                                      u_hist ? u_hist + i * (size_t)H * 3 : NULL, NULL, NULL, NULL,
                                      &J_out[i]);
    if (st != ORC_OK) return st;
  }
  return ORC_OK;
}

int orc_solve(const orc_params *P, const double *x0, const double *U_nom, const double *obs,
              int n_obs, const double *path, int n_pts, double ds, uint64_t seed,
              uint64_t counter, double *U_out, double *traj_out, double *J_out, double *u_hist,
              double *states_out) {
  const int S = P->S, H = P->H;
  const int nx = (P->flags & ORC_JERK) ? 8 : 7;
  if (S <= 0 || H <= 0 || n_obs < 0 || n_pts < 2) return ORC_EINVAL;
  double *J = (double *)malloc(sizeof(double) * (size_t)S);
  double *uh = u_hist ? u_hist : (double *)malloc(sizeof(double) * (size_t)S * (size_t)H * 3);
  double *gb = (double *)malloc(sizeof(double) * (size_t)S);
  int status = ORC_OK;
  for (int s = 0; s < S && status == ORC_OK; ++s) {
    status = orc_rollout_sample(P, x0, U_nom, obs, n_obs, path, n_pts, ds, seed, counter,
                                (uint32_t)s,
                                states_out ? states_out + (size_t)s * (size_t)(H + 1) * (size_t)nx
                                           : NULL,
                                uh + (size_t)s * (size_t)H * 3, NULL, NULL, NULL, &J[s]);
  }
  if (status == ORC_OK) {
    status = orc_update(S, H, J, uh, P->lambda, U_nom, gb, U_out);
    if (traj_out) {
      if (P->flags & ORC_JERK)
        orc_jerk_integrate(P, x0, U_out, H, traj_out);
      else
        orc_integrate(P, x0, U_out, H, traj_out);
    }
    if (J_out) memcpy(J_out, J, sizeof(double) * (size_t)S);
  }
  free(J);
  free(gb);
  if (!u_hist) free(uh);
  return status;
}
