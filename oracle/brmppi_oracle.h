/*
 * brmppi_oracle.h -- plain FP64 CPU oracle for one BR-MPPI control solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, step-by-step restatement of
 * the method that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no source, header, helper or constant table with the CUDA
 * library: every formula here is written out again from the paper.
 *
 * Paper: "GPU-Accelerated Barrier-Rate Guided MPPI Control for
 * Tractor-Trailer Systems" (arXiv 2508.05773).  Section / equation labels
 * below are the paper's.
 *
 * Conventions (identical to the CUDA path's inputs, not its code):
 *   state  x = (px, py, th1, th2, v, delta, psi)             7 doubles
 *   input  u = (a, omega, nu)                                3 doubles
 *   augmented z = (a, omega, nu, ua_0 .. ua_{Nc-1})          d = 3 + Nc
 *   constraint 0 is the hitch-angle barrier, 1..No the obstacles
 *   obstacle row  (cx, cy, mx, my, theta_o, e)                6 doubles
 *   path row      (x, y, theta_unwrapped) at arc length j*ds  3 doubles
 *
 * All functions are pure; none keeps state between calls.
 */
#ifndef BRMPPI_ORACLE_H
#define BRMPPI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENONFINITE (-5)

/* flags */
#define ORC_PROJ_NONE 1      /* standard MPPI: skip the barrier-rate projection */
#define ORC_COLLISION_COST 2 /* add q_coll * sum_o max(0, -h_o) to the stage cost */
#define ORC_OBS8 4           /* obstacle rows of 8: (cx, cy, mx, my, theta_o, e, vx, vy),
                                the centre moving at (vx, vy) from t = 0 */
#define ORC_ALPHA_BUFFER 8   /* barrier-rate buffer cost on the obstacle rows */
#define ORC_THIRD_ORDER 16   /* obstacle rows to third order (one rear-axle disc only) */
#define ORC_JERK 32          /* jerk-input model: state (px, py, th1, th2, v, delta, psi, a),
                                input (jerk, omega, nu); one rear-axle disc only */

typedef struct {
  int32_t S, H, flags;
  double Ts, lambda;                  /* sample time, softmin temperature */
  double l1, lh, l2;                  /* wheelbase, hitch offset, trailer length */
  double dtheta_max, kappa;           /* hitch limit  dtheta_max - kappa * v */
  double r_inflate;                   /* footprint disc radius added to semi-axes */
  double Qc, Ql, Qth, R[3], mu, nu_bar; /* contouring cost weights */
  double z_lo[3], z_hi[3], sigma[3];  /* input bounds and noise std */
  double alpha0, sigma_alpha, ua_lo, ua_hi; /* barrier-rate variables */
  double w_u[3], w_alpha, rho, h_floor;     /* projection weights */
  double q_coll;                      /* collision-cost weight (ORC_COLLISION_COST) */
  double alpha_stab, q_stab[2];       /* hitch stabilizer: CBF rate, Q_h on (a, omega) */
  double q_abuf, h_buf;               /* buffer cost weight and zone width (ORC_ALPHA_BUFFER) */
  int32_t n_discs;                    /* footprint discs (>= 1) */
  int32_t disc_trailer_mask;          /* bit m: disc m sits on the trailer */
  double disc_off[8];                 /* disc m: offset along its body's heading from the
                                         tractor rear axle / the trailer axle */
} orc_params;

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Standard normals n[0..d) of sample s at step tau (noise mapping of the
   solve: key = seed, counter = (q/4, tau, s, counter mod 2^32), Box-Muller on
   word pairs). */
void orc_normals(uint64_t seed, uint64_t counter, uint32_t s, uint32_t tau, int d, double *n);

/* The noise stream as a table: Philox words (uint32) and normals (double) of
   samples s < n_samples, steps tau < H, blocks b < n_blocks at
   ((s*H + tau)*n_blocks + b)*4 + j; either output may be NULL. */
void orc_noise_table(uint64_t seed, uint64_t counter, int n_samples, int H, int n_blocks, uint32_t *words,
                     double *normals);

/* One explicit-Euler step of the tractor-trailer kinematics. */
void orc_dynamics_step(const orc_params *P, const double x[7], const double u[3], double xn[7]);

/* Super-ellipse obstacle barrier h_o(x) (Sec. IV-C).  Returns NaN when the
   exponent is not an even integer >= 2. */
double orc_obstacle_h(const orc_params *P, const double obs[6], const double x[7]);

/* Barrier-rate equality row of one obstacle: A_u (3 entries), h, and the
   part of b that does not depend on alpha, b = -alpha*h + b_rest. */
void orc_obstacle_row(const orc_params *P, const double obs[6], const double x[7],
                      double A_u[3], double *h, double *b_rest);

/* Time-varying obstacles (predicted pedestrians, Sec. IV-C): a row of
   `stride` (6 or 8) doubles; with 8 the centre at time t is
   (cx + t vx, cy + t vy).  h and the barrier-rate row at time t. */
double orc_obstacle_h_at(const orc_params *P, const double *obs, int stride, double t,
                         const double x[7]);
void orc_obstacle_row_at(const orc_params *P, const double *obs, int stride, double t,
                         const double x[7], double A_u[3], double *h, double *b_rest);

/* Footprint discs (Sec. IV-C: the body covered by discs of radius r, the
   obstacles inflated by r).  Disc m of the tractor sits at p + d e1, of the
   trailer at p - lh e1 - (l2 - d) e2, with e1, e2 the unit headings and d =
   disc_off[m].  Constraint 1 + o * n_discs + m is obstacle o seen from disc
   m.  Centre of disc m at state x: */
void orc_disc_position(const orc_params *P, int m, const double x[7], double pos[2]);
/* h of obstacle row `obs` (stride 6 or 8) seen from disc m at time t, and
   its barrier-rate row (second-order expansion along the field with the
   input held; the steer rate enters through the heading accelerations of
   offset discs). */
double orc_disc_h(const orc_params *P, const double *obs, int stride, double t, int m,
                  const double x[7]);
void orc_disc_row(const orc_params *P, const double *obs, int stride, double t, int m,
                  const double x[7], double A_u[3], double *h, double *b_rest);

/* Jerk-input model (Sec. III-A, Eq. tt_discrete_kinematics as the paper
   writes it: acceleration a is a state driven by the jerk).  State x[8] =
   (px, py, th1, th2, v, delta, psi, a), input u = (jerk, omega, nu). */
void orc_jerk_step(const orc_params *P, const double x[8], const double u[3], double xn[8]);
void orc_jerk_integrate(const orc_params *P, const double x0[8], const double *U, int H,
                        double *traj);
/* Barrier-rate rows of the jerk model (same expansion orders as the
   acceleration model: hitch second order, obstacles second or -- with
   ORC_THIRD_ORDER -- third). */
void orc_jerk_hitch_row(const orc_params *P, const double x[8], double A_u[3], double *h,
                        double *b_rest);
void orc_jerk_obstacle_row(const orc_params *P, const double *obs, int stride, double t,
                           const double x[8], double A_u[3], double *h, double *b_rest);

/* Third-order barrier-rate row of obstacle `obs` at the rear axle:
   Ts hdot + Ts^2/2 hddot + Ts^3/6 hdddot along the field with the input held
   (affine in (a, omega): the steer rate enters through th1ddot). */
void orc_obstacle_row3(const orc_params *P, const double *obs, int stride, double t,
                       const double x[7], double A_u[3], double *h, double *b_rest);

/* MPPI + collision cost baseline: q_coll * sum_o max(0, -h_o(x, t)) over
   every obstacle and footprint disc. */
double orc_collision_cost(const orc_params *P, const double *obs, int stride, int n_obs, double t,
                          const double x[7]);

/* Barrier-rate buffer cost: q_abuf * sum_i w(h_i) max(0, alpha_i)^2 with the
   ramp w(h) = clip(1 - h/h_buf, 0, 1) for h >= 0 and 1 for h < 0. */
double orc_alpha_buffer_cost(const orc_params *P, int n, const double *h, const double *alpha);

/* Hitch-angle barrier h_h(x) (Sec. IV-D) and its barrier-rate row. */
double orc_hitch_h(const orc_params *P, const double x[7]);
void orc_hitch_row(const orc_params *P, const double x[7], double A_u[3], double *h, double *b_rest);

/* Hitch-angle stabilizer CBF-QP (Sec. IV-D, Eq. hitch_angle_qp): u_out[0..2]
   is the (a, omega) nearest u_ref in the Q_h norm inside the input box whose
   hitch increment meets the discrete CBF condition, nu passed through;
   *slack = increment + alpha_stab h (>= 0 when met).  Returns 0, or 1 when
   no input in the box meets it (u_out then maximises the increment). */
int orc_hitch_stabilize(const orc_params *P, const double *x, const double u_ref[3],
                        double u_out[3], double *slack); /* x: 8 entries under ORC_JERK */

/* Soft-bound equality projection, closed form (Sec. IV-A), dense.
   A is nc x d row-major, w the diagonal of W (d entries).  Returns ORC_OK or
   ORC_EINVAL if A M^-1 A^T is singular. nc may be 0. */
int orc_project(int d, int nc, const double *A, const double *b, const double *w, double rho,
                const double *z_lo, const double *z_hi, const double *z_des, double *z_star);

/* Reference path lookup at arc length psi: linear interpolation in a table of
   n >= 2 rows sampled every ds. */
void orc_path_lookup(const double *path, int n, double ds, double psi, double *xr, double *yr,
                     double *thr);

/* Contouring stage cost r(x, u, psi) (Sec. IV-B). */
double orc_stage_cost(const orc_params *P, const double x[7], const double u[3], const double *path,
                      int n, double ds);

/* Softmin weights gamma_bar_s (Sec. II-B); non-finite J gets weight 0.
   Returns ORC_ENONFINITE if no J is finite. */
int orc_softmin(int S, const double *J, double lambda, double *gamma_bar);

/* One rollout of sample s.  Any output pointer may be NULL:
   states (H+1)*NX, u (H)*3 applied inputs, alpha (H+1)*Nc, z_des H*d,
   z_star H*d, J scalar; NX = 8 under ORC_JERK (x0 then has 8 entries),
   else 7.  Returns ORC_OK or ORC_EINVAL. */
int orc_rollout_sample(const orc_params *P, const double *x0, const double *U_nom,
                       const double *obs, int n_obs, const double *path, int n_pts, double ds,
                       uint64_t seed, uint64_t counter, uint32_t s, double *states, double *u,
                       double *alpha, double *z_des, double *z_star, double *J);

/* The MPPI update (Sec. II-B): softmin weights of J, then the weighted sum of
   the applied inputs u_hist (S*H*3) in sample order into U_out (H*3).
   gamma_bar: S doubles (workspace; the weights on return).  No finite J:
   U_out = U_nom and ORC_ENONFINITE. */
int orc_update(int S, int H, const double *J, const double *u_hist, double lambda,
               const double *U_nom, double *gamma_bar, double *U_out);

/* Rollouts of samples s0 .. s1-1, each as orc_rollout_sample: J_out (s1-s0),
   u_hist (s1-s0)*H*3 and states_out (s1-s0)*(H+1)*NX optional (NULL). */
int orc_rollout_range(const orc_params *P, const double *x0, const double *U_nom, const double *obs,
                      int n_obs, const double *path, int n_pts, double ds, uint64_t seed,
                      uint64_t counter, uint32_t s0, uint32_t s1, double *J_out, double *u_hist,
                      double *states_out);

/* The full solve.  U_out H*3 (required); traj_out (H+1)*NX, J_out S,
   u_hist S*H*3, states_out S*(H+1)*NX optional (NX as for rollouts).  On
   ORC_ENONFINITE U_out is the nominal sequence. */
int orc_solve(const orc_params *P, const double *x0, const double *U_nom, const double *obs,
              int n_obs, const double *path, int n_pts, double ds, uint64_t seed,
              uint64_t counter, double *U_out, double *traj_out, double *J_out, double *u_hist,
              double *states_out);

/* Euler rollout of a fixed input sequence (no projection): traj (H+1)*7. */
void orc_integrate(const orc_params *P, const double x0[7], const double *U, int H, double *traj);

#ifdef __cplusplus
}
#endif
#endif
