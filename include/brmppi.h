/*
 * brmppi.h -- C ABI of the GB300 (sm_103a) BR-MPPI solver library
 * (libbrmppi.so).
 *
 * One solve is one control update of Barrier-Rate guided MPPI for a
 * tractor-trailer, as defined in "GPU-Accelerated Barrier-Rate Guided MPPI
 * Control for Tractor-Trailer Systems" (arXiv 2508.05773):
 *   - S rollouts over H steps of the kinematics of Sec. III-A
 *     (Eq. tt_discrete_kinematics, explicit Euler, acceleration as input and
 *     the path progress psi driven by the progress rate nu, Sec. IV-B);
 *   - at every step the sampled augmented input z = (a, omega, nu, u^alpha)
 *     is projected onto the barrier-rate equalities of Eq. cbf_equality with
 *     the soft-bound closed form of Eq. closed-form_projection (Sec. IV-A),
 *     one row per elliptical obstacle (Eq. barrier_function with the
 *     second-order expansion of Eq. barrier_function_approx, Sec. IV-C) and
 *     one for the velocity-scaled hitch limit (Eq. hitch_angle_barrier,
 *     Sec. IV-D);
 *   - each rollout accumulates the contouring cost of
 *     Eq. cost_function_contour / contour_lag_errors (Sec. IV-B);
 *   - the solve ends with the softmin weights and the weighted update of
 *     Eq. MPPI_update_rule (Sec. II-B), computed as a max-subtracted
 *     log-sum-exp, and the optimal trajectory (x0 integrated with U*).
 *
 * Layouts (all row-major, caller-owned):
 *   state      x0[7]        double  (px, py, theta1, theta2, v, delta, psi)
 *   inputs     U[H][3]      float   (a, omega, nu)
 *   obstacles  obs[n][6]    float   (cx, cy, mx, my, theta_o, e); e must be 2
              obs[n][8]    float   with BRMPPI_FLAG_OBS8: + (vx, vy), e in {2, 4}
 *   path       path[n][3]   float   (x, y, heading unwrapped) at s = j*ds;
 *                                   consecutive headings at most pi/4 apart
 *                                   (else BRMPPI_EINVAL)
 *   trajectory traj[H+1][7] float
 *   costs      J[S]         float
 *
 * Noise: normal q of sample s at step tau is lane q%4 of the Philox4x32-10
 * block at counter (q/4, tau, s, counter mod 2^32) with key
 * (seed mod 2^32, seed / 2^32), Box-Muller on word pairs (0,1), (2,3);
 * q = 0,1,2 perturb (a, omega, nu), q = 3 + i the barrier-rate input of
 * constraint i (0 = hitch, 1.. = obstacles in input order).
 *
 * Conventions: every function returns a brmppi_status; on failure the
 * context's last-error string says why and no output is written (host entry
 * points) or written outputs are unspecified (device entry points). The
 * library never throws. All computation runs in the library's CUDA kernels;
 * there is no CPU fallback.  A context is used by one host thread at a time
 * for solve / solve_device; submit / poll are thread-safe.
 */
#ifndef BRMPPI_H
#define BRMPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BRMPPI_ABI_VERSION 7u

typedef enum {
  BRMPPI_OK = 0,
  BRMPPI_EINVAL = -1,     /* bad argument (sizes, NULL, e != 2, ...) */
  BRMPPI_ENOMEM = -2,     /* device or pinned allocation failed */
  BRMPPI_EAGAIN = -3,     /* result not ready yet (poll) */
  BRMPPI_ETIMEDOUT = -4,  /* a bounded wait gave up */
  BRMPPI_ENONFINITE = -5, /* non-finite input, or no rollout had a finite cost
                             (U_out then holds the nominal sequence) */
  BRMPPI_ECUDA = -6,      /* CUDA runtime error (message in last_error) */
  BRMPPI_EBUSY = -7       /* no free slot / queue full */
} brmppi_status;

/* Flags */
#define BRMPPI_FLAG_PROJ_NONE 0x1u /* standard MPPI: skip the projection (baseline) */
/* MPPI + collision cost (the comparison method of Sec. V): every stage cost
   adds q_coll * sum_o max(0, -h_o(x)) at the state after the step.  The
   paper does not give the penalty's form; this is a penetration hinge. */
#define BRMPPI_FLAG_COLLISION_COST 0x2u
/* Obstacle rows of 8 floats (cx, cy, mx, my, theta_o, e, vx, vy): super-
   ellipses with e in {2, 4} whose centre moves at (vx, vy) from the solve's
   start (predicted pedestrians, Sec. IV-C); the rows of step tau use the
   centre at tau*Ts and the relative velocity.  Without this flag rows are 6
   floats and e must be 2. */
#define BRMPPI_FLAG_OBS8 0x4u
/* Barrier-rate buffer cost (Sec. IV-A): each obstacle row built at step tau
   adds q_abuf * w(h) * max(0, alpha)^2 with its h and rate alpha, where
   w(h) = clip(1 - h/h_buf, 0, 1): positive rates are charged near an
   obstacle, pushing the samples toward hdot >= 0 there. */
#define BRMPPI_FLAG_ALPHA_BUFFER 0x8u
/* Obstacle rows to third order: Ts hdot + Ts^2/2 hddot + Ts^3/6 hdddot with
   the input held, which brings the steer rate into obstacle rows (through
   the tractor's yaw acceleration).  Needs the single rear-axle disc (offset
   discs make the third-order term quadratic in the input). */
#define BRMPPI_FLAG_THIRD_ORDER 0x10u
/* The paper's jerk-input model (Sec. III-A): the longitudinal acceleration
   a is a state and input 0 is the jerk (bounds z_lo[0], z_hi[0] and noise
   sigma[0] apply to the jerk).  x0 then holds 8 doubles, (px, py, theta1,
   theta2, v, delta, psi, a); outputs keep 7 columns.  The hitch row sees the
   jerk at second order, obstacle rows only with BRMPPI_FLAG_THIRD_ORDER
   (relative degree 3).  Needs the single rear-axle disc. */
#define BRMPPI_FLAG_JERK_MODEL 0x20u

/* Every constant of the solve; POD. Fields the paper leaves open take the
   documented readings (alpha init, noise and bounds of u^alpha, W, rho, the
   floor on |h| in A's alpha column). */
typedef struct brmppi_params {
  uint32_t abi_version;          /* must be BRMPPI_ABI_VERSION */
  int32_t S, H;                  /* samples, horizon steps (S >= 1, 1 <= H <= 1024) */
  int32_t max_obstacles;         /* capacity: obstacles per solve (<= 124) */
  int32_t max_path_pts;          /* capacity: path rows per solve, in [2, 8192] */
  int32_t flags;                 /* BRMPPI_FLAG_* */
  int32_t threads_per_sample;    /* plain solves: 0 = tuned/heuristic, else 1, 2, 4, 8, 16, 32 */
  int32_t block_threads;         /* plain solves: 0 = tuned/heuristic, else 64..512, multiple of 32 */
  int32_t max_batch;             /* capacity: instances per batch (0 = no batches) */
  int32_t batch_threads_per_sample; /* batches: 0 = tuned/heuristic, else as above */
  int32_t batch_block_threads;   /* batches: 0 = tuned/heuristic, else as above */
  int32_t max_vehicles;          /* serving: registered vehicles (0 = no serving loop) */
  int32_t serve_lanes;           /* serving: batches in flight at once (0 = 2) */
  int32_t serve_max_batch;       /* serving: solves per launch (0 = 64) */
  int32_t serve_queue;           /* serving: request slots, further capped by free
                                    device memory at create (0 = 1024) */
  int32_t wait_timeout_ms;       /* limit of the library's host-side waits for the
                                    GPU (serving completions, destroy): 0 = 10000 */
  float Ts, lambda;              /* sample time [s]; softmin temperature */
  float l1, lh, l2;              /* wheelbase, hitch offset, trailer length [m] */
  float dtheta_max, kappa;       /* hitch limit dtheta_max - kappa*v */
  float r_inflate;               /* footprint disc radius added to semi-axes */
  float Qc, Ql, Qth, R[3], mu, nu_bar; /* contouring cost weights, progress target */
  float z_lo[3], z_hi[3];        /* bounds of (a, omega, nu) */
  float sigma[3];                /* noise std of (a, omega, nu) */
  float alpha0, sigma_alpha;     /* barrier-rate init, noise std of u^alpha */
  float ua_lo, ua_hi;            /* bounds of u^alpha */
  float w_u[3], w_alpha;         /* diagonal of W */
  float rho, h_floor;            /* soft-bound penalty; floor on |h| in A */
  float q_coll;                  /* BRMPPI_FLAG_COLLISION_COST weight (>= 0) */
  float alpha_stab;              /* hitch stabilizer: discrete CBF rate, (0, 1] */
  float q_stab[2];               /* hitch stabilizer: Q_h = diag(q_stab) on (a, omega), > 0 */
  float q_abuf, h_buf;           /* BRMPPI_FLAG_ALPHA_BUFFER weight (>= 0), zone width (> 0) */
  /* Footprint discs (Sec. IV-C: the body covered by discs whose radius,
     r_inflate, inflates the obstacles).  Disc m sits on the tractor at
     p + disc_off[m] e1, or (bit m of disc_trailer_mask) on the trailer at
     p - lh e1 - (l2 - disc_off[m]) e2, e1 / e2 the unit headings; obstacle o
     seen from disc m is constraint 1 + o * n_discs + m (so
     max_obstacles * n_discs <= 124).  Default: one disc at the tractor's
     rear axle. */
  int32_t n_discs;               /* 1..8 */
  int32_t disc_trailer_mask;     /* bits below n_discs */
  float disc_off[8];             /* [m] */
} brmppi_params;

typedef struct brmppi_ctx brmppi_ctx; /* opaque: device buffers, stream */

/* One solve of a batch; every pointer is DEVICE memory with the layouts
   above.  S <= params.S, H <= params.H, n_obs <= max_obstacles,
   2 <= n_pts <= max_path_pts.  Outputs as for brmppi_solve_device. */
typedef struct brmppi_instance {
  const double *x0;
  const float *U_nom, *obs, *path;
  int32_t n_obs, n_pts;
  float ds;
  int32_t S, H;
  uint64_t seed, counter;
  float *U_out, *traj_out, *J_out, *U_next; /* U_out required; others may be NULL */
  int32_t *status;                          /* may be NULL */
  float *states_out; /* may be NULL: stored-trajectory variant, every sample's
                        states S x (H+1) x 7 (world frame, x0 first) */
  float *u_safe_out; /* may be NULL: U*[0] after the hitch stabilizer (see
                        brmppi_hitch_stabilize_device), 4 floats, written by
                        a small launch that follows the solve on its stream */
  float *inputs_out; /* may be NULL: every sample's applied (clipped) inputs,
                        S x H x 3 -- the u_s of the update */
  float *J_lo_out;   /* may be NULL: S floats; the cost of sample s that the
                        softmin uses is the unevaluated pair
                        J_out[s] + J_lo_out[s] (|J_lo_out[s]| <= half an ulp
                        of J_out[s]) */
} brmppi_instance;

typedef struct brmppi_graph brmppi_graph; /* a captured batch launch */

/* Fill *p with the library defaults (abi_version set). */
void brmppi_default_params(brmppi_params *p);

/* Create a context on CUDA device `device`; allocates every buffer a solve
   of the given capacities needs (device + pinned host). */
brmppi_status brmppi_create(const brmppi_params *p, int device, brmppi_ctx **out);

/* Destroy a context (NULL is a no-op): waits for its work to finish, at
   most params.wait_timeout_ms for each of its streams and batch lanes, then
   frees everything.  BRMPPI_ETIMEDOUT if a wait gave up: the buffers that
   the unfinished work may still use are then left allocated (leaked) rather
   than freed under it; the context itself is released either way.  Returns
   BRMPPI_OK otherwise. */
brmppi_status brmppi_destroy(brmppi_ctx *ctx);

/* Testing hook for the out-of-memory paths (no paper counterpart): the n-th
   device or pinned-host allocation that the library makes from now on
   (counting every context, batch lane, serving slot and vehicle buffer)
   fails as if the device were out of memory, without calling CUDA; n <= 0
   disarms it.  The failing call returns BRMPPI_ENOMEM and unwinds what it had
   allocated.  Process-wide; not for production use. */
void brmppi_inject_alloc_failure(int32_t n);

/* Message of the last failure on this context ("" if none); valid until the
   next call on the context. A NULL ctx gives the last create() failure. */
const char *brmppi_last_error(const brmppi_ctx *ctx);

/* One solve from HOST buffers: copies the inputs to the device (one copy
   from the context's pinned staging buffer), runs the solve, whose kernel
   writes U* (H*3), the optimal trajectory ((H+1)*7) and its status straight
   into a pinned host buffer of the context, and copies the per-sample costs
   (S) back when asked for; returns when the outputs are in the caller's
   buffers.  n_obs in [0, max_obstacles], n_pts in [2, max_path_pts], ds > 0. */
brmppi_status brmppi_solve(brmppi_ctx *ctx, const double x0[7], const float *U_nom,
                           const float *obs, int32_t n_obs, const float *path, int32_t n_pts,
                           float ds, uint64_t seed, uint64_t counter, float *U_out,
                           float *traj_out, float *J_out);

/* The same solve on DEVICE buffers, enqueued on `stream` (a cudaStream_t;
   NULL = the legacy default stream). Allocates nothing and does not
   synchronise: outputs are valid once the stream reaches this point.
   status_dev (device int32, may be NULL) receives BRMPPI_OK,
   BRMPPI_ENONFINITE or BRMPPI_EINVAL from the kernel. U_next (device H*3,
   may be NULL) receives the warm start for the next tick: U* shifted by one
   step with its last row repeated. */
brmppi_status brmppi_solve_device(brmppi_ctx *ctx, const double *x0_dev, const float *U_nom_dev,
                                  const float *obs_dev, int32_t n_obs, const float *path_dev,
                                  int32_t n_pts, float ds, uint64_t seed, uint64_t counter,
                                  float *U_out_dev, float *traj_out_dev, float *J_out_dev,
                                  float *U_next_dev, int32_t *status_dev, void *stream);

/* One solve described by an instance (device pointers): as
   brmppi_solve_device, with S <= params.S and H <= params.H per call and the
   optional stored-trajectory output.  Allocates nothing, does not
   synchronise. */
brmppi_status brmppi_solve_device_ex(brmppi_ctx *ctx, const brmppi_instance *inst, void *stream);

/* Hitch-angle stabilizer (Sec. IV-D, Eq. hitch_angle_qp) for n states at
   once, one GPU thread each.  For state x_i (x_dev[i][7], double) and the
   reference u_ref_dev[i][3] = (a, omega, nu) from BR-MPPI, u_out_dev[i][4]
   receives (a, omega, nu, slack): (a, omega) minimises
   (u - u_ref)^T diag(q_stab) (u - u_ref) over the input box z_lo..z_hi
   subject to the discrete CBF condition of Eq. barrier_constraint_prelim on
   the hitch barrier,  Ts hdot + Ts^2/2 hddot >= -alpha_stab h_h(x)  (the
   increment of the rollout's hitch row; sign as in Eq. cbf_equality); nu
   passes through.  slack = increment + alpha_stab h_h at the result: >= 0
   (up to rounding) when the condition is met; < 0 means no input in the box
   meets it and (a, omega) is the box corner that maximises the increment.
   Solved in closed form (KKT of a one-row QP with a diagonal weight and a
   box).  Under BRMPPI_FLAG_JERK_MODEL x_dev is n x 8 (a last) and the QP is
   over (jerk, omega).  Enqueued on `stream`; allocates nothing.  n = 0 is a
   no-op. */
brmppi_status brmppi_hitch_stabilize_device(brmppi_ctx *ctx, const double *x_dev,
                                            const float *u_ref_dev, int32_t n, float *u_out_dev,
                                            void *stream);

/* A batch of independent solves (uneven S, H, obstacle count, path) in ONE
   launch of a persistent kernel: work items (instance, sample tile) are
   taken longest-first from an atomic counter; each instance's partials are
   merged in tile order by the CTA that finishes its last tile, so a solve
   gives the same result alone (as a batch of one) or in any mix.  Uploads
   the instance table and work list (host -> device, pinned) and enqueues
   the kernel on `stream`; allocates nothing, does not synchronise (the next
   call on this context waits for the previous upload to be consumed). */
brmppi_status brmppi_solve_batch(brmppi_ctx *ctx, const brmppi_instance *inst, int32_t n,
                                 void *stream);

/* Capture the upload and the persistent launch of a batch into a CUDA graph
   (the instance table is snapshotted; the instances' device buffers are
   read at every replay, so updating their contents in place between replays
   is the intended use). */
brmppi_status brmppi_batch_capture(brmppi_ctx *ctx, const brmppi_instance *inst, int32_t n,
                                   brmppi_graph **out);
brmppi_status brmppi_graph_launch(brmppi_graph *g, void *stream);
void brmppi_graph_destroy(brmppi_graph *g);

/* Autotuner: time every supported launch shape (threads per sample x Philox
   blocks per lane x block size) on the given device inputs, `reps` launches
   each, and keep the fastest for later plain solves with this obstacle
   count (used when params.threads_per_sample == 0). */
brmppi_status brmppi_autotune(brmppi_ctx *ctx, const double *x0_dev, const float *U_nom_dev,
                              const float *obs_dev, int32_t n_obs, const float *path_dev,
                              int32_t n_pts, float ds, int32_t reps, void *stream);

/* Autotuner for batches: as above on a batch, keeping the fastest shape for
   later batches (used when params.batch_threads_per_sample == 0). */
brmppi_status brmppi_autotune_batch(brmppi_ctx *ctx, const brmppi_instance *inst, int32_t n,
                                    int32_t reps, void *stream);

/* A solve that allocates nothing and needs no context.  The paper has no
   counterpart: it serves callers that cannot call cudaMalloc once running --
   code enqueued while a CUDA graph is being captured, and controllers whose
   device memory is fixed at start-up -- and so cannot create a brmppi_ctx.
   Same inputs, outputs and results as brmppi_solve_device (all pointers
   device memory, enqueued on `stream`, no synchronisation); the launch shape
   is fixed (4 lanes per sample, 128-thread blocks) and the scratch lives in
   a file-scope device array of about 3.1 MiB that every device loading the
   library keeps until exit.  Maxima: S <= 4096, H <= 64, n_obs <= 16,
   n_pts <= 4096; larger sizes return BRMPPI_EINVAL with the reason in
   brmppi_last_error(NULL), and so does a shared-memory need above the
   device's limit.  The first call on a device sets the kernels'
   shared-memory limit for that device; make that first call before any
   stream capture.  Every call looks up the array's device address with
   cudaGetSymbolAddress (a host-side query that allocates nothing) and
   repeats that set-up if the address changed (after a cudaDeviceReset).
   All calls on a device share the array (counters are cleared on `stream`
   before each launch): calls that overlap on the GPU race, so serialise
   them. */
brmppi_status brmppi_solve_device_noalloc(const brmppi_params *p, const double *x0_dev,
                                          const float *U_nom_dev, const float *obs_dev,
                                          int32_t n_obs, const float *path_dev, int32_t n_pts,
                                          float ds, uint64_t seed, uint64_t counter,
                                          float *U_out_dev, float *traj_out_dev, float *J_out_dev,
                                          float *U_next_dev, int32_t *status_dev, void *stream);

/* ---- Serving loop (contexts created with max_vehicles > 0) ----------------
   A scheduler thread admits submitted requests into batches as request slots
   and batch lanes free up, launches each batch (one persistent launch) on its
   lane's stream while earlier batches still run, and a completion thread
   publishes results.  Every vehicle keeps its path, its warm-started nominal
   sequence (shifted in place on the device after each solve) and its noise
   counter (+1 per solve) resident; requests of one vehicle run in
   submission order.  Results do not depend on what else is in a batch: the
   serving launch shape is fixed at create (params.batch_threads_per_sample
   and batch_block_threads when set, else one lane per sample in 128-thread
   blocks), and a batch of one on the same context (batch shape not changed
   by brmppi_autotune_batch) reproduces a served solve bit for bit. */

/* Register (or re-register) a vehicle: its reference path (host, n_pts*3),
   initial nominal sequence (host H*3, NULL = zeros) and noise seed; its
   counter starts at 0.  EBUSY while the vehicle has requests in flight. */
brmppi_status brmppi_vehicle_register(brmppi_ctx *ctx, uint32_t vehicle_id, const float *path,
                                      int32_t n_pts, float ds, const float *U_init, uint64_t seed);

/* Queue one solve for a vehicle from host buffers (state x0[7], obstacles
   n_obs*6); copies them before returning.  *ticket identifies the result.
   EBUSY when no request slot is free (retry after polling). */
brmppi_status brmppi_submit(brmppi_ctx *ctx, uint32_t vehicle_id, const double x0[7],
                            const float *obs, int32_t n_obs, uint64_t *ticket);

/* Non-blocking: EAGAIN until the ticket's solve has finished, then copies
   U* (H*3) and, if traj_out is not NULL, the optimal trajectory, reports
   the submit-to-completion latency, releases the ticket and returns the
   solve's status.  EINVAL for an unknown or released ticket. */
brmppi_status brmppi_poll(brmppi_ctx *ctx, uint64_t ticket, float *U_out, float *traj_out,
                          double *latency_s);

/* Snapshot / restore a vehicle's solver state (nominal sequence, seed,
   counter): the whole state, so a restored vehicle replays bit-identically.
   EBUSY while the vehicle has requests in flight. */
brmppi_status brmppi_vehicle_export(brmppi_ctx *ctx, uint32_t vehicle_id, float *U_nom,
                                    uint64_t *seed, uint64_t *counter);
brmppi_status brmppi_vehicle_import(brmppi_ctx *ctx, uint32_t vehicle_id, const float *U_nom,
                                    uint64_t seed, uint64_t counter);

typedef struct brmppi_server_stats {
  uint64_t submitted, completed, batches, solves_in_batches;
  int32_t request_slots, lanes, max_inflight_batches, max_batch;
} brmppi_server_stats;

brmppi_status brmppi_server_stats_get(brmppi_ctx *ctx, brmppi_server_stats *out);

/* Launch configuration the context will use for a solve with n_obs
   obstacles (after autotuning if requested). */
brmppi_status brmppi_get_launch(brmppi_ctx *ctx, int32_t n_obs, int32_t *threads_per_sample,
                                int32_t *block_threads, int32_t *blocks);

/* Launch configuration batches (and serving batches) of this context use:
   the autotuned shape after brmppi_autotune_batch, else the default for the
   context's obstacle capacity.  Threads per block exclude noise warps. */
brmppi_status brmppi_get_batch_launch(brmppi_ctx *ctx, int32_t *threads_per_sample, int32_t *block_threads);

/* The noise stream of the solves, for checking it (paper Sec. II-B: the
   sampled perturbations; reading R15 of the noise generator): for samples
   s < n_samples, steps tau < H and Philox blocks b < n_blocks, the four
   Philox4x32-10 words of key (seed lo, seed hi) and counter (b, tau, s,
   counter lo), and the four standard normals the solve kernel draws from
   them (Box-Muller on the word pairs (0, 1) and (2, 3) after the map
   ((w >> 9) + 1/2) 2^-23), computed by the same device functions as the
   solves.  Layout: words_dev (uint32) and normals_dev (float), both
   n_samples*H*n_blocks*4 entries at ((s*H + tau)*n_blocks + b)*4 + j, device
   memory owned by the caller, 16-byte aligned; either may be NULL.  Enqueued
   on `stream` (no synchronisation, no allocation, no context).  EINVAL for
   negative sizes, more than 2^31 blocks, H or n_blocks above 2^16, or a
   misaligned output, with the reason in brmppi_last_error(NULL). */
brmppi_status brmppi_noise_blocks(uint64_t seed, uint64_t counter, int32_t n_samples, int32_t H,
                                  int32_t n_blocks, uint32_t *words_dev, float *normals_dev,
                                  void *stream);

/* ---- One solve partitioned by samples (several GPUs; SURVEY's only
   exchange of the path: the softmin and update of Sec. II-B, Eq.
   MPPI_update_rule, need every sample's cost).  The samples of a solve are
   cut into tiles of the context's plain launch shape; rank r runs a
   contiguous range of tiles (brmppi_solve_tiles), the ranks all-gather
   their tile partials in rank order (tile order), and every rank merges
   the complete set (brmppi_merge_tiles).  The merge is the one a single
   launch ends with, over the same tiles in the same order: U*, the optimal
   trajectory and the warm start are bit-identical to brmppi_solve_device_ex
   on one GPU.  Every rank's context must have the same parameters. */

/* The partition's layout for instance q: *n_tiles tiles of *tile_floats
   floats each (the launch shape of the context's plain solves). */
brmppi_status brmppi_tile_layout(brmppi_ctx *ctx, const brmppi_instance *q, int32_t *n_tiles,
                                 int32_t *tile_floats);

/* Roll out tiles [tile0, tile0 + n_tiles) of instance q (device buffers;
   U_out, traj_out, U_next, status and u_safe_out are not used) and write
   their partials to tiles_out (device, n_tiles * tile_floats floats,
   16-byte aligned, tile tile0 first); J_out, J_lo_out, inputs_out and
   states_out, if given (sized for all S samples), receive the range's
   samples.  Enqueued on `stream`, no synchronisation.  An input error
   (exponent, non-finite x0) is recorded on the context and reported by the
   next brmppi_merge_tiles on it. */
brmppi_status brmppi_solve_tiles(brmppi_ctx *ctx, const brmppi_instance *q, int32_t tile0,
                                 int32_t n_tiles, float *tiles_out, void *stream);

/* Merge all n_tiles tile partials of instance q (device, in tile order, as
   brmppi_solve_tiles wrote them) into U_out and, if given, traj_out,
   U_next and the status word (q's x0, U_nom, obstacles and path must be the
   solve's).  EINVAL unless n_tiles is the instance's tile count.  One CTA,
   enqueued on `stream`. */
brmppi_status brmppi_merge_tiles(brmppi_ctx *ctx, const brmppi_instance *q, const float *tiles,
                                 int32_t n_tiles, void *stream);

/* Issue-rate microbenchmark of one SM pipe on the current device, for the
   roofline denominators of the solve (no paper counterpart): pipe 0 = FP32
   fused multiply-add, 1 = 32-bit integer multiply-add, 2 = the XU's
   reciprocal square root (the special-function unit that also evaluates
   log, sin, cos, exp and reciprocals).  4 CTAs of 512 threads per SM, each
   thread eight independent chains of `iters` x 16 operations; one untimed
   warm-up launch, then one launch timed with CUDA events on `stream` (waits
   for it).  *lane_ops_per_s = lane operations of the pipe per second,
   *seconds (may be NULL) the timed launch.  Changes no device setting;
   allocates nothing.  EINVAL for a bad pipe or iters < 1. */
brmppi_status brmppi_measure_pipe(int32_t pipe, int64_t iters, double *lane_ops_per_s, double *seconds,
                                  void *stream);

/* Bytes the host entry point brmppi_solve moves per call for a solve with
   n_obs obstacles and n_pts path rows: *h2d (inputs, one copy) and *d2h
   (U*, trajectory and status, written by the kernel into pinned host
   memory; plus 4*S when costs are asked for). */
brmppi_status brmppi_transfer_bytes(brmppi_ctx *ctx, int32_t n_obs, int32_t n_pts, uint64_t *h2d,
                                    uint64_t *d2h);

#ifdef __cplusplus
}
#endif
#endif
