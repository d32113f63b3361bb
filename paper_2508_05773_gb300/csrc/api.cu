// api.cu -- the C ABI of libbrmppi.so (see include/brmppi.h).
//
// The context owns every buffer a solve needs, sized at create time for the
// declared capacities, so the solve paths allocate nothing.  Host entry
// points stage inputs through one pinned buffer (one H2D copy), run the
// kernel and read the outputs back (one D2H copy, plus the costs when asked
// for).  Batches upload an instance table and a longest-first work list and
// run one persistent launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace brmppi_host;

// The layouts the Python binding mirrors.
static_assert(sizeof(brmppi_params) == 4 * 16 + 4 * 41 + 4 * 10, "brmppi_params layout");
static_assert(sizeof(brmppi_instance) == 8 * 4 + 4 * 5 + 4 + 8 * 2 + 8 * 9, "brmppi_instance layout");

namespace brmppi_host {

namespace {
std::mutex g_err_mu;
std::string g_create_err;

}  // namespace

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

namespace {
std::atomic<int> g_fail_alloc_in{0};  // > 0: the allocation that brings it to 0 fails

bool injected_alloc_failure() {
  int n = g_fail_alloc_in.load();
  while (n > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}
}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

cudaError_t wait_event(cudaEvent_t ev, int timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q != cudaErrorNotReady) return q;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) return cudaErrorNotReady;
    std::this_thread::yield();
  }
}

cudaError_t wait_stream(cudaStream_t s, int timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(s);
    if (q != cudaErrorNotReady) return q;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) return cudaErrorNotReady;
    std::this_thread::yield();
  }
}

brmppi_status fail(brmppi_ctx* c, brmppi_status st, const std::string& msg) {
  if (c) {
    c->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
  }
  return st;
}

brmppi_status cuda_fail(brmppi_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? BRMPPI_ENOMEM : BRMPPI_ECUDA, m);
}

int philox_blocks(int n_rows) { return (4 + n_rows + 3) / 4; }  // d = 3 + (1 + n_rows), rows = obstacles x discs

int ext_team_width(int P) { return P <= 4 ? 2 : (P <= 8 ? 4 : (P <= 16 ? 8 : 16)); }

namespace {

bool is_pow2_tps(int t) { return t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32; }

bool valid_threads(int t) { return t == 0 || (t >= kMinThreads && t <= kMaxThreads && t % 32 == 0); }

}  // namespace

std::string check_params(const brmppi_params* p) {
  if (!p) return "params is NULL";
  if (p->abi_version != BRMPPI_ABI_VERSION) return "abi_version mismatch";
  if (p->S < 1) return "S must be >= 1";
  if (p->H < 1 || p->H > kMaxH) return "H must be in [1, 1024]";
  if (p->max_obstacles < 0 || p->max_obstacles > kMaxObstacles) return "max_obstacles must be in [0, 124]";
  if (p->max_path_pts < 2 || p->max_path_pts > kMaxPathPts) return "max_path_pts must be in [2, 8192]";
  if (p->flags & ~static_cast<int32_t>(BRMPPI_FLAG_PROJ_NONE | BRMPPI_FLAG_COLLISION_COST | BRMPPI_FLAG_OBS8 |
                                        BRMPPI_FLAG_ALPHA_BUFFER | BRMPPI_FLAG_THIRD_ORDER | BRMPPI_FLAG_JERK_MODEL))
    return "unknown flag";
  if (p->threads_per_sample != 0 && !is_pow2_tps(p->threads_per_sample))
    return "threads_per_sample must be 0, 1, 2, 4, 8, 16 or 32";
  if (p->batch_threads_per_sample != 0 && !is_pow2_tps(p->batch_threads_per_sample))
    return "batch_threads_per_sample must be 0, 1, 2, 4, 8, 16 or 32";
  if (!valid_threads(p->block_threads) || !valid_threads(p->batch_block_threads))
    return "block_threads must be 0 or a multiple of 32 in [64, 512]";
  if ((p->threads_per_sample != 1 && p->block_threads > kMaxThreads - 32) ||
      (p->batch_threads_per_sample != 1 && p->batch_block_threads > kMaxThreads - 32))
    return "block_threads above 480 needs threads_per_sample = 1 (wider teams add a noise warp)";
  if (p->max_batch < 0 || p->max_batch > 65536) return "max_batch must be in [0, 65536]";
  if (p->max_vehicles < 0 || p->max_vehicles > 65536) return "max_vehicles must be in [0, 65536]";
  if (p->serve_lanes < 0 || p->serve_lanes > 16) return "serve_lanes must be in [0, 16]";
  if (p->serve_max_batch < 0 || p->serve_max_batch > 4096) return "serve_max_batch must be in [0, 4096]";
  if (p->serve_queue < 0 || p->serve_queue > (1 << 20)) return "serve_queue must be in [0, 2^20]";
  if (p->wait_timeout_ms < 0) return "wait_timeout_ms must be >= 0";
  const float pos[] = {p->Ts, p->lambda, p->l1, p->l2, p->h_floor};
  for (float v : pos)
    if (!(v > 0.f) || !std::isfinite(v)) return "Ts, lambda, l1, l2, h_floor must be positive and finite";
  const float fin[] = {p->lh, p->dtheta_max, p->kappa, p->r_inflate, p->Qc, p->Ql, p->Qth, p->R[0],
                       p->R[1], p->R[2], p->mu, p->nu_bar, p->alpha0, p->sigma_alpha, p->ua_lo,
                       p->ua_hi, p->w_alpha, p->rho};
  for (float v : fin)
    if (!std::isfinite(v)) return "parameters must be finite";
  for (int j = 0; j < 3; ++j) {
    if (!std::isfinite(p->z_lo[j]) || !std::isfinite(p->z_hi[j]) || !(p->z_lo[j] <= p->z_hi[j]))
      return "z_lo <= z_hi required";
    if (!(p->sigma[j] >= 0.f) || !std::isfinite(p->sigma[j])) return "sigma must be >= 0";
    if (!(p->w_u[j] + p->rho > 0.f) || !(p->w_u[j] >= 0.f)) return "w_u >= 0 and w_u + rho > 0 required";
  }
  if (!(p->ua_lo <= p->ua_hi)) return "ua_lo <= ua_hi required";
  if (!(p->sigma_alpha >= 0.f)) return "sigma_alpha must be >= 0";
  if (!(p->w_alpha + p->rho > 0.f) || !(p->w_alpha >= 0.f) || !(p->rho >= 0.f))
    return "w_alpha >= 0, rho >= 0 and w_alpha + rho > 0 required";
  if (!(p->q_coll >= 0.f) || !std::isfinite(p->q_coll)) return "q_coll must be >= 0 and finite";
  if (!(p->alpha_stab > 0.f && p->alpha_stab <= 1.f)) return "alpha_stab must be in (0, 1]";
  if (!(p->q_stab[0] > 0.f) || !(p->q_stab[1] > 0.f) || !std::isfinite(p->q_stab[0]) || !std::isfinite(p->q_stab[1]))
    return "q_stab must be positive and finite";
  if (!(p->q_abuf >= 0.f) || !std::isfinite(p->q_abuf)) return "q_abuf must be >= 0 and finite";
  if (!(p->h_buf > 0.f) || !std::isfinite(p->h_buf)) return "h_buf must be positive and finite";
  if (p->n_discs < 1 || p->n_discs > 8) return "n_discs must be in [1, 8]";
  if (p->disc_trailer_mask & ~((1 << p->n_discs) - 1)) return "disc_trailer_mask has bits at or above n_discs";
  for (int m = 0; m < 8; ++m)
    if (!std::isfinite(p->disc_off[m])) return "disc_off must be finite";
  if (p->max_obstacles * p->n_discs > kMaxObstacles) return "max_obstacles * n_discs must be <= 124";
  if ((p->flags & BRMPPI_FLAG_THIRD_ORDER) && (p->n_discs != 1 || p->disc_trailer_mask != 0 || p->disc_off[0] != 0.f))
    return "third-order rows need the single rear-axle disc";
  if ((p->flags & BRMPPI_FLAG_JERK_MODEL) && (p->n_discs != 1 || p->disc_trailer_mask != 0 || p->disc_off[0] != 0.f))
    return "the jerk-input model needs the single rear-axle disc";
  return "";
}

brmppi::KConst make_kconst(const brmppi_params& q) {
  brmppi::KConst k{};
  k.proj = (q.flags & BRMPPI_FLAG_PROJ_NONE) ? 0 : 1;
  k.coll = (q.flags & BRMPPI_FLAG_COLLISION_COST) ? 1 : 0;
  k.obs8 = (q.flags & BRMPPI_FLAG_OBS8) ? 1 : 0;
  k.abuf = (q.flags & BRMPPI_FLAG_ALPHA_BUFFER) ? 1 : 0;
  k.Ts = q.Ts;
  k.hTs2 = 0.5f * q.Ts * q.Ts;
  k.Ts2 = q.Ts * q.Ts;
  k.inv_lambda = 1.0f / q.lambda;
  k.inv_l1 = 1.0f / q.l1;
  k.inv_l2 = 1.0f / q.l2;
  k.k_hitch = q.lh / q.l1;
  k.dtheta_max = q.dtheta_max;
  k.kappa = q.kappa;
  k.r_inflate = q.r_inflate;
  k.Qc = q.Qc;
  k.Ql = q.Ql;
  k.Qth = q.Qth;
  k.R0 = q.R[0];
  k.R1 = q.R[1];
  k.R2 = q.R[2];
  k.mu = q.mu;
  k.nu_bar = q.nu_bar;
  k.zlo0 = q.z_lo[0];
  k.zlo1 = q.z_lo[1];
  k.zlo2 = q.z_lo[2];
  k.zhi0 = q.z_hi[0];
  k.zhi1 = q.z_hi[1];
  k.zhi2 = q.z_hi[2];
  k.sig0 = q.sigma[0];
  k.sig1 = q.sigma[1];
  k.sig2 = q.sigma[2];
  k.alpha0 = q.alpha0;
  k.sigma_alpha = q.sigma_alpha;
  k.ua_lo = q.ua_lo;
  k.ua_hi = q.ua_hi;
  k.w_u0 = q.w_u[0];
  k.w_u1 = q.w_u[1];
  k.w_u2 = q.w_u[2];
  k.pc_u0 = 0.5f * q.rho * (q.z_hi[0] + q.z_lo[0]);
  k.pc_u1 = 0.5f * q.rho * (q.z_hi[1] + q.z_lo[1]);
  k.pc_u2 = 0.5f * q.rho * (q.z_hi[2] + q.z_lo[2]);
  k.m_u0 = q.w_u[0] + q.rho;
  k.m_u1 = q.w_u[1] + q.rho;
  k.inv_m_u0 = 1.0f / (q.w_u[0] + q.rho);
  k.inv_m_u1 = 1.0f / (q.w_u[1] + q.rho);
  k.inv_m_u2 = 1.0f / (q.w_u[2] + q.rho);
  const double m_alpha = static_cast<double>(q.w_alpha) + static_cast<double>(q.rho);
  k.w_am = static_cast<float>(q.w_alpha / m_alpha);
  k.pc_am = static_cast<float>(0.5 * q.rho * (static_cast<double>(q.ua_hi) + q.ua_lo) / m_alpha);
  k.m_a = q.w_alpha + q.rho;
  k.h_floor = q.h_floor;
  k.q_coll = q.q_coll;
  k.q_abuf = q.q_abuf;
  k.inv_hbuf = 1.0f / q.h_buf;
  k.alpha_stab = q.alpha_stab;
  k.inv_qs0 = 1.0f / q.q_stab[0];
  k.inv_qs1 = 1.0f / q.q_stab[1];
  k.third = (q.flags & BRMPPI_FLAG_THIRD_ORDER) ? 1 : 0;
  k.jerk = (q.flags & BRMPPI_FLAG_JERK_MODEL) ? 1 : 0;
  k.Ts3_6 = q.Ts * q.Ts * q.Ts / 6.0f;
  k.nd = q.n_discs;
  k.inv_nd = 1.0f / static_cast<float>(q.n_discs);
  k.discs = (q.n_discs != 1 || q.disc_trailer_mask != 0 || q.disc_off[0] != 0.f) ? 1 : 0;
  for (int m = 0; m < 8; ++m) {
    // lever arms along e1 and e2 (tractor: d, 0; trailer: -lh, -(l2 - d))
    const bool tr = (q.disc_trailer_mask >> m) & 1;
    k.disc_e1[m] = (m < q.n_discs) ? (tr ? -q.lh : q.disc_off[m]) : 0.f;
    k.disc_e2[m] = (m < q.n_discs && tr) ? -(q.l2 - q.disc_off[m]) : 0.f;
  }
  return k;
}

brmppi::SmemCaps make_caps(int n_obs, int n_rows, int n_pts, int H, int tps) {
  brmppi::SmemCaps c{};
  c.obs = 8 * n_obs;
  c.path = brmppi::SmemCaps::pad4(3 * n_pts);
  c.phead = brmppi::SmemCaps::pad4(2 * n_pts);
  c.unom = brmppi::SmemCaps::pad4(3 * H);
  c.ustar = brmppi::SmemCaps::pad4(3 * H + 1);
  c.noise_per_team = tps > 1 ? 8 * philox_blocks(n_rows) : 0;
  c.uh_per_team = 0;
  c.merge = 0;
  return c;
}

size_t smem_bytes(const brmppi::SmemCaps& c, int spb) { return sizeof(float) * static_cast<size_t>(c.total(spb)); }

bool pick_bpt(int tps, int P, int* bpt) {
  // one lane: the lane draws every block (b >= P); wider teams: the row
  // slots of a lane (4 b) must hold its share of the at most 4 P - 4 rows
  // (their blocks are drawn by producer warps or staged in passes)
  for (int b : {1, 2, 3, 4, 5, 6, 8})
    if ((tps == 1 ? b >= P : (4 * P - 4 + tps - 1) / tps <= 4 * b) && brmppi::variant_exists(tps, b)) {
      *bpt = b;
      return true;
    }
  return false;
}

int part_stride_for(int H) { return static_cast<int>(align_up(3 + 3 * static_cast<size_t>(H) + 1, 4)); }

// Heuristic plain shape: a team just wide enough for the Philox blocks (one
// block per lane), 128-thread blocks while that leaves at least two CTAs per
// SM, else 64.  Narrower blocks (then wider teams) while the shared-memory
// tables do not fit.
bool heuristic_plain(const brmppi_ctx* c, int n_obs, int n_pts, Shape* out) {
  const int P = philox_blocks(rows_of(c->prm, n_obs));
  const bool fixed_tps = c->prm.threads_per_sample != 0;
  int tps = c->prm.threads_per_sample;
  if (!fixed_tps) {
    // latency shape: one Philox block per lane; then, while the GPU stays
    // full (at least 4 warps per SM), fewer lanes per sample and more blocks
    // per lane (less work repeated across a team)
    tps = 1;
    while (tps < P && tps < 32) tps <<= 1;
    int b2 = 0;
    while (tps > 1 && pick_bpt(tps / 2, P, &b2) &&
           static_cast<long long>(c->prm.S) * (tps / 2) / 32 >= 4LL * c->num_sms)
      tps >>= 1;
  }
  int bpt = 0;
  if (!pick_bpt(tps, P, &bpt)) return false;
  int threads = c->prm.block_threads;
  const bool fixed_threads = threads != 0;
  if (!fixed_threads) {
    // 128 threads, one CTA per SM where the tiles fit; just over one wave:
    // 64 (a short second wave of small CTAs); more: 256; very few tiles: 64
    // (shapes measured on GB300; the autotuner refines per workload)
    threads = 128;
    const long long tiles = (c->prm.S + threads / tps - 1) / (threads / tps);
    const bool small_ok = 64 / tps >= 2;
    // (producer-warp variants stay at 128: their CTAs grow by up to four
    // warps, and 256 + 128 threads of 128 registers fit one CTA per SM)
    const bool producers = tps > 1 && bpt <= 2;
    if (tiles > c->num_sms)
      threads = (tiles <= c->num_sms + c->num_sms / 4 && small_ok) ? 64 : (producers ? 128 : 256);
    else if (tiles < c->num_sms / 2 && small_ok)
      threads = 64;
  }
  if (threads < tps) return false;
  while (smem_bytes(make_caps(n_obs, rows_of(c->prm, n_obs), n_pts, c->prm.H, tps), threads / tps) > c->smem_limit) {
    if (!fixed_threads && threads > kMinThreads) {
      threads -= 32;
    } else if (!fixed_tps && tps < 32) {
      tps <<= 1;
      if (!pick_bpt(tps, P, &bpt)) return false;
    } else {
      return false;
    }
  }
  out->tps = tps;
  out->bpt = bpt;
  out->threads = threads;
  return true;
}

bool plain_shape(const brmppi_ctx* c, int n_obs, int n_pts, Shape* out) {
  if (c->prm.threads_per_sample == 0 && c->prm.block_threads == 0) {
    auto it = c->tuned.find(n_obs);
    if (it != c->tuned.end()) {
      const brmppi::SmemCaps caps = make_caps(n_obs, rows_of(c->prm, n_obs), n_pts, c->prm.H, it->second.tps);
      if (smem_bytes(caps, it->second.threads / it->second.tps) <= c->smem_limit) {
        *out = it->second;
        return true;
      }
    }
  }
  return heuristic_plain(c, n_obs, n_pts, out);
}

brmppi::Inst make_inst(const double* x0, const float* U_nom, const float* obs, int n_obs, const float* path,
                       int n_pts, float ds, int S, int H, uint64_t seed, uint64_t counter, float* U_out,
                       float* traj_out, float* J_out, float* U_next, int32_t* status, float* part,
                       unsigned int* sync, int spb, int n_discs) {
  brmppi::Inst in{};
  in.x0 = x0;
  in.U_nom = U_nom;
  in.obs = obs;
  in.path = path;
  in.U_out = U_out;
  in.traj_out = traj_out;
  in.J_out = J_out;
  in.U_next = U_next;
  in.status = status;
  in.part = part;
  in.sync = sync;
  in.S = S;
  in.H = H;
  in.n_obs = n_obs;
  in.n_pts = n_pts;
  in.tiles = (S + spb - 1) / spb;
  in.part_stride = part_stride_for(H);
  in.ds = ds;
  in.inv_ds = 1.0f / ds;
  in.inv_ds_d = 1.0 / static_cast<double>(ds);
  in.key0 = static_cast<uint32_t>(seed);
  in.key1 = static_cast<uint32_t>(seed >> 32);
  in.ctr = static_cast<uint32_t>(counter);
  in.P = philox_blocks(n_obs * n_discs);
  return in;
}

void single_launch_options(brmppi::LaunchDesc& L, const Shape& sh, const brmppi::KConst& k, int n_rows, int H,
                           size_t smem_limit) {
  // a single solve on a noise-warp shape: the instantiation with exactly the
  // rows a lane holds, with the tile's applied-input history in shared
  // memory, where both the variant exists and the history fits
  const int spb = sh.threads / sh.tps;
  const int rows = brmppi::exact_rows_variant(sh.tps, sh.bpt, k, n_rows);
  if (rows <= 0) return;
  // those instantiations are compiled for blocks of at most 384 threads
  // (more registers a thread)
  if (brmppi::block_threads(sh.tps, sh.bpt, sh.threads, L.single.P) > brmppi::kMaxRowsBlockThreads) return;
  brmppi::SmemCaps caps = L.caps;
  caps.uh_per_team = 3 * H;
  // those variants merge the instance's tile partials in shared memory
  // (unless the launch only produces its share of the tiles)
  caps.merge = L.single.no_merge ? 0 : L.single.tiles * L.single.part_stride;
  if (smem_bytes(caps, spb) > smem_limit) return;
  L.caps = caps;
  L.rows = rows;
}

brmppi_status check_sizes(brmppi_ctx* c, int32_t n_obs, int32_t n_pts, float ds) {
  if (n_obs < 0 || n_obs > c->prm.max_obstacles) return fail(c, BRMPPI_EINVAL, "n_obs out of [0, max_obstacles]");
  if (n_pts < 2 || n_pts > c->prm.max_path_pts) return fail(c, BRMPPI_EINVAL, "n_pts out of [2, max_path_pts]");
  if (!(ds > 0.f) || !std::isfinite(ds)) return fail(c, BRMPPI_EINVAL, "ds must be positive and finite");
  return BRMPPI_OK;
}

brmppi_status enqueue_plain_sized(brmppi_ctx* c, const Shape& sh, int S, int H, const double* x0,
                                  const float* U_nom, const float* obs, int32_t n_obs, const float* path,
                                  int32_t n_pts, float ds, uint64_t seed, uint64_t counter, float* U_out,
                                  float* traj_out, float* J_out, float* U_next, int32_t* status, float* states_out,
                                  float* u_safe, cudaStream_t stream, float* inputs_out = nullptr,
                                  float* J_lo_out = nullptr, float* tiles_out = nullptr, int tile0 = 0,
                                  int n_tiles = 0) {
  const int spb = sh.threads / sh.tps;
  brmppi::LaunchDesc L{};
  L.single = make_inst(x0, U_nom, obs, n_obs, path, n_pts, ds, S, H, seed, counter, U_out, traj_out, J_out,
                       U_next, status, c->d_part, c->d_sync, spb, c->prm.n_discs);
  L.single.states_out = states_out;
  L.single.u_safe = u_safe;
  L.single.inputs_out = inputs_out;
  L.single.J_lo_out = J_lo_out;
  if (tiles_out) {
    // a share of the instance's tiles: partials to the caller, no merge
    L.single.part = tiles_out;
    L.single.tile_base = tile0;
    L.single.no_merge = 1;
  }
  L.caps = make_caps(n_obs, rows_of(c->prm, n_obs), n_pts, H, sh.tps);
  L.uh = c->d_uh;
  L.uh_stride = 3 * H * spb;
  const brmppi::KConst k = make_kconst(c->prm);
  single_launch_options(L, sh, k, rows_of(c->prm, n_obs), H, c->smem_limit);
  const size_t smem = smem_bytes(L.caps, spb);
  const int tiles = tiles_out ? n_tiles : L.single.tiles;  // CTAs of the launch
  if (smem > c->smem_limit) return fail(c, BRMPPI_EINVAL, "shared memory need exceeds the device limit");
  if ((!tiles_out && static_cast<size_t>(tiles) > c->part_tiles) ||
      static_cast<size_t>(tiles) * static_cast<size_t>(L.uh_stride) > c->uh_floats)
    return fail(c, BRMPPI_EINVAL, "launch shape exceeds the context's scratch");
  cudaError_t e = brmppi::launch_solve(sh.tps, sh.bpt, tiles, sh.threads, smem, stream, k, L, L.single.P);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  if (u_safe) {
    // the stabilizer on (x0, U*[0]): one thread, after the solve
    e = brmppi::launch_stabilize(k, x0, U_out, 1, u_safe, stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stabilizer launch");
  }
  return BRMPPI_OK;
}

brmppi_status enqueue_plain(brmppi_ctx* c, const Shape& sh, const double* x0, const float* U_nom,
                            const float* obs, int32_t n_obs, const float* path, int32_t n_pts, float ds,
                            uint64_t seed, uint64_t counter, float* U_out, float* traj_out, float* J_out,
                            float* U_next, int32_t* status, cudaStream_t stream) {
  return enqueue_plain_sized(c, sh, c->prm.S, c->prm.H, x0, U_nom, obs, n_obs, path, n_pts, ds, seed, counter,
                             U_out, traj_out, J_out, U_next, status, nullptr, nullptr, stream);
}

// ------------------------------------------------------------- batches
cudaError_t lane_alloc(Lane& L, int max_batch, size_t S, size_t H, int num_sms, size_t part_stride) {
  const size_t nb = static_cast<size_t>(max_batch);
  const size_t tiles_per_inst = (S + kMinBatchSpb - 1) / kMinBatchSpb;
  L.max_batch = max_batch;
  L.max_work = nb * tiles_per_inst;
  L.bpart_floats = L.max_work * part_stride;
  L.buh_floats = static_cast<size_t>(num_sms) * kMaxResidentThreads * 3 * H;
  cudaError_t e;
  if ((e = dev_alloc(&L.d_inst, sizeof(brmppi::Inst) * nb)) != cudaSuccess) return e;
  if ((e = dev_alloc(&L.d_work, sizeof(int2) * L.max_work)) != cudaSuccess) return e;
  if ((e = dev_alloc(&L.d_work_ctr, sizeof(unsigned int) * 2)) != cudaSuccess) return e;
  if ((e = cudaMemset(L.d_work_ctr, 0, sizeof(unsigned int) * 2)) != cudaSuccess) return e;
  if ((e = dev_alloc(&L.d_bpart, sizeof(float) * L.bpart_floats)) != cudaSuccess) return e;
  if ((e = dev_alloc(&L.d_bsync, sizeof(unsigned int) * 2 * nb)) != cudaSuccess) return e;
  if ((e = cudaMemset(L.d_bsync, 0, sizeof(unsigned int) * 2 * nb)) != cudaSuccess) return e;
  if ((e = dev_alloc(&L.d_buh, sizeof(float) * L.buh_floats)) != cudaSuccess) return e;
  if ((e = host_alloc(&L.h_inst, sizeof(brmppi::Inst) * nb)) != cudaSuccess) return e;
  if ((e = host_alloc(&L.h_work, sizeof(int2) * L.max_work)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&L.upload_done, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&L.batch_done, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaSuccess;
}

bool lane_free(Lane& L, int timeout_ms) {
  if (L.pending && L.batch_done && wait_event(L.batch_done, timeout_ms) == cudaErrorNotReady) {
    // the lane's last batch is still running: leave its buffers allocated
    if (L.stream) cudaStreamDestroy(L.stream);
    L = Lane();
    return false;
  }
  cudaFree(L.d_inst);
  cudaFree(L.d_work);
  cudaFree(L.d_work_ctr);
  cudaFree(L.d_bpart);
  cudaFree(L.d_bsync);
  cudaFree(L.d_buh);
  cudaFreeHost(L.h_inst);
  cudaFreeHost(L.h_work);
  if (L.upload_done) cudaEventDestroy(L.upload_done);
  if (L.batch_done) cudaEventDestroy(L.batch_done);
  if (L.stream) cudaStreamDestroy(L.stream);
  L = Lane();
  return true;
}

namespace {

bool batch_shape_default(const brmppi_ctx* c, int max_P, Shape* out) {
  Shape s;
  s.tps = c->prm.batch_threads_per_sample;
  s.threads = c->prm.batch_block_threads;
  if (s.tps == 0 && s.threads == 0 && c->batch_tuned) {
    s = c->batch_shape;
  } else {
    // the optional terms' rows carry a steer-rate column: teams wide enough
    // for at most two Philox blocks per lane keep them out of local memory
    const bool ext = brmppi::needs_ext(make_kconst(c->prm));
    if (s.tps == 0) s.tps = ext ? ext_team_width(max_P) : 1;
    if (s.threads == 0) s.threads = std::max(128, kMinBatchSpb * s.tps);
  }
  while (!pick_bpt(s.tps, max_P, &s.bpt)) {
    if (s.tps >= 32) return false;
    s.tps <<= 1;
  }
  if (s.threads < s.tps || s.threads / s.tps < kMinBatchSpb) return false;
  *out = s;
  return true;
}

brmppi_status launch_batch(brmppi_ctx* c, Lane& L, const BatchPlan& plan, cudaStream_t stream) {
  brmppi::LaunchDesc D{};
  D.inst = L.d_inst;
  D.work = L.d_work;
  D.n_work = plan.n_work;
  D.work_ctr = L.d_work_ctr;
  D.uh = L.d_buh;
  D.uh_stride = 3 * plan.Hmax * (plan.shape.threads / plan.shape.tps);
  D.caps = plan.caps;
  const brmppi::KConst k = make_kconst(c->prm);
  cudaError_t e = brmppi::launch_solve(plan.shape.tps, plan.shape.bpt, plan.grid, plan.shape.threads, plan.smem,
                                       stream, k, D, plan.P);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch kernel launch");
  if (plan.any_u_safe && (e = brmppi::launch_stabilize_table(k, L.d_inst, plan.n_inst, stream)) != cudaSuccess)
    return cuda_fail(c, e, "stabilizer launch");
  return BRMPPI_OK;
}

}  // namespace

// Validate the instances, fill the instance table and the longest-first
// work list (host staging), and size the launch.
brmppi_status plan_batch(brmppi_ctx* c, Lane& L, const brmppi_instance* inst, int32_t n, const Shape* forced,
                         brmppi::Inst* h_inst, int2* h_work, BatchPlan* plan) {
  if (L.max_batch <= 0) return fail(c, BRMPPI_EINVAL, "context created without batch capacity (max_batch)");
  if (!inst || n < 1 || n > L.max_batch) return fail(c, BRMPPI_EINVAL, "n out of [1, max_batch]");
  int max_P = 1, Hmax = 1, nobs_max = 0, npts_max = 2;
  for (int i = 0; i < n; ++i) {
    const brmppi_instance& q = inst[i];
    if (!q.x0 || !q.U_nom || !q.path || !q.U_out || (q.n_obs > 0 && !q.obs))
      return fail(c, BRMPPI_EINVAL, "instance " + std::to_string(i) + ": NULL buffer");
    if (q.S < 1 || q.S > c->prm.S || q.H < 1 || q.H > c->prm.H)
      return fail(c, BRMPPI_EINVAL, "instance " + std::to_string(i) + ": S or H beyond the capacity");
    brmppi_status st = check_sizes(c, q.n_obs, q.n_pts, q.ds);
    if (st != BRMPPI_OK) return fail(c, st, "instance " + std::to_string(i) + ": " + c->err);
    max_P = std::max(max_P, philox_blocks(rows_of(c->prm, q.n_obs)));
    Hmax = std::max(Hmax, static_cast<int>(q.H));
    nobs_max = std::max(nobs_max, static_cast<int>(q.n_obs));
    npts_max = std::max(npts_max, static_cast<int>(q.n_pts));
  }
  // The kernel variant follows the context's obstacle capacity, not this
  // batch's content: every batch on a context runs the same instantiation,
  // so a solve gives the same bits alone and in any mix.
  const int P_cap = std::max(max_P, philox_blocks(rows_of(c->prm, c->prm.max_obstacles)));
  Shape sh;
  if (forced) {
    sh = *forced;
    if (!pick_bpt(sh.tps, P_cap, &sh.bpt)) return fail(c, BRMPPI_EINVAL, "no variant for this team width");
  } else if (!batch_shape_default(c, P_cap, &sh)) {
    return fail(c, BRMPPI_EINVAL, "no batch launch shape for these instances");
  }
  const int spb = sh.threads / sh.tps;
  const brmppi::SmemCaps caps = make_caps(nobs_max, rows_of(c->prm, nobs_max), npts_max, Hmax, sh.tps);
  const size_t smem = smem_bytes(caps, spb);
  if (smem > c->smem_limit) return fail(c, BRMPPI_EINVAL, "batch tables exceed shared memory");
  size_t pool = 0;
  std::vector<std::pair<long long, int2>> items;
  items.reserve(L.max_work);
  for (int i = 0; i < n; ++i) {
    const brmppi_instance& q = inst[i];
    const int H = q.H;
    brmppi::Inst in = make_inst(q.x0, q.U_nom, q.obs, q.n_obs, q.path, q.n_pts, q.ds, q.S, H, q.seed, q.counter,
                                q.U_out, q.traj_out, q.J_out, q.U_next, q.status, nullptr, L.d_bsync + 2 * i, spb,
                                c->prm.n_discs);
    in.states_out = q.states_out;
    in.u_safe = q.u_safe_out;
    in.inputs_out = q.inputs_out;
    in.J_lo_out = q.J_lo_out;
    if (q.u_safe_out) plan->any_u_safe = true;
    in.part = L.d_bpart + pool;
    pool += static_cast<size_t>(in.tiles) * static_cast<size_t>(in.part_stride);
    if (pool > L.bpart_floats) return fail(c, BRMPPI_EINVAL, "batch partials exceed the context's pool");
    h_inst[i] = in;
    const long long cost = static_cast<long long>(H) * (8 + q.n_obs);
    for (int t = 0; t < in.tiles; ++t) items.push_back({cost, make_int2(i, t)});
  }
  if (items.size() > L.max_work) return fail(c, BRMPPI_EINVAL, "too many work items");
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<long long, int2>& a, const std::pair<long long, int2>& b) {
                     return a.first > b.first;
                   });
  for (size_t j = 0; j < items.size(); ++j) h_work[j] = items[j].second;
  const int occ =
      brmppi::variant_occupancy(sh.tps, sh.bpt, sh.threads, smem, brmppi::needs_ext(make_kconst(c->prm)), P_cap);
  if (occ < 1) return fail(c, BRMPPI_EINVAL, "batch launch shape cannot be resident");
  int grid = occ * c->num_sms;
  if (grid > static_cast<int>(items.size())) grid = static_cast<int>(items.size());
  if (static_cast<size_t>(grid) * 3 * Hmax * spb > L.buh_floats)
    return fail(c, BRMPPI_EINVAL, "batch history scratch too small");
  plan->shape = sh;
  plan->P = P_cap;
  plan->n_inst = n;
  plan->n_work = static_cast<int>(items.size());
  plan->grid = grid;
  plan->Hmax = Hmax;
  plan->caps = caps;
  plan->smem = smem;
  return BRMPPI_OK;
}

brmppi_status upload_and_launch(brmppi_ctx* c, Lane& L, const BatchPlan& plan, const brmppi::Inst* h_inst,
                                const int2* h_work, cudaStream_t stream) {
  cudaError_t e;
  if (L.pending && (e = cudaStreamWaitEvent(stream, L.batch_done, 0)) != cudaSuccess)
    return cuda_fail(c, e, "wait for the previous batch");
  if ((e = cudaMemcpyAsync(L.d_inst, h_inst, sizeof(brmppi::Inst) * plan.n_inst, cudaMemcpyHostToDevice,
                           stream)) != cudaSuccess)
    return cuda_fail(c, e, "instance table upload");
  if ((e = cudaMemcpyAsync(L.d_work, h_work, sizeof(int2) * plan.n_work, cudaMemcpyHostToDevice, stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "work list upload");
  return launch_batch(c, L, plan, stream);
}

}  // namespace brmppi_host

extern "C" {

void brmppi_default_params(brmppi_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->abi_version = BRMPPI_ABI_VERSION;
  p->S = 256;
  p->H = 30;
  p->max_obstacles = 16;
  p->max_path_pts = 4096;
  p->Ts = 0.05f;
  p->lambda = 1.0f;
  p->l1 = 4.0f;
  p->lh = 0.5f;
  p->l2 = 8.0f;
  p->dtheta_max = 0.9f;
  p->kappa = 0.1f;
  p->Qc = 10.f;
  p->Ql = 10.f;
  p->Qth = 5.f;
  p->R[0] = 0.1f;
  p->R[1] = 0.1f;
  p->R[2] = 0.01f;
  p->mu = 1.f;
  p->nu_bar = 3.f;
  p->z_lo[0] = -2.f;
  p->z_lo[1] = -0.6f;
  p->z_lo[2] = 0.f;
  p->z_hi[0] = 2.f;
  p->z_hi[1] = 0.6f;
  p->z_hi[2] = 3.f;
  p->sigma[0] = 0.5f;
  p->sigma[1] = 0.3f;
  p->sigma[2] = 0.5f;
  p->alpha0 = 0.5f;
  p->sigma_alpha = 0.1f;
  p->ua_lo = -0.5f;
  p->ua_hi = 0.5f;
  p->w_u[0] = p->w_u[1] = p->w_u[2] = 1.f;
  p->w_alpha = 1.f;
  p->rho = 0.01f;
  p->h_floor = 1e-6f;
  p->q_coll = 100.0f;
  p->alpha_stab = 0.5f;
  p->q_stab[0] = 1.0f;
  p->q_stab[1] = 1.0f;
  p->q_abuf = 10.0f;
  p->h_buf = 0.5f;
  p->n_discs = 1;
  p->disc_trailer_mask = 0;
  for (int m = 0; m < 8; ++m) p->disc_off[m] = 0.f;
}

brmppi_status brmppi_create(const brmppi_params* p, int device, brmppi_ctx** out) {
  if (!out) return fail(nullptr, BRMPPI_EINVAL, "out is NULL");
  *out = nullptr;
  const std::string bad = check_params(p);
  if (!bad.empty()) return fail(nullptr, BRMPPI_EINVAL, bad);
  brmppi_ctx* c = new (std::nothrow) brmppi_ctx();
  if (!c) return fail(nullptr, BRMPPI_ENOMEM, "host allocation failed");
  c->prm = *p;
  c->device = device;
  auto bail = [&](cudaError_t err, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(err);
    brmppi_destroy(c);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? BRMPPI_ENOMEM : BRMPPI_ECUDA, m);
  };
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return bail(e, "cudaSetDevice");
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return bail(e, "cudaDeviceGetAttribute");
  int dev_smem = 0;
  if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess)
    return bail(e, "cudaDeviceGetAttribute");
  c->smem_limit = static_cast<size_t>(dev_smem) - 1024;  // static shared memory of the kernel
  if ((e = brmppi::set_smem_limit(c->smem_limit)) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  {
    Shape s;
    if (!heuristic_plain(c, p->max_obstacles, p->max_path_pts, &s)) {
      brmppi_destroy(c);
      return fail(nullptr, BRMPPI_EINVAL, "no launch shape fits these capacities in shared memory");
    }
  }
  const size_t H = static_cast<size_t>(p->H), S = static_cast<size_t>(p->S);
  c->off_unom = 64;
  c->off_obs = align_up(c->off_unom + sizeof(float) * 3 * H, 16);
  c->off_path = align_up(c->off_obs + sizeof(float) * obs_floats(*p) * static_cast<size_t>(p->max_obstacles), 16);
  c->in_bytes = align_up(c->off_path + sizeof(float) * 3 * static_cast<size_t>(p->max_path_pts), 16);
  c->out_floats = 3 * H + 7 * (H + 1) + 1;
  c->part_stride = static_cast<size_t>(part_stride_for(p->H));
  c->part_tiles = (S + 1) / 2;               // tiles of at least two samples
  c->uh_floats = (S + kMaxThreads) * 3 * H;  // one tile slot per CTA, rounded up
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "cudaStreamCreate");
  if ((e = dev_alloc(&c->d_in, c->in_bytes)) != cudaSuccess) return bail(e, "cudaMalloc(in)");
  if ((e = dev_alloc(&c->d_J, sizeof(float) * S)) != cudaSuccess) return bail(e, "cudaMalloc(J)");
  if ((e = dev_alloc(&c->d_part, sizeof(float) * c->part_stride * c->part_tiles)) != cudaSuccess)
    return bail(e, "cudaMalloc(partials)");
  if ((e = dev_alloc(&c->d_uh, sizeof(float) * c->uh_floats)) != cudaSuccess) return bail(e, "cudaMalloc(history)");
  if ((e = dev_alloc(&c->d_sync, sizeof(unsigned int) * 4)) != cudaSuccess) return bail(e, "cudaMalloc(sync)");
  if ((e = cudaMemset(c->d_sync, 0, sizeof(unsigned int) * 4)) != cudaSuccess) return bail(e, "cudaMemset");
  if ((e = dev_alloc(&c->d_out, sizeof(float) * c->out_floats)) != cudaSuccess) return bail(e, "cudaMalloc(out)");
  if ((e = host_alloc(&c->h_in, c->in_bytes)) != cudaSuccess) return bail(e, "cudaMallocHost(in)");
  if ((e = host_alloc(&c->h_out, sizeof(float) * c->out_floats)) != cudaSuccess)
    return bail(e, "cudaMallocHost(out)");
  if (p->max_batch > 0 && (e = lane_alloc(c->batch, p->max_batch, S, H, c->num_sms, c->part_stride)) != cudaSuccess)
    return bail(e, "batch buffers");
  if (p->max_vehicles > 0) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "cudaDeviceSynchronize");
    brmppi_status st = server_create(c);
    if (st != BRMPPI_OK) {
      std::string m = c->err;
      brmppi_destroy(c);
      return fail(nullptr, st, "serving loop: " + m);
    }
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "cudaDeviceSynchronize");
  *out = c;
  return BRMPPI_OK;
}

brmppi_status brmppi_destroy(brmppi_ctx* c) {
  if (!c) return BRMPPI_OK;
  cudaSetDevice(c->device);
  const int limit = wait_limit_ms(c->prm);
  // every wait bounded; once one gives up nothing more is freed (a free may
  // wait for the device), the buffers stay allocated and the context goes
  bool done = server_destroy(c);
  if (done && c->stream && wait_stream(c->stream, limit) != cudaSuccess) done = false;
  if (done) done = lane_free(c->batch, limit);
  if (done) {
    cudaFree(c->d_in);
    cudaFree(c->d_J);
    cudaFree(c->d_part);
    cudaFree(c->d_uh);
    cudaFree(c->d_sync);
    cudaFreeHost(c->h_in);
    cudaFreeHost(c->h_out);
    cudaFree(c->d_out);
  } else if (c->batch.stream) {
    cudaStreamDestroy(c->batch.stream);
  }
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return done ? BRMPPI_OK : BRMPPI_ETIMEDOUT;
}

void brmppi_inject_alloc_failure(int32_t n) { g_fail_alloc_in.store(n > 0 ? n : 0); }

const char* brmppi_last_error(const brmppi_ctx* c) {
  if (!c) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_err.c_str();
  }
  return c->err.c_str();
}

brmppi_status brmppi_solve(brmppi_ctx* c, const double x0[7], const float* U_nom, const float* obs,
                           int32_t n_obs, const float* path, int32_t n_pts, float ds, uint64_t seed,
                           uint64_t counter, float* U_out, float* traj_out, float* J_out) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (!x0 || !U_nom || !path || !U_out || (n_obs > 0 && !obs)) return fail(c, BRMPPI_EINVAL, "NULL buffer");
  brmppi_status st = check_sizes(c, n_obs, n_pts, ds);
  if (st != BRMPPI_OK) return st;
  const int nx = state_dim(c->prm);
  for (int j = 0; j < nx; ++j)
    if (!std::isfinite(x0[j])) return fail(c, BRMPPI_ENONFINITE, "x0 is not finite");
  const int of = obs_floats(c->prm);
  for (int o = 0; o < n_obs; ++o)
    if (!exponent_ok(c->prm, obs[of * o + 5])) return fail(c, BRMPPI_EINVAL, "unsupported obstacle exponent");
  if (!path_turns_ok(path, n_pts)) return fail(c, BRMPPI_EINVAL, "path headings of consecutive rows differ by more than pi/4");
  Shape sh;
  if (!plain_shape(c, n_obs, n_pts, &sh)) return fail(c, BRMPPI_EINVAL, "no launch shape for this size");
  const int H = c->prm.H;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  // stage: x0 | U_nom | obs | path  (one pinned buffer, one copy)
  std::memcpy(c->h_in, x0, nx * sizeof(double));
  std::memcpy(c->h_in + c->off_unom, U_nom, sizeof(float) * 3 * H);
  if (n_obs > 0) std::memcpy(c->h_in + c->off_obs, obs, sizeof(float) * of * n_obs);
  std::memcpy(c->h_in + c->off_path, path, sizeof(float) * 3 * n_pts);
  const size_t in_used = c->off_path + sizeof(float) * 3 * n_pts;
  if ((e = cudaMemcpyAsync(c->d_in, c->h_in, in_used, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "H2D copy");
  // the kernel writes U*, the optimal trajectory and the status word
  // straight into the pinned output buffer (mapped into the device's
  // address space): no device-to-host copy follows the launch
  float* dU = reinterpret_cast<float*>(c->h_out);
  float* dT = dU + 3 * H;
  int32_t* dS = reinterpret_cast<int32_t*>(dT + 7 * (H + 1));
  st = enqueue_plain(c, sh, reinterpret_cast<const double*>(c->d_in),
                     reinterpret_cast<const float*>(c->d_in + c->off_unom),
                     reinterpret_cast<const float*>(c->d_in + c->off_obs), n_obs,
                     reinterpret_cast<const float*>(c->d_in + c->off_path), n_pts, ds, seed, counter, dU, dT,
                     J_out ? c->d_J : nullptr, nullptr, dS, c->stream);
  if (st != BRMPPI_OK) return st;
  if (J_out && (e = cudaMemcpyAsync(J_out, c->d_J, sizeof(float) * c->prm.S, cudaMemcpyDeviceToHost, c->stream)) !=
                   cudaSuccess)
    return cuda_fail(c, e, "D2H copy (J)");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "stream sync");
  int32_t kst;
  std::memcpy(&kst, c->h_out + 3 * H + 7 * (H + 1), sizeof(int32_t));
  if (kst == BRMPPI_EINVAL) return fail(c, BRMPPI_EINVAL, "kernel rejected the inputs");
  std::memcpy(U_out, c->h_out, sizeof(float) * 3 * H);
  if (traj_out) std::memcpy(traj_out, c->h_out + 3 * H, sizeof(float) * 7 * (H + 1));
  if (kst == BRMPPI_ENONFINITE) return fail(c, BRMPPI_ENONFINITE, "no rollout had a finite cost");
  return BRMPPI_OK;
}

brmppi_status brmppi_solve_device(brmppi_ctx* c, const double* x0_dev, const float* U_nom_dev,
                                  const float* obs_dev, int32_t n_obs, const float* path_dev, int32_t n_pts,
                                  float ds, uint64_t seed, uint64_t counter, float* U_out_dev,
                                  float* traj_out_dev, float* J_out_dev, float* U_next_dev, int32_t* status_dev,
                                  void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (!x0_dev || !U_nom_dev || !path_dev || !U_out_dev || (n_obs > 0 && !obs_dev))
    return fail(c, BRMPPI_EINVAL, "NULL buffer");
  brmppi_status st = check_sizes(c, n_obs, n_pts, ds);
  if (st != BRMPPI_OK) return st;
  Shape sh;
  if (!plain_shape(c, n_obs, n_pts, &sh)) return fail(c, BRMPPI_EINVAL, "no launch shape for this size");
  return enqueue_plain(c, sh, x0_dev, U_nom_dev, obs_dev, n_obs, path_dev, n_pts, ds, seed, counter, U_out_dev,
                       traj_out_dev, J_out_dev, U_next_dev, status_dev, static_cast<cudaStream_t>(stream));
}

brmppi_status brmppi_solve_device_ex(brmppi_ctx* c, const brmppi_instance* q, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (!q) return fail(c, BRMPPI_EINVAL, "NULL instance");
  if (!q->x0 || !q->U_nom || !q->path || !q->U_out || (q->n_obs > 0 && !q->obs))
    return fail(c, BRMPPI_EINVAL, "NULL buffer");
  if (q->S < 1 || q->S > c->prm.S || q->H < 1 || q->H > c->prm.H)
    return fail(c, BRMPPI_EINVAL, "S or H beyond the context's capacity");
  brmppi_status st = check_sizes(c, q->n_obs, q->n_pts, q->ds);
  if (st != BRMPPI_OK) return st;
  Shape sh;
  if (!plain_shape(c, q->n_obs, q->n_pts, &sh)) return fail(c, BRMPPI_EINVAL, "no launch shape for this size");
  return enqueue_plain_sized(c, sh, q->S, q->H, q->x0, q->U_nom, q->obs, q->n_obs, q->path, q->n_pts, q->ds,
                             q->seed, q->counter, q->U_out, q->traj_out, q->J_out, q->U_next, q->status,
                             q->states_out, q->u_safe_out, static_cast<cudaStream_t>(stream), q->inputs_out,
                             q->J_lo_out);
}

namespace {

// Validation and launch shape shared by the tile-partition entry points.
brmppi_status tile_plan(brmppi_ctx* c, const brmppi_instance* q, bool need_u_out, Shape* sh, int* n_tiles) {
  if (!q) return fail(c, BRMPPI_EINVAL, "NULL instance");
  if (!q->x0 || !q->U_nom || !q->path || (need_u_out && !q->U_out) || (q->n_obs > 0 && !q->obs))
    return fail(c, BRMPPI_EINVAL, "NULL buffer");
  if (q->S < 1 || q->S > c->prm.S || q->H < 1 || q->H > c->prm.H)
    return fail(c, BRMPPI_EINVAL, "S or H beyond the context's capacity");
  brmppi_status st = check_sizes(c, q->n_obs, q->n_pts, q->ds);
  if (st != BRMPPI_OK) return st;
  if (!plain_shape(c, q->n_obs, q->n_pts, sh)) return fail(c, BRMPPI_EINVAL, "no launch shape for this size");
  const int spb = sh->threads / sh->tps;
  *n_tiles = (q->S + spb - 1) / spb;
  return BRMPPI_OK;
}

}  // namespace

brmppi_status brmppi_tile_layout(brmppi_ctx* c, const brmppi_instance* q, int32_t* n_tiles, int32_t* tile_floats) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  Shape sh;
  int nt = 0;
  brmppi_status st = tile_plan(c, q, false, &sh, &nt);
  if (st != BRMPPI_OK) return st;
  if (n_tiles) *n_tiles = nt;
  if (tile_floats) *tile_floats = part_stride_for(q->H);
  return BRMPPI_OK;
}

brmppi_status brmppi_solve_tiles(brmppi_ctx* c, const brmppi_instance* q, int32_t tile0, int32_t n_tiles,
                                 float* tiles_out, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  Shape sh;
  int nt = 0;
  brmppi_status st = tile_plan(c, q, false, &sh, &nt);
  if (st != BRMPPI_OK) return st;
  if (!tiles_out) return fail(c, BRMPPI_EINVAL, "NULL tiles_out");
  if ((reinterpret_cast<uintptr_t>(tiles_out) & 15) != 0) return fail(c, BRMPPI_EINVAL, "tiles_out not 16-byte aligned");
  if (tile0 < 0 || n_tiles < 1 || tile0 + n_tiles > nt)
    return fail(c, BRMPPI_EINVAL, "tile range out of [0, " + std::to_string(nt) + ")");
  return enqueue_plain_sized(c, sh, q->S, q->H, q->x0, q->U_nom, q->obs, q->n_obs, q->path, q->n_pts, q->ds,
                             q->seed, q->counter, q->U_out, nullptr, q->J_out, nullptr, nullptr, q->states_out,
                             nullptr, static_cast<cudaStream_t>(stream), q->inputs_out, q->J_lo_out, tiles_out, tile0,
                             n_tiles);
}

brmppi_status brmppi_merge_tiles(brmppi_ctx* c, const brmppi_instance* q, const float* tiles, int32_t n_tiles,
                                 void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  Shape sh;
  int nt = 0;
  brmppi_status st = tile_plan(c, q, true, &sh, &nt);
  if (st != BRMPPI_OK) return st;
  if (!tiles) return fail(c, BRMPPI_EINVAL, "NULL tiles");
  if (n_tiles != nt) return fail(c, BRMPPI_EINVAL, "the merge needs all " + std::to_string(nt) + " tiles of the instance");
  const int spb = sh.threads / sh.tps;
  brmppi::Inst in = make_inst(q->x0, q->U_nom, q->obs, q->n_obs, q->path, q->n_pts, q->ds, q->S, q->H, q->seed,
                              q->counter, q->U_out, q->traj_out, q->J_out, q->U_next, q->status,
                              const_cast<float*>(tiles), c->d_sync, spb, c->prm.n_discs);
  const brmppi::SmemCaps caps = make_caps(q->n_obs, rows_of(c->prm, q->n_obs), q->n_pts, q->H, sh.tps);
  const size_t smem = smem_bytes(caps, 1);
  if (smem > c->smem_limit) return fail(c, BRMPPI_EINVAL, "shared memory need exceeds the device limit");
  const cudaError_t e = brmppi::launch_merge_tiles(make_kconst(c->prm), in, caps, smem, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "merge launch");
  return BRMPPI_OK;
}

brmppi_status brmppi_solve_batch(brmppi_ctx* c, const brmppi_instance* inst, int32_t n, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  cudaError_t e;
  Lane& L = c->batch;
  if (L.pending && (e = cudaEventSynchronize(L.upload_done)) != cudaSuccess)
    return cuda_fail(c, e, "wait for the previous upload");
  BatchPlan plan;
  brmppi_status st = plan_batch(c, L, inst, n, nullptr, L.h_inst, L.h_work, &plan);
  if (st != BRMPPI_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = upload_and_launch(c, L, plan, L.h_inst, L.h_work, s);
  if (st != BRMPPI_OK) return st;
  // the uploads are consumed once the kernel has finished
  if ((e = cudaEventRecord(L.upload_done, s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  if ((e = cudaEventRecord(L.batch_done, s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  L.pending = true;
  return BRMPPI_OK;
}

brmppi_status brmppi_batch_capture(brmppi_ctx* c, const brmppi_instance* inst, int32_t n, brmppi_graph** out) {
  if (!c || !out) return BRMPPI_EINVAL;
  c->err.clear();
  *out = nullptr;
  Lane& L = c->batch;
  if (L.max_batch <= 0) return fail(c, BRMPPI_EINVAL, "context created without batch capacity (max_batch)");
  brmppi_graph* g = new (std::nothrow) brmppi_graph();
  if (!g) return fail(c, BRMPPI_ENOMEM, "host allocation failed");
  g->ctx = c;
  cudaError_t e;
  auto bail = [&](brmppi_status st) {
    brmppi_graph_destroy(g);
    return st;
  };
  if ((e = host_alloc(&g->h_inst, sizeof(brmppi::Inst) * L.max_batch)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMallocHost(graph table)"));
  if ((e = host_alloc(&g->h_work, sizeof(int2) * L.max_work)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMallocHost(graph work)"));
  BatchPlan plan;
  brmppi_status st = plan_batch(c, L, inst, n, nullptr, g->h_inst, g->h_work, &plan);
  if (st != BRMPPI_OK) return bail(st);
  if (L.pending && (e = cudaEventSynchronize(L.batch_done)) != cudaSuccess)
    return bail(cuda_fail(c, e, "wait for the previous batch"));
  L.pending = false;
  if ((e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaStreamBeginCapture"));
  st = upload_and_launch(c, L, plan, g->h_inst, g->h_work, c->stream);
  e = cudaStreamEndCapture(c->stream, &g->graph);
  if (st != BRMPPI_OK) return bail(st);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamEndCapture"));
  if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaGraphInstantiate"));
  *out = g;
  return BRMPPI_OK;
}

brmppi_status brmppi_graph_launch(brmppi_graph* g, void* stream) {
  if (!g || !g->exec) return BRMPPI_EINVAL;
  brmppi_ctx* c = g->ctx;
  Lane& L = c->batch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (L.pending && (e = cudaStreamWaitEvent(s, L.batch_done, 0)) != cudaSuccess)
    return cuda_fail(c, e, "wait for the previous batch");
  if ((e = cudaGraphLaunch(g->exec, s)) != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  if ((e = cudaEventRecord(L.batch_done, s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  if ((e = cudaEventRecord(L.upload_done, s)) != cudaSuccess) return cuda_fail(c, e, "cudaEventRecord");
  L.pending = true;
  return BRMPPI_OK;
}

void brmppi_graph_destroy(brmppi_graph* g) {
  if (!g) return;
  if (g->exec) {
    if (g->ctx->batch.pending) cudaEventSynchronize(g->ctx->batch.batch_done);
    cudaGraphExecDestroy(g->exec);
  }
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFreeHost(g->h_inst);
  cudaFreeHost(g->h_work);
  delete g;
}

brmppi_status brmppi_autotune(brmppi_ctx* c, const double* x0, const float* U_nom, const float* obs, int32_t n_obs,
                              const float* path, int32_t n_pts, float ds, int32_t reps, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (!x0 || !U_nom || !path || (n_obs > 0 && !obs)) return fail(c, BRMPPI_EINVAL, "NULL buffer");
  brmppi_status st = check_sizes(c, n_obs, n_pts, ds);
  if (st != BRMPPI_OK) return st;
  if (reps < 1) reps = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int P = philox_blocks(rows_of(c->prm, n_obs));
  const int H = c->prm.H;
  float* dU = c->d_out;  // device scratch: the timed launches' outputs are not read
  float* dT = dU + 3 * H;
  Shape best;
  float best_ms = 1e30f;
  for (int tps : {1, 2, 4, 8, 16, 32}) {
    const brmppi::SmemCaps caps = make_caps(n_obs, rows_of(c->prm, n_obs), n_pts, H, tps);
    int bpt;
    if (!pick_bpt(tps, P, &bpt)) continue;
    for (int threads : {64, 128, 256}) {
      if (threads < tps || threads / tps < 2) continue;
      const int spb = threads / tps;
      if (smem_bytes(caps, spb) > c->smem_limit) continue;
      const size_t tiles = (static_cast<size_t>(c->prm.S) + spb - 1) / spb;
      if (tiles > c->part_tiles || tiles * 3 * H * spb > c->uh_floats) continue;
      Shape sh;
      sh.tps = tps;
      sh.bpt = bpt;
      sh.threads = threads;
      st = enqueue_plain(c, sh, x0, U_nom, obs, n_obs, path, n_pts, ds, 0, 0, dU, dT, nullptr, nullptr, nullptr, s);
      if (st != BRMPPI_OK) continue;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r)
        enqueue_plain(c, sh, x0, U_nom, obs, n_obs, path, n_pts, ds, 0, r, dU, dT, nullptr, nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  if (best.tps == 0) return fail(c, BRMPPI_EINVAL, "no launch shape could run");
  c->err.clear();
  c->tuned[n_obs] = best;
  return BRMPPI_OK;
}

brmppi_status brmppi_autotune_batch(brmppi_ctx* c, const brmppi_instance* inst, int32_t n, int32_t reps,
                                    void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (reps < 1) reps = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  Lane& L = c->batch;
  if (L.pending && (e = cudaEventSynchronize(L.batch_done)) != cudaSuccess) return cuda_fail(c, e, "sync");
  L.pending = false;
  int max_P = philox_blocks(rows_of(c->prm, c->prm.max_obstacles));
  for (int i = 0; inst && i < n; ++i) max_P = std::max(max_P, philox_blocks(rows_of(c->prm, inst[i].n_obs)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Shape best;
  float best_ms = 1e30f;
  std::string last_err;
  for (int tps : {1, 2, 4, 8}) {
    int bpt;
    if (!pick_bpt(tps, max_P, &bpt)) continue;
    for (int threads : {64, 128, 256}) {
      if (threads / tps < kMinBatchSpb) continue;
      Shape sh;
      sh.tps = tps;
      sh.bpt = bpt;
      sh.threads = threads;
      BatchPlan plan;
      if (plan_batch(c, L, inst, n, &sh, L.h_inst, L.h_work, &plan) != BRMPPI_OK) {
        last_err = c->err;
        continue;
      }
      if (upload_and_launch(c, L, plan, L.h_inst, L.h_work, s) != BRMPPI_OK) {
        last_err = c->err;
        continue;
      }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) launch_batch(c, L, plan, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  if (best.tps == 0) return fail(c, BRMPPI_EINVAL, "no batch launch shape could run: " + last_err);
  c->err.clear();
  c->batch_tuned = true;
  c->batch_shape = best;
  return BRMPPI_OK;
}

brmppi_status brmppi_get_batch_launch(brmppi_ctx* c, int32_t* tps, int32_t* threads) {
  if (!c) return BRMPPI_EINVAL;
  Shape sh;
  if (!batch_shape_default(c, philox_blocks(rows_of(c->prm, c->prm.max_obstacles)), &sh))
    return fail(c, BRMPPI_EINVAL, "no batch launch shape");
  if (tps) *tps = sh.tps;
  if (threads) *threads = sh.threads;
  return BRMPPI_OK;
}

brmppi_status brmppi_get_launch(brmppi_ctx* c, int32_t n_obs, int32_t* tps, int32_t* threads, int32_t* blocks) {
  if (!c) return BRMPPI_EINVAL;
  if (n_obs < 0 || n_obs > c->prm.max_obstacles) return fail(c, BRMPPI_EINVAL, "n_obs out of range");
  Shape sh;
  if (!plain_shape(c, n_obs, c->prm.max_path_pts, &sh)) return fail(c, BRMPPI_EINVAL, "no launch shape");
  const int spb = sh.threads / sh.tps;
  if (tps) *tps = sh.tps;
  if (threads) *threads = sh.threads;
  if (blocks) *blocks = (c->prm.S + spb - 1) / spb;
  return BRMPPI_OK;
}

brmppi_status brmppi_hitch_stabilize_device(brmppi_ctx* c, const double* x_dev, const float* u_ref_dev, int32_t n,
                                            float* u_out_dev, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (n < 0) return fail(c, BRMPPI_EINVAL, "n must be >= 0");
  if (n == 0) return BRMPPI_OK;
  if (!x_dev || !u_ref_dev || !u_out_dev) return fail(c, BRMPPI_EINVAL, "NULL buffer");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  e = brmppi::launch_stabilize(make_kconst(c->prm), x_dev, u_ref_dev, n, u_out_dev, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "stabilizer launch");
  return BRMPPI_OK;
}

brmppi_status brmppi_noise_blocks(uint64_t seed, uint64_t counter, int32_t n_samples, int32_t H, int32_t n_blocks,
                                  uint32_t* words_dev, float* normals_dev, void* stream) {
  if (n_samples < 0 || H < 0 || n_blocks < 0) return fail(nullptr, BRMPPI_EINVAL, "negative size");
  if (static_cast<long long>(n_samples) * H * n_blocks > (1LL << 31))
    return fail(nullptr, BRMPPI_EINVAL, "more than 2^31 blocks");
  if (n_blocks > (1 << 16) || H > (1 << 16)) return fail(nullptr, BRMPPI_EINVAL, "H or n_blocks above 2^16");
  if ((words_dev && (reinterpret_cast<uintptr_t>(words_dev) & 15)) ||
      (normals_dev && (reinterpret_cast<uintptr_t>(normals_dev) & 15)))
    return fail(nullptr, BRMPPI_EINVAL, "outputs must be 16-byte aligned");
  const cudaError_t e =
      brmppi::launch_noise_blocks(seed, counter, n_samples, H, n_blocks, words_dev, normals_dev,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "noise-table launch");
  return BRMPPI_OK;
}

brmppi_status brmppi_transfer_bytes(brmppi_ctx* c, int32_t n_obs, int32_t n_pts, uint64_t* h2d, uint64_t* d2h) {
  if (!c) return BRMPPI_EINVAL;
  brmppi_status st = check_sizes(c, n_obs, n_pts, 1.0f);
  if (st != BRMPPI_OK) return st;
  if (h2d) *h2d = c->off_path + sizeof(float) * 3 * static_cast<size_t>(n_pts);
  if (d2h) *d2h = sizeof(float) * c->out_floats;
  return BRMPPI_OK;
}

}  // extern "C"
