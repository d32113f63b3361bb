// api.cu -- the C ABI of libbrmppi.so (see include/brmppi.h).
//
// The context owns every buffer a solve needs, sized at create time for
// the declared capacities, so the solve paths allocate nothing.  Host entry
// points stage inputs through one pinned buffer (one H2D copy), run the
// kernel and read the outputs back (one D2H copy, plus the costs when
// asked for).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "brmppi.h"
#include "launch.h"

struct brmppi_ctx {
  brmppi_params prm{};
  int device = 0;
  cudaStream_t stream = nullptr;
  // device
  unsigned char* d_in = nullptr;  // x0 | U_nom | obs | path
  float* d_out = nullptr;         // U | traj | status
  float* d_J = nullptr;
  float* d_part = nullptr;
  unsigned int* d_sync = nullptr;  // ticket, err
  // pinned host
  unsigned char* h_in = nullptr;
  float* h_out = nullptr;
  // layout
  size_t off_unom = 0, off_obs = 0, off_path = 0, in_bytes = 0;
  size_t out_floats = 0;
  size_t part_stride = 0, part_blocks = 0;
  size_t smem_limit = 0;
  std::string err;
};

namespace {

std::mutex g_err_mu;
std::string g_create_err;

constexpr int kMaxObstacles = 124;  // ceil((4 + n)/4) <= 32 Philox blocks
constexpr int kMaxPathPts = 12000;
constexpr int kMaxH = 1024;
constexpr int kMinThreads = 64;
constexpr int kMaxThreads = 512;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

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

bool is_pow2_tps(int t) { return t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32; }

int philox_blocks(int n_obs) { return (4 + n_obs + 3) / 4; }  // d = 3 + (1 + n_obs)

std::string check_params(const brmppi_params* p) {
  if (!p) return "params is NULL";
  if (p->abi_version != BRMPPI_ABI_VERSION) return "abi_version mismatch";
  if (p->S < 1) return "S must be >= 1";
  if (p->H < 1 || p->H > kMaxH) return "H must be in [1, 1024]";
  if (p->max_obstacles < 0 || p->max_obstacles > kMaxObstacles) return "max_obstacles must be in [0, 124]";
  if (p->max_path_pts < 2 || p->max_path_pts > kMaxPathPts) return "max_path_pts must be in [2, 12000]";
  if (p->flags & ~static_cast<int32_t>(BRMPPI_FLAG_PROJ_NONE)) return "unknown flag";
  if (p->threads_per_sample != 0 && !is_pow2_tps(p->threads_per_sample))
    return "threads_per_sample must be 0, 1, 2, 4, 8, 16 or 32";
  if (p->block_threads != 0 &&
      (p->block_threads < kMinThreads || p->block_threads > kMaxThreads || p->block_threads % 32 != 0))
    return "block_threads must be 0 or a multiple of 32 in [64, 512]";
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
  return "";
}

struct Launch {
  int tps, bpt, threads, blocks;
  size_t smem;
};

// Launch shape for a solve with n_obs obstacles: a team just wide enough
// for the Philox blocks (one block per lane), blocks of 128 threads, halved
// while that leaves fewer than two blocks per SM; narrower blocks (then
// wider teams) while the shared-memory tables do not fit.
bool pick_bpt(int tps, int P, int* bpt) {
  for (int b : {1, 2, 4})
    if (tps * b >= P && brmppi::variant_exists(tps, b)) {
      *bpt = b;
      return true;
    }
  return false;
}

bool choose_launch(const brmppi_ctx* c, int n_obs, int n_pts, Launch* L) {
  const int P = philox_blocks(n_obs);
  const bool fixed_tps = c->prm.threads_per_sample != 0;
  int tps = c->prm.threads_per_sample;
  if (!fixed_tps) {
    tps = 1;
    while (tps < P && tps < 32) tps <<= 1;
  }
  int bpt = 0;
  if (!pick_bpt(tps, P, &bpt)) return false;
  int threads = c->prm.block_threads;
  const bool fixed_threads = threads != 0;
  const int S = c->prm.S;
  if (!fixed_threads) {
    threads = 128;
    while (threads > kMinThreads) {
      const int spb = threads / tps;
      const int blocks = (S + spb - 1) / spb;
      if (blocks >= 2 * 152) break;
      threads >>= 1;
    }
  }
  if (threads < tps) return false;
  for (;;) {
    const size_t smem = brmppi::smem_bytes(n_obs, n_pts, c->prm.H, threads / tps);
    if (smem <= c->smem_limit) break;
    if (!fixed_threads && threads > kMinThreads) {
      threads -= 32;
    } else if (!fixed_tps && tps < 32) {
      tps <<= 1;
      if (!pick_bpt(tps, P, &bpt)) return false;
    } else {
      return false;
    }
  }
  const int spb = threads / tps;
  L->tps = tps;
  L->bpt = bpt;
  L->threads = threads;
  L->blocks = (S + spb - 1) / spb;
  L->smem = brmppi::smem_bytes(n_obs, n_pts, c->prm.H, spb);
  return true;
}

brmppi::KParams make_kparams(const brmppi_params& q, int n_obs, int n_pts, float ds, uint64_t seed,
                             uint64_t counter, int part_stride) {
  brmppi::KParams k{};
  k.S = q.S;
  k.H = q.H;
  k.n_obs = n_obs;
  k.n_pts = n_pts;
  k.Nc = 1 + n_obs;
  k.P = philox_blocks(n_obs);
  k.proj = (q.flags & BRMPPI_FLAG_PROJ_NONE) ? 0 : 1;
  k.Ts = q.Ts;
  k.hTs2 = 0.5f * q.Ts * q.Ts;
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
  k.w_a = q.w_alpha;
  k.pc_a = 0.5f * q.rho * (q.ua_hi + q.ua_lo);
  k.m_a = q.w_alpha + q.rho;
  k.inv_m_a = 1.0f / (q.w_alpha + q.rho);
  k.h_floor = q.h_floor;
  k.ds = ds;
  k.inv_ds = 1.0f / ds;
  k.key0 = static_cast<uint32_t>(seed);
  k.key1 = static_cast<uint32_t>(seed >> 32);
  k.ctr = static_cast<uint32_t>(counter);
  k.part_stride = part_stride;
  return k;
}

brmppi_status check_sizes(brmppi_ctx* c, int32_t n_obs, int32_t n_pts, float ds) {
  if (n_obs < 0 || n_obs > c->prm.max_obstacles) return fail(c, BRMPPI_EINVAL, "n_obs out of [0, max_obstacles]");
  if (n_pts < 2 || n_pts > c->prm.max_path_pts) return fail(c, BRMPPI_EINVAL, "n_pts out of [2, max_path_pts]");
  if (!(ds > 0.f) || !std::isfinite(ds)) return fail(c, BRMPPI_EINVAL, "ds must be positive and finite");
  return BRMPPI_OK;
}

brmppi_status enqueue(brmppi_ctx* c, const double* x0, const float* U_nom, const float* obs, int32_t n_obs,
                      const float* path, int32_t n_pts, float ds, uint64_t seed, uint64_t counter,
                      float* U_out, float* traj_out, float* J_out, float* U_next, int32_t* status,
                      cudaStream_t stream) {
  Launch L;
  if (!choose_launch(c, n_obs, n_pts, &L)) return fail(c, BRMPPI_EINVAL, "no kernel variant for this size");
  if (L.smem > c->smem_limit) return fail(c, BRMPPI_EINVAL, "shared memory need exceeds the context's limit");
  if (static_cast<size_t>(L.blocks) > c->part_blocks) return fail(c, BRMPPI_EINVAL, "too many blocks");
  const brmppi::KParams kp =
      make_kparams(c->prm, n_obs, n_pts, ds, seed, counter, static_cast<int>(c->part_stride));
  brmppi::KIO io{};
  io.x0 = x0;
  io.U_nom = U_nom;
  io.obs = obs;
  io.path = path;
  io.U_out = U_out;
  io.traj_out = traj_out;
  io.J_out = J_out;
  io.U_next = U_next;
  io.status = status;
  io.part = c->d_part;
  io.ticket = c->d_sync;
  io.err = c->d_sync + 1;
  cudaError_t e = brmppi::launch_rollout(L.tps, L.bpt, L.blocks, L.threads, L.smem, stream, kp, io);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return BRMPPI_OK;
}

}  // namespace

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
  cudaError_t e = cudaSetDevice(device);
  auto bail = [&](cudaError_t err, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(err);
    brmppi_destroy(c);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? BRMPPI_ENOMEM : BRMPPI_ECUDA, m);
  };
  if (e != cudaSuccess) return bail(e, "cudaSetDevice");
  const int H = p->H, S = p->S;
  c->off_unom = 64;
  c->off_obs = align_up(c->off_unom + sizeof(float) * 3 * H, 16);
  c->off_path = align_up(c->off_obs + sizeof(float) * 6 * static_cast<size_t>(p->max_obstacles), 16);
  c->in_bytes = align_up(c->off_path + sizeof(float) * 3 * static_cast<size_t>(p->max_path_pts), 16);
  c->out_floats = 3 * static_cast<size_t>(H) + 7 * static_cast<size_t>(H + 1) + 1;
  c->part_stride = align_up(3 + 3 * static_cast<size_t>(H) + 1, 4);
  c->part_blocks = static_cast<size_t>((S + 1) / 2);  // at least two samples per block
  if (c->part_blocks < 1) c->part_blocks = 1;
  int dev_smem = 0;
  if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess)
    return bail(e, "cudaDeviceGetAttribute");
  c->smem_limit = static_cast<size_t>(dev_smem) - 2048;  // static shared memory of the kernel
  if ((e = brmppi::set_smem_limit(c->smem_limit)) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  {
    Launch L;
    if (!choose_launch(c, p->max_obstacles, p->max_path_pts, &L)) {
      brmppi_destroy(c);
      return fail(nullptr, BRMPPI_EINVAL, "no launch shape fits these capacities in shared memory");
    }
  }
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "cudaStreamCreate");
  if ((e = cudaMalloc(&c->d_in, c->in_bytes)) != cudaSuccess) return bail(e, "cudaMalloc(in)");
  if ((e = cudaMalloc(&c->d_out, sizeof(float) * c->out_floats)) != cudaSuccess) return bail(e, "cudaMalloc(out)");
  if ((e = cudaMalloc(&c->d_J, sizeof(float) * S)) != cudaSuccess) return bail(e, "cudaMalloc(J)");
  if ((e = cudaMalloc(&c->d_part, sizeof(float) * c->part_stride * c->part_blocks)) != cudaSuccess)
    return bail(e, "cudaMalloc(partials)");
  if ((e = cudaMalloc(&c->d_sync, sizeof(unsigned int) * 4)) != cudaSuccess) return bail(e, "cudaMalloc(sync)");
  if ((e = cudaMemset(c->d_sync, 0, sizeof(unsigned int) * 4)) != cudaSuccess) return bail(e, "cudaMemset");
  if ((e = cudaMallocHost(&c->h_in, c->in_bytes)) != cudaSuccess) return bail(e, "cudaMallocHost(in)");
  if ((e = cudaMallocHost(&c->h_out, sizeof(float) * c->out_floats)) != cudaSuccess)
    return bail(e, "cudaMallocHost(out)");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "cudaDeviceSynchronize");
  *out = c;
  return BRMPPI_OK;
}

void brmppi_destroy(brmppi_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->d_in);
  cudaFree(c->d_out);
  cudaFree(c->d_J);
  cudaFree(c->d_part);
  cudaFree(c->d_sync);
  cudaFreeHost(c->h_in);
  cudaFreeHost(c->h_out);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

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
  for (int j = 0; j < 7; ++j)
    if (!std::isfinite(x0[j])) return fail(c, BRMPPI_ENONFINITE, "x0 is not finite");
  for (int o = 0; o < n_obs; ++o)
    if (obs[6 * o + 5] != 2.0f) return fail(c, BRMPPI_EINVAL, "obstacle exponent must be 2");
  const int H = c->prm.H;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  // stage: x0 | U_nom | obs | path  (one pinned buffer, one copy)
  std::memcpy(c->h_in, x0, 7 * sizeof(double));
  std::memcpy(c->h_in + c->off_unom, U_nom, sizeof(float) * 3 * H);
  if (n_obs > 0) std::memcpy(c->h_in + c->off_obs, obs, sizeof(float) * 6 * n_obs);
  std::memcpy(c->h_in + c->off_path, path, sizeof(float) * 3 * n_pts);
  const size_t in_used = c->off_path + sizeof(float) * 3 * n_pts;
  if ((e = cudaMemcpyAsync(c->d_in, c->h_in, in_used, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "H2D copy");
  float* dU = c->d_out;
  float* dT = dU + 3 * H;
  int32_t* dS = reinterpret_cast<int32_t*>(dT + 7 * (H + 1));
  st = enqueue(c, reinterpret_cast<const double*>(c->d_in), reinterpret_cast<const float*>(c->d_in + c->off_unom),
               reinterpret_cast<const float*>(c->d_in + c->off_obs), n_obs,
               reinterpret_cast<const float*>(c->d_in + c->off_path), n_pts, ds, seed, counter, dU, dT,
               J_out ? c->d_J : nullptr, nullptr, dS, c->stream);
  if (st != BRMPPI_OK) return st;
  if ((e = cudaMemcpyAsync(c->h_out, c->d_out, sizeof(float) * c->out_floats, cudaMemcpyDeviceToHost,
                           c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "D2H copy");
  if (J_out && (e = cudaMemcpyAsync(J_out, c->d_J, sizeof(float) * c->prm.S, cudaMemcpyDeviceToHost,
                                    c->stream)) != cudaSuccess)
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
                                  float* traj_out_dev, float* J_out_dev, float* U_next_dev,
                                  int32_t* status_dev, void* stream) {
  if (!c) return BRMPPI_EINVAL;
  c->err.clear();
  if (!x0_dev || !U_nom_dev || !path_dev || !U_out_dev || (n_obs > 0 && !obs_dev))
    return fail(c, BRMPPI_EINVAL, "NULL buffer");
  brmppi_status st = check_sizes(c, n_obs, n_pts, ds);
  if (st != BRMPPI_OK) return st;
  return enqueue(c, x0_dev, U_nom_dev, obs_dev, n_obs, path_dev, n_pts, ds, seed, counter, U_out_dev,
                 traj_out_dev, J_out_dev, U_next_dev, status_dev, static_cast<cudaStream_t>(stream));
}

brmppi_status brmppi_get_launch(brmppi_ctx* c, int32_t n_obs, int32_t* tps, int32_t* threads, int32_t* blocks) {
  if (!c) return BRMPPI_EINVAL;
  if (n_obs < 0 || n_obs > c->prm.max_obstacles) return fail(c, BRMPPI_EINVAL, "n_obs out of range");
  Launch L;
  if (!choose_launch(c, n_obs, c->prm.max_path_pts, &L)) return fail(c, BRMPPI_EINVAL, "no variant");
  if (tps) *tps = L.tps;
  if (threads) *threads = L.threads;
  if (blocks) *blocks = L.blocks;
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
