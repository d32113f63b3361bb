// serve.cu -- continuous-batching serving loop of libbrmppi.so.
//
// Requests (vehicle, state, obstacles) enter a pinned request slot and a
// FIFO queue.  A scheduler thread forms a batch whenever a lane is free:
// queued requests in order, one per vehicle (a vehicle's next request waits
// for its previous solve, whose warm start it needs), up to the lane's
// capacity; it copies their inputs to the device, launches one persistent
// solve over them on the lane's stream and queues the read-back of their
// outputs.  With several lanes, batches admitted while others still run
// overlap on the device.  A completion thread waits for each batch's event
// and publishes its results; brmppi_poll hands them out.
//
// Per vehicle the path, the nominal sequence and the noise counter stay
// resident: each solve writes its warm start (U* shifted by one step) over
// the vehicle's nominal sequence in place, and the counter advances by one
// per solve in submission order.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "internal.h"

namespace brmppi_host {

brmppi::KConst make_kconst(const brmppi_params& q);  // api.cu

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum SlotState { kFree = 0, kQueued, kRunning, kDone };

struct Vehicle {
  bool registered = false;
  float* d_path = nullptr;  // max_path_pts * 3
  float* d_unom = nullptr;  // 3H, overwritten by each solve's warm start
  int n_pts = 0;
  float ds = 0.f;
  uint64_t seed = 0, counter = 0;
  int queued = 0;       // requests submitted and not yet finished
  bool running = false;  // a solve of this vehicle is on the device
};

struct Slot {
  SlotState state = kFree;
  uint64_t ticket = 0;
  uint32_t vid = 0;
  int n_obs = 0;
  double t_submit = 0.0, t_done = 0.0;
  int32_t status = 0;
  bool held = false;    // its batch's wait gave up: the GPU may still use the slot
  bool polled = false;  // handed out while held: free it when the batch finishes
};

struct InFlight {
  int lane;
  std::vector<int> slots;
};

}  // namespace

struct Server {
  brmppi_ctx shadow;  // parameters and limits for planning; its own error string
  int H = 0, S = 0, max_obs = 0;
  // request slots: device inputs / outputs and pinned mirrors
  int n_slots = 0;
  size_t in_stride = 0;    // bytes: x0 (64) | obstacles
  size_t out_stride = 0;   // floats: U (3H) | traj (7(H+1)) | status
  unsigned char* d_in = nullptr;
  unsigned char* h_in = nullptr;
  float* d_out = nullptr;
  float* h_out = nullptr;
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  std::unordered_map<uint64_t, int> by_ticket;
  uint64_t next_ticket = 1;
  std::deque<int> queue;
  std::vector<Vehicle> veh;
  std::vector<Lane> lanes;
  std::vector<bool> lane_busy;
  std::deque<InFlight> inflight;
  // batches whose bounded wait gave up (their requests answered ETIMEDOUT):
  // their lane, vehicles and request slots stay reserved until they finish
  std::deque<InFlight> stuck;
  int wait_ms = 10000;
  Shape shape;
  int max_batch = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_comp;
  bool stop = false;
  std::thread sched, comp;
  uint64_t submitted = 0, completed = 0, batches = 0, solves = 0;
  int running_batches = 0, max_running = 0;

  void scheduler_loop();
  void completion_loop();
  void release(const InFlight& f);  // a stuck batch finished (mu held)
  void reap_stuck();                // release the stuck batches that have finished (mu held)
};

void Server::release(const InFlight& f) {
  for (int s : f.slots) {
    Slot& sl = slots[s];
    veh[sl.vid].running = false;
    sl.held = false;
    if (sl.polled) {
      sl.polled = false;
      sl.state = kFree;
      free_slots.push_back(s);
    }
  }
  lane_busy[f.lane] = false;
  lanes[f.lane].pending = false;
  --running_batches;
  cv_sched.notify_one();
}

void Server::reap_stuck() {
  for (auto it = stuck.begin(); it != stuck.end();) {
    if (cudaEventQuery(lanes[it->lane].batch_done) != cudaErrorNotReady) {
      release(*it);
      it = stuck.erase(it);
    } else {
      ++it;
    }
  }
}

void Server::scheduler_loop() {
  cudaSetDevice(shadow.device);
  std::vector<brmppi_instance> inst;
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    int lane = -1;
    for (size_t i = 0; i < lanes.size(); ++i)
      if (!lane_busy[i]) {
        lane = static_cast<int>(i);
        break;
      }
    std::vector<int> pick;
    if (lane >= 0 && !queue.empty()) {
      std::unordered_set<uint32_t> used;
      for (auto it = queue.begin(); it != queue.end() && static_cast<int>(pick.size()) < max_batch;) {
        const uint32_t v = slots[*it].vid;
        if (veh[v].running || used.count(v)) {
          ++it;  // this vehicle's earlier solve comes first
          continue;
        }
        used.insert(v);
        pick.push_back(*it);
        it = queue.erase(it);
      }
    }
    if (pick.empty()) {
      cv_sched.wait(lk);
      continue;
    }
    lane_busy[lane] = true;
    ++running_batches;
    if (running_batches > max_running) max_running = running_batches;
    inst.assign(pick.size(), brmppi_instance{});
    for (size_t j = 0; j < pick.size(); ++j) {
      Slot& sl = slots[pick[j]];
      Vehicle& V = veh[sl.vid];
      V.running = true;
      sl.state = kRunning;
      unsigned char* din = d_in + static_cast<size_t>(pick[j]) * in_stride;
      float* dout = d_out + static_cast<size_t>(pick[j]) * out_stride;
      brmppi_instance& q = inst[j];
      q.x0 = reinterpret_cast<const double*>(din);
      q.obs = reinterpret_cast<const float*>(din + 64);
      q.n_obs = sl.n_obs;
      q.U_nom = V.d_unom;
      q.path = V.d_path;
      q.n_pts = V.n_pts;
      q.ds = V.ds;
      q.S = S;
      q.H = H;
      q.seed = V.seed;
      q.counter = V.counter++;
      q.U_out = dout;
      q.traj_out = dout + 3 * H;
      q.J_out = nullptr;
      q.U_next = V.d_unom;  // warm start in place (read by every tile before the merge writes it)
      q.status = reinterpret_cast<int32_t*>(dout + 3 * H + 7 * (H + 1));
    }
    lk.unlock();

    Lane& L = lanes[lane];
    brmppi_status st = BRMPPI_OK;
    cudaError_t e = cudaSuccess;
    const size_t in_bytes = 64 + sizeof(float) * obs_floats(shadow.prm) * static_cast<size_t>(max_obs);
    for (int s : pick) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_in + static_cast<size_t>(s) * in_stride, h_in + static_cast<size_t>(s) * in_stride,
                            in_bytes, cudaMemcpyHostToDevice, L.stream);
    }
    BatchPlan plan;
    if (e == cudaSuccess) st = plan_batch(&shadow, L, inst.data(), static_cast<int32_t>(inst.size()), &shape,
                                          L.h_inst, L.h_work, &plan);
    if (e == cudaSuccess && st == BRMPPI_OK) st = upload_and_launch(&shadow, L, plan, L.h_inst, L.h_work, L.stream);
    for (int s : pick) {
      if (e == cudaSuccess && st == BRMPPI_OK)
        e = cudaMemcpyAsync(h_out + static_cast<size_t>(s) * out_stride, d_out + static_cast<size_t>(s) * out_stride,
                            sizeof(float) * out_stride, cudaMemcpyDeviceToHost, L.stream);
    }
    if (e == cudaSuccess && st == BRMPPI_OK) e = cudaEventRecord(L.batch_done, L.stream);
    L.pending = true;

    lk.lock();
    if (e != cudaSuccess || st != BRMPPI_OK) {
      // the batch never ran: fail its requests, free the lane
      const double t = now_s();
      for (int s : pick) {
        Slot& sl = slots[s];
        sl.state = kDone;
        sl.t_done = t;
        sl.status = (e != cudaSuccess) ? BRMPPI_ECUDA : st;
        veh[sl.vid].running = false;
        veh[sl.vid].queued -= 1;
        ++completed;
      }
      lane_busy[lane] = false;
      --running_batches;
      L.pending = false;
      continue;
    }
    ++batches;
    solves += pick.size();
    inflight.push_back(InFlight{lane, std::move(pick)});
    cv_comp.notify_one();
  }
}

void Server::completion_loop() {
  cudaSetDevice(shadow.device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    reap_stuck();
    while (inflight.empty() && !stop) {
      if (stuck.empty()) {
        cv_comp.wait(lk);
      } else {
        cv_comp.wait_for(lk, std::chrono::milliseconds(1));
        reap_stuck();
      }
    }
    if (inflight.empty() && stop) return;
    const int lane = inflight.front().lane;
    lk.unlock();
    const cudaError_t e = wait_event(lanes[lane].batch_done, wait_ms);
    const double t = now_s();
    lk.lock();
    InFlight f = std::move(inflight.front());
    inflight.pop_front();
    const bool timed_out = e == cudaErrorNotReady;
    for (int s : f.slots) {
      Slot& sl = slots[s];
      int32_t kst = timed_out ? BRMPPI_ETIMEDOUT : BRMPPI_ECUDA;
      if (e == cudaSuccess) std::memcpy(&kst, h_out + static_cast<size_t>(s) * out_stride + 3 * H + 7 * (H + 1), 4);
      sl.status = kst;
      sl.t_done = t;
      sl.state = kDone;
      sl.held = timed_out;
      if (!timed_out) veh[sl.vid].running = false;
      veh[sl.vid].queued -= 1;
      ++completed;
    }
    if (timed_out) {
      stuck.push_back(std::move(f));  // the lane stays busy until the batch finishes
      continue;
    }
    lane_busy[f.lane] = false;
    --running_batches;
    cv_sched.notify_one();
  }
}

brmppi_status server_create(brmppi_ctx* c) {
  const brmppi_params& p = c->prm;
  Server* sv = new (std::nothrow) Server();
  if (!sv) return fail(c, BRMPPI_ENOMEM, "host allocation failed");
  sv->shadow.prm = p;
  sv->shadow.device = c->device;
  sv->shadow.num_sms = c->num_sms;
  sv->shadow.smem_limit = c->smem_limit;
  sv->H = p.H;
  sv->S = p.S;
  sv->max_obs = p.max_obstacles;
  sv->max_batch = p.serve_max_batch > 0 ? p.serve_max_batch : 64;
  sv->wait_ms = wait_limit_ms(p);
  // the launch shape of every serving batch, fixed here so that a solve's
  // bits do not depend on what else is in its batch: the context's batch
  // shape parameters when given, else one lane per sample (teams just wide
  // enough for two Philox blocks a lane when rows carry a steer-rate column)
  // in 128-thread blocks
  const int P_cap = philox_blocks(rows_of(p, p.max_obstacles));
  sv->shape.tps = p.batch_threads_per_sample != 0
                      ? p.batch_threads_per_sample
                      : (brmppi::needs_ext(make_kconst(p)) ? ext_team_width(P_cap) : 1);
  sv->shape.threads =
      p.batch_block_threads != 0 ? p.batch_block_threads : std::max(128, kMinBatchSpb * sv->shape.tps);
  if (!pick_bpt(sv->shape.tps, P_cap, &sv->shape.bpt) || sv->shape.threads / sv->shape.tps < kMinBatchSpb) {
    c->server = sv;
    return fail(c, BRMPPI_EINVAL, "no serving launch shape for the batch shape parameters");
  }
  const int n_lanes = p.serve_lanes > 0 ? p.serve_lanes : 2;
  sv->in_stride = align_up(64 + sizeof(float) * obs_floats(p) * static_cast<size_t>(p.max_obstacles), 256);
  sv->out_stride = align_up(3 * static_cast<size_t>(p.H) + 7 * static_cast<size_t>(p.H + 1) + 1, 64);
  c->server = sv;
  cudaError_t e;
  // lanes first (the large buffers), then as many request slots as the
  // remaining device memory comfortably holds, capped by serve_queue
  sv->lanes.resize(n_lanes);
  sv->lane_busy.assign(n_lanes, false);
  for (Lane& L : sv->lanes) {
    if ((e = lane_alloc(L, sv->max_batch, p.S, p.H, c->num_sms, c->part_stride)) != cudaSuccess)
      return cuda_fail(c, e, "serving lane buffers");
    if ((e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(c, e, "serving lane stream");
  }
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda_fail(c, e, "cudaMemGetInfo");
  const size_t slot_bytes = sv->in_stride + sizeof(float) * sv->out_stride;
  const size_t want = p.serve_queue > 0 ? static_cast<size_t>(p.serve_queue) : 1024;
  const size_t fit = (free_b / 4) / slot_bytes;
  sv->n_slots = static_cast<int>(want < fit ? want : fit);
  if (sv->n_slots < 1) return fail(c, BRMPPI_ENOMEM, "no device memory for request slots");
  const size_t ns = static_cast<size_t>(sv->n_slots);
  if ((e = dev_alloc(&sv->d_in, sv->in_stride * ns)) != cudaSuccess) return cuda_fail(c, e, "request slots");
  if ((e = dev_alloc(&sv->d_out, sizeof(float) * sv->out_stride * ns)) != cudaSuccess)
    return cuda_fail(c, e, "request slots");
  if ((e = host_alloc(&sv->h_in, sv->in_stride * ns)) != cudaSuccess) return cuda_fail(c, e, "request slots");
  if ((e = host_alloc(&sv->h_out, sizeof(float) * sv->out_stride * ns)) != cudaSuccess)
    return cuda_fail(c, e, "request slots");
  sv->slots.resize(ns);
  sv->free_slots.reserve(ns);
  for (int i = sv->n_slots - 1; i >= 0; --i) sv->free_slots.push_back(i);
  sv->veh.resize(static_cast<size_t>(p.max_vehicles));
  sv->sched = std::thread([sv] { sv->scheduler_loop(); });
  sv->comp = std::thread([sv] { sv->completion_loop(); });
  return BRMPPI_OK;
}

bool server_destroy(brmppi_ctx* c) {
  Server* sv = c->server;
  if (!sv) return true;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_sched.notify_all();
  sv->cv_comp.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  if (sv->comp.joinable()) sv->comp.join();
  // every lane's last batch, within the limit; a lane still running keeps its
  // buffers, and then nothing else is freed either (a free may wait for the
  // device)
  bool done = true;
  for (Lane& L : sv->lanes)
    if (L.stream && wait_stream(L.stream, sv->wait_ms) != cudaSuccess) done = false;
  if (done) {
    for (Lane& L : sv->lanes) lane_free(L, sv->wait_ms);
    for (Vehicle& V : sv->veh) {
      cudaFree(V.d_path);
      cudaFree(V.d_unom);
    }
    cudaFree(sv->d_in);
    cudaFree(sv->d_out);
    cudaFreeHost(sv->h_in);
    cudaFreeHost(sv->h_out);
  } else {
    for (Lane& L : sv->lanes)
      if (L.stream) cudaStreamDestroy(L.stream);  // released once its work is done
  }
  delete sv;
  c->server = nullptr;
  return done;
}

}  // namespace brmppi_host

using namespace brmppi_host;

extern "C" {

brmppi_status brmppi_vehicle_register(brmppi_ctx* c, uint32_t vid, const float* path, int32_t n_pts, float ds,
                                      const float* U_init, uint64_t seed) {
  if (!c) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv) return fail(c, BRMPPI_EINVAL, "context created without a serving loop (max_vehicles)");
  if (vid >= sv->veh.size()) return fail(c, BRMPPI_EINVAL, "vehicle id out of [0, max_vehicles)");
  if (!path) return fail(c, BRMPPI_EINVAL, "NULL path");
  if (n_pts < 2 || n_pts > c->prm.max_path_pts) return fail(c, BRMPPI_EINVAL, "n_pts out of [2, max_path_pts]");
  if (!(ds > 0.f) || !std::isfinite(ds)) return fail(c, BRMPPI_EINVAL, "ds must be positive and finite");
  if (!path_turns_ok(path, n_pts)) return fail(c, BRMPPI_EINVAL, "path headings of consecutive rows differ by more than pi/4");
  std::lock_guard<std::mutex> lk(sv->mu);
  Vehicle& V = sv->veh[vid];
  if (V.queued > 0 || V.running) return fail(c, BRMPPI_EBUSY, "vehicle has requests in flight");
  cudaError_t e;
  cudaSetDevice(c->device);
  if (!V.d_path && (e = dev_alloc(&V.d_path, sizeof(float) * 3 * static_cast<size_t>(c->prm.max_path_pts))) != cudaSuccess)
    return cuda_fail(c, e, "vehicle path");
  if (!V.d_unom && (e = dev_alloc(&V.d_unom, sizeof(float) * 3 * static_cast<size_t>(sv->H))) != cudaSuccess)
    return cuda_fail(c, e, "vehicle nominal");
  if ((e = cudaMemcpy(V.d_path, path, sizeof(float) * 3 * n_pts, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "vehicle path upload");
  if (U_init) {
    e = cudaMemcpy(V.d_unom, U_init, sizeof(float) * 3 * sv->H, cudaMemcpyHostToDevice);
  } else {
    e = cudaMemset(V.d_unom, 0, sizeof(float) * 3 * sv->H);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "vehicle nominal upload");
  V.n_pts = n_pts;
  V.ds = ds;
  V.seed = seed;
  V.counter = 0;
  V.registered = true;
  return BRMPPI_OK;
}

brmppi_status brmppi_submit(brmppi_ctx* c, uint32_t vid, const double x0[7], const float* obs, int32_t n_obs,
                            uint64_t* ticket) {
  if (!c || !ticket) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv) return BRMPPI_EINVAL;
  if (!x0 || (n_obs > 0 && !obs) || n_obs < 0 || n_obs > sv->max_obs) return BRMPPI_EINVAL;
  for (int j = 0; j < state_dim(c->prm); ++j)
    if (!std::isfinite(x0[j])) return BRMPPI_ENONFINITE;
  for (int o = 0; o < n_obs; ++o)
    if (!exponent_ok(c->prm, obs[obs_floats(c->prm) * o + 5])) return BRMPPI_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (vid >= sv->veh.size() || !sv->veh[vid].registered) return BRMPPI_EINVAL;
    if (sv->free_slots.empty()) return BRMPPI_EBUSY;
    const int s = sv->free_slots.back();
    sv->free_slots.pop_back();
    unsigned char* h = sv->h_in + static_cast<size_t>(s) * sv->in_stride;
    std::memcpy(h, x0, state_dim(c->prm) * sizeof(double));  // 64 bytes reserved
    if (n_obs > 0) std::memcpy(h + 64, obs, sizeof(float) * obs_floats(c->prm) * n_obs);
    Slot& sl = sv->slots[s];
    sl.state = kQueued;
    sl.ticket = sv->next_ticket++;
    sl.vid = vid;
    sl.n_obs = n_obs;
    sl.t_submit = now_s();
    sl.status = 0;
    sv->by_ticket[sl.ticket] = s;
    sv->veh[vid].queued += 1;
    sv->queue.push_back(s);
    ++sv->submitted;
    *ticket = sl.ticket;
  }
  sv->cv_sched.notify_one();
  return BRMPPI_OK;
}

brmppi_status brmppi_poll(brmppi_ctx* c, uint64_t ticket, float* U_out, float* traj_out, double* latency_s) {
  if (!c) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv) return BRMPPI_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->by_ticket.find(ticket);
  if (it == sv->by_ticket.end()) return BRMPPI_EINVAL;
  const int s = it->second;
  Slot& sl = sv->slots[s];
  if (sl.state != kDone) return BRMPPI_EAGAIN;
  const float* out = sv->h_out + static_cast<size_t>(s) * sv->out_stride;
  const int32_t st = sl.status;
  if (st == BRMPPI_OK || st == BRMPPI_ENONFINITE) {
    if (U_out) std::memcpy(U_out, out, sizeof(float) * 3 * sv->H);
    if (traj_out) std::memcpy(traj_out, out + 3 * sv->H, sizeof(float) * 7 * (sv->H + 1));
  }
  if (latency_s) *latency_s = sl.t_done - sl.t_submit;
  sv->by_ticket.erase(it);
  if (sl.held) {
    sl.polled = true;  // freed when its batch finishes
  } else {
    sl.state = kFree;
    sv->free_slots.push_back(s);
  }
  return static_cast<brmppi_status>(st);
}

brmppi_status brmppi_vehicle_export(brmppi_ctx* c, uint32_t vid, float* U_nom, uint64_t* seed, uint64_t* counter) {
  if (!c) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv || vid >= sv->veh.size()) return BRMPPI_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  Vehicle& V = sv->veh[vid];
  if (!V.registered) return BRMPPI_EINVAL;
  if (V.queued > 0 || V.running) return BRMPPI_EBUSY;
  cudaSetDevice(c->device);
  if (U_nom && cudaMemcpy(U_nom, V.d_unom, sizeof(float) * 3 * sv->H, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BRMPPI_ECUDA;
  if (seed) *seed = V.seed;
  if (counter) *counter = V.counter;
  return BRMPPI_OK;
}

brmppi_status brmppi_vehicle_import(brmppi_ctx* c, uint32_t vid, const float* U_nom, uint64_t seed, uint64_t counter) {
  if (!c || !U_nom) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv || vid >= sv->veh.size()) return BRMPPI_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  Vehicle& V = sv->veh[vid];
  if (!V.registered) return BRMPPI_EINVAL;
  if (V.queued > 0 || V.running) return BRMPPI_EBUSY;
  cudaSetDevice(c->device);
  if (cudaMemcpy(V.d_unom, U_nom, sizeof(float) * 3 * sv->H, cudaMemcpyHostToDevice) != cudaSuccess)
    return BRMPPI_ECUDA;
  V.seed = seed;
  V.counter = counter;
  return BRMPPI_OK;
}

brmppi_status brmppi_server_stats_get(brmppi_ctx* c, brmppi_server_stats* out) {
  if (!c || !out) return BRMPPI_EINVAL;
  Server* sv = c->server;
  if (!sv) return BRMPPI_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->batches = sv->batches;
  out->solves_in_batches = sv->solves;
  out->request_slots = sv->n_slots;
  out->lanes = static_cast<int32_t>(sv->lanes.size());
  out->max_inflight_batches = sv->max_running;
  out->max_batch = sv->max_batch;
  return BRMPPI_OK;
}

}  // extern "C"
