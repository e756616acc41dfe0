// Continuous-batching request loop over the tracker: the serving form of
// processing several events at once (Sec. 2), fed with continuous-readout
// timeframes (Sec. 5) as requests.  Built on the public C ABI only.
//
// Requests queue in submission order.  A worker thread admits the head of the
// queue whenever a slot is free and the slot's arena for that request fits
// the HBM budget and the device's free memory.  Each slot owns a tracker
// context on its own CUDA stream, so a request admitted while others run
// overlaps with them on the GPU.  A slot keeps its arena (grid, links,
// tracklet and track buffers) between requests and grows it only for a
// larger request; idle slots give their arenas back when the budget would
// otherwise block the head of the queue.  Completion is seen through one
// CUDA event per slot; the worker then copies the results to host memory
// and frees the slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/tpcca.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Request {
  int64_t id = 0;
  const tpc_cluster* clusters = nullptr;
  int64_t n = 0;
  int state = RQ_QUEUED;
  int rc = TPC_OK;
  Clock::time_point t_submit, t_start, t_done;
  std::vector<tpc_track> tracks;
  std::vector<int32_t> cluster_track;
};

struct Slot {
  tpc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  size_t arena = 0;   // device bytes held by this slot's context
  Request* req = nullptr;  // running request (worker thread only)
};

constexpr size_t kHeadroom = size_t(256) << 20;  // free memory kept for other allocations

}  // namespace

struct tpc_server {
  tpc_config cfg{};
  int device = 0;
  size_t budget = 0;
  int32_t queue_cap = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<Request*> queue;
  std::map<int64_t, Request> reqs;
  std::thread worker;
  std::atomic<bool> stop{false};
  size_t reserved = 0;  // sum of the slots' arenas
  int64_t admitted = 0, completed = 0, peak_running = 0;

  void loop();
  int pick_slot_locked(size_t need, bool* any_busy);
  bool admit_one();
  void finish(Slot& s);
  void complete_locked(Request* r, int rc);
  int trim_idle_locked(size_t want);
};

void tpc_server::complete_locked(Request* r, int rc) {
  r->rc = rc;
  r->state = rc == TPC_OK ? RQ_DONE : RQ_FAILED;
  r->t_done = Clock::now();
  completed++;
  cv_done.notify_all();
}

// Recreate idle slots' contexts (dropping their arenas) until `want` more
// bytes fit the budget.  Returns the number of slots trimmed.
int tpc_server::trim_idle_locked(size_t want) {
  int trimmed = 0;
  for (Slot& s : slots) {
    if (budget == 0 || reserved + want <= budget) break;
    if (s.req || s.arena == 0) continue;
    tpc_ctx* fresh = nullptr;
    tpc_destroy(s.ctx);
    s.ctx = nullptr;
    reserved -= s.arena;
    s.arena = 0;
    if (tpc_create(&fresh, &cfg, device, s.stream, 0) == TPC_OK) s.ctx = fresh;
    trimmed++;
  }
  return trimmed;
}

// A free slot for a request needing `need` arena bytes: one that already
// holds enough, else one that may grow within the budget and free memory.
int tpc_server::pick_slot_locked(size_t need, bool* any_busy) {
  *any_busy = false;
  int fits = -1, grows = -1;
  for (size_t i = 0; i < slots.size(); i++) {
    if (slots[i].req) {
      *any_busy = true;
      continue;
    }
    if (!slots[i].ctx) continue;
    if (slots[i].arena >= need && fits < 0) fits = (int)i;
    if (grows < 0 || slots[i].arena > slots[grows].arena) grows = (int)i;
  }
  if (fits >= 0) return fits;
  if (grows < 0) return -1;
  size_t grow = need - slots[grows].arena;
  if (budget && reserved + grow > budget) {
    trim_idle_locked(grow);
    if (!slots[grows].ctx) return -1;
    grow = need - std::min(need, slots[grows].arena);
    if (reserved + grow > budget) return -1;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || grow + kHeadroom > free_b) return -1;
  return grows;
}

bool tpc_server::admit_one() {
  Request* r = nullptr;
  Slot* s = nullptr;
  size_t grow = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (queue.empty()) return false;
    r = queue.front();
    const size_t need = tpc_arena_bytes(r->n, 1);
    bool any_busy = false;
    const int pick = pick_slot_locked(need, &any_busy);
    if (pick < 0) {
      if (!any_busy && budget && need > budget) {  // can never fit
        queue.pop_front();
        complete_locked(r, TPC_ENOMEM);
        return true;
      }
      return false;
    }
    s = &slots[pick];
    grow = need > s->arena ? need - s->arena : 0;
    reserved += grow;
    s->arena += grow;
    queue.pop_front();
    r->state = RQ_RUNNING;
    r->t_start = Clock::now();
    s->req = r;
    admitted++;
    int64_t running = 0;
    for (const Slot& t : slots) running += t.req != nullptr;
    peak_running = std::max(peak_running, running);
  }
  // enqueue outside the lock: reserve, copy in, graph launch, completion event
  int rc = grow ? tpc_reserve(s->ctx, r->n, 1, 0, 0) : TPC_OK;
  if (rc == TPC_OK) rc = tpc_load_clusters(s->ctx, r->clusters, r->n, 0);
  if (rc == TPC_OK) rc = tpc_run_graph(s->ctx);
  if (rc == TPC_OK && cudaEventRecord(s->done, s->stream) != cudaSuccess) rc = TPC_ECUDA;
  if (rc != TPC_OK) {
    std::lock_guard<std::mutex> lk(mu);
    s->req = nullptr;
    complete_locked(r, rc);
  }
  return true;
}

void tpc_server::finish(Slot& s) {
  Request* r = s.req;
  int64_t nt = 0;
  // size query (TPC_EOVERFLOW with *n_out set when tracks exist), then copy
  int rc = tpc_get_tracks(s.ctx, nullptr, 0, &nt, nullptr, nullptr);
  if (rc == TPC_OK || (rc == TPC_EOVERFLOW && nt > 0)) {
    r->tracks.resize((size_t)nt);
    r->cluster_track.resize((size_t)r->n);
    rc = tpc_get_tracks(s.ctx, r->tracks.data(), nt, &nt, r->n ? r->cluster_track.data() : nullptr, nullptr);
  }
  if (rc == TPC_EOVERFLOW) {
    // an internal capacity (tracklets) overflowed: rerun once with the
    // worst-case capacity, synchronously on this slot
    rc = tpc_reserve(s.ctx, r->n, 1, 0, r->n / 3 + 16);
    if (rc == TPC_OK) rc = tpc_load_clusters(s.ctx, r->clusters, r->n, 0);
    if (rc == TPC_OK) rc = tpc_run_graph(s.ctx);
    if (rc == TPC_OK) rc = tpc_get_tracks(s.ctx, nullptr, 0, &nt, nullptr, nullptr);
    if (rc == TPC_OK || (rc == TPC_EOVERFLOW && nt > 0)) {
      r->tracks.resize((size_t)nt);
      r->cluster_track.resize((size_t)r->n);
      rc = tpc_get_tracks(s.ctx, r->tracks.data(), nt, &nt, r->n ? r->cluster_track.data() : nullptr, nullptr);
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  s.req = nullptr;
  complete_locked(r, rc);
}

void tpc_server::loop() {
  cudaSetDevice(device);
  while (!stop.load()) {
    bool active = false;
    for (Slot& s : slots) {
      if (!s.req) continue;
      active = true;
      if (cudaEventQuery(s.done) != cudaErrorNotReady) finish(s);
    }
    while (admit_one()) active = true;
    std::this_thread::sleep_for(std::chrono::microseconds(active ? 20 : 100));
  }
}

extern "C" {

int tpc_server_create(tpc_server** out, const tpc_config* cfg, int device, int32_t max_slots, size_t hbm_budget,
                      int32_t queue_cap) {
  if (!out || max_slots < 1 || max_slots > 64 || queue_cap < 1) return TPC_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return TPC_ECUDA;
  tpc_server* srv = new tpc_server();
  if (cfg) srv->cfg = *cfg;
  else tpc_default_config(&srv->cfg);
  srv->device = device;
  srv->budget = hbm_budget;
  srv->queue_cap = queue_cap;
  srv->slots.resize((size_t)max_slots);
  for (Slot& s : srv->slots) {
    int rc = TPC_OK;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
      rc = TPC_ECUDA;
    if (rc == TPC_OK) rc = tpc_create(&s.ctx, &srv->cfg, device, s.stream, 0);
    if (rc != TPC_OK) {
      tpc_server_destroy(srv);
      return rc;
    }
  }
  srv->worker = std::thread([srv] { srv->loop(); });
  *out = srv;
  return TPC_OK;
}

int tpc_server_submit(tpc_server* srv, int64_t request_id, const tpc_cluster* clusters, int64_t n) {
  if (!srv || n < 0 || (n > 0 && !clusters)) return TPC_EINVAL;
  if (srv->budget && tpc_arena_bytes(n, 1) > srv->budget) return TPC_ENOMEM;
  std::lock_guard<std::mutex> lk(srv->mu);
  if ((int32_t)srv->queue.size() >= srv->queue_cap) return TPC_EBUSY;
  if (srv->reqs.count(request_id)) return TPC_EINVAL;
  Request& r = srv->reqs[request_id];
  r.id = request_id;
  r.clusters = clusters;
  r.n = n;
  r.t_submit = Clock::now();
  srv->queue.push_back(&r);
  return TPC_OK;
}

int tpc_server_poll(tpc_server* srv, int64_t request_id, int* state) {
  if (!srv || !state) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  *state = it == srv->reqs.end() ? -1 : it->second.state;
  return TPC_OK;
}

int tpc_server_result(tpc_server* srv, int64_t request_id, tpc_track* out, int64_t cap, int64_t* n_out,
                      int32_t* cluster_track, double times_ms[3]) {
  if (!srv) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return TPC_EINVAL;
  Request& r = it->second;
  if (r.state < RQ_DONE) return TPC_EBUSY;
  if (n_out) *n_out = (int64_t)r.tracks.size();
  if (times_ms) {
    times_ms[0] = ms_between(r.t_submit, r.t_start);
    times_ms[1] = ms_between(r.t_start, r.t_done);
    times_ms[2] = ms_between(r.t_submit, r.t_done);
  }
  if (r.state == RQ_FAILED) {
    const int rc = r.rc;
    srv->reqs.erase(it);
    return rc;
  }
  if (!out && !cluster_track) return TPC_OK;  // size and time query
  if ((int64_t)r.tracks.size() > cap) return TPC_EOVERFLOW;
  if (out && !r.tracks.empty()) memcpy(out, r.tracks.data(), sizeof(tpc_track) * r.tracks.size());
  if (cluster_track && r.n) memcpy(cluster_track, r.cluster_track.data(), sizeof(int32_t) * (size_t)r.n);
  srv->reqs.erase(it);
  return TPC_OK;
}

int tpc_server_drain(tpc_server* srv, double timeout_s) {
  if (!srv) return TPC_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto idle = [srv] {
    for (auto& kv : srv->reqs)
      if (kv.second.state < RQ_DONE) return false;
    return true;
  };
  if (timeout_s <= 0) {
    srv->cv_done.wait(lk, idle);
    return TPC_OK;
  }
  return srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle) ? TPC_OK : TPC_ETIMEOUT;
}

int tpc_server_stats(tpc_server* srv, int64_t stats[5]) {
  if (!srv || !stats) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  stats[0] = srv->admitted;
  stats[1] = srv->completed;
  stats[2] = (int64_t)srv->queue.size();
  stats[3] = (int64_t)srv->reserved;
  stats[4] = srv->peak_running;
  return TPC_OK;
}

void tpc_server_destroy(tpc_server* srv) {
  if (!srv) return;
  srv->stop.store(true);
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->device);
  for (Slot& s : srv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.ctx) tpc_destroy(s.ctx);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  delete srv;
}

}  // extern "C"
