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
// larger request (stream-ordered, so other slots keep running); idle slots
// give their arenas back when the budget would otherwise block the head of
// the queue (outside the server's lock).  The worker polls one CUDA event per
// slot, then enqueues the copy of the results into the caller's buffers and
// polls again, so one request's copies overlap the others' kernels.  A
// request whose run overflowed a device capacity goes back to the head of
// the queue with the worst-case capacities and is admitted again under the
// same budget and free-memory checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
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
  tpc_track* out = nullptr;
  int64_t cap = 0;
  int32_t* cluster_track = nullptr;
  int state = RQ_QUEUED;
  int rc = TPC_OK;
  int64_t n_tracks = -1;
  bool retried = false;
  int64_t retry_bins = 0, retry_tl = 0;  // capacities of a rerun after a device capacity overflow
  Clock::time_point t_submit, t_start, t_done;
};

enum { SL_FREE = 0, SL_RUN = 1, SL_COPY = 2, SL_TRIM = 3 };

struct Slot {
  tpc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  size_t arena = 0;        // device bytes held by this slot's context
  int phase = SL_FREE;     // worker thread only
  Request* req = nullptr;  // worker thread only
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
  int pick_slot_locked(const Request* r, size_t* grow_out, bool* any_busy, bool* blocked_by_budget);
  bool admit_one();
  void advance(Slot& s);
  void complete(Slot& s, int rc);
  bool trim_idle(size_t want);
  int launch(Slot& s);
  void account(Slot& s);
};

// Book the slot's actual arena size (capacities only grow, and may exceed
// tpc_arena_bytes after a retry with larger tracklet capacity).
void tpc_server::account(Slot& s) {
  size_t b = 0;
  tpc_get_arena_bytes(s.ctx, &b);
  std::lock_guard<std::mutex> lk(mu);
  reserved = reserved - s.arena + b;
  s.arena = b;
}

// Drops the arenas of idle slots (destroying and re-creating their
// contexts) until `want` more bytes fit the budget.  The slots are taken out
// under the lock and rebuilt outside it, so tpc_server_submit and _poll never
// wait on the device meanwhile.  Returns whether any slot was trimmed.
bool tpc_server::trim_idle(size_t want) {
  std::vector<Slot*> victims;
  {
    std::lock_guard<std::mutex> lk(mu);
    size_t freed = 0;
    for (Slot& s : slots) {
      if (budget == 0 || reserved - freed + want <= budget) break;
      if (s.phase != SL_FREE || s.arena == 0 || !s.ctx) continue;
      s.phase = SL_TRIM;  // not picked while it is rebuilt
      freed += s.arena;
      victims.push_back(&s);
    }
  }
  for (Slot* s : victims) {
    tpc_destroy(s->ctx);  // frees the arena
    s->ctx = nullptr;
    tpc_ctx* fresh = nullptr;
    if (tpc_create(&fresh, &cfg, device, s->stream, 0) == TPC_OK) s->ctx = fresh;  // else rebuilt when next picked
    std::lock_guard<std::mutex> lk(mu);
    reserved -= s->arena;
    s->arena = 0;
    s->phase = SL_FREE;
  }
  return !victims.empty();
}

// A free slot for request r and the bytes its arena must grow by: the
// smallest arena that needs no growth, else the slot that grows least,
// within the budget and the free device memory.  *blocked_by_budget: a slot
// could take r if idle arenas were dropped.
int tpc_server::pick_slot_locked(const Request* r, size_t* grow_out, bool* any_busy, bool* blocked_by_budget) {
  *any_busy = false;
  *blocked_by_budget = false;
  int best = -1;
  size_t best_grow = 0;
  for (size_t i = 0; i < slots.size(); i++) {
    Slot& s = slots[i];
    if (s.phase != SL_FREE) {
      *any_busy = *any_busy || s.phase != SL_TRIM;
      continue;
    }
    if (!s.ctx) {  // a context that could not be re-created after a trim: try again
      tpc_ctx* fresh = nullptr;
      if (tpc_create(&fresh, &cfg, device, s.stream, 0) != TPC_OK) continue;
      s.ctx = fresh;
    }
    size_t after = 0;
    if (tpc_reserve_bytes(s.ctx, r->n, 1, r->retry_bins, r->retry_tl, &after) != TPC_OK) continue;
    const size_t grow = after > s.arena ? after - s.arena : 0;
    if (best < 0 || grow < best_grow || (grow == best_grow && s.arena < slots[best].arena)) {
      best = (int)i;
      best_grow = grow;
    }
  }
  if (best < 0) return -1;
  if (budget && reserved + best_grow > budget) {
    *blocked_by_budget = true;
    return -1;
  }
  size_t free_b = 0, total_b = 0;
  if (best_grow && (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || best_grow + kHeadroom > free_b)) return -1;
  *grow_out = best_grow;
  return best;
}

int tpc_server::launch(Slot& s) {
  Request* r = s.req;
  int rc = tpc_load_clusters(s.ctx, r->clusters, r->n, 0);
  if (rc == TPC_OK) rc = tpc_run_graph(s.ctx);
  if (rc == TPC_OK && cudaEventRecord(s.done, s.stream) != cudaSuccess) rc = TPC_ECUDA;
  return rc;
}

bool tpc_server::admit_one() {
  Request* r = nullptr;
  Slot* s = nullptr;
  size_t grow = 0;
  size_t trim_want = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (queue.empty()) return false;
    r = queue.front();
    const size_t need = tpc_arena_bytes_for(r->n, 1, r->retry_bins, r->retry_tl);
    bool any_busy = false, blocked = false;
    const int pick = pick_slot_locked(r, &grow, &any_busy, &blocked);
    if (pick < 0) {
      if (!any_busy && budget && need > budget) {  // can never fit
        queue.pop_front();
        r->rc = TPC_ENOMEM;
        r->state = RQ_FAILED;
        r->t_start = r->t_done = Clock::now();
        completed++;
        cv_done.notify_all();
        return true;
      }
      if (!blocked) return false;
      trim_want = need;
    } else {
      s = &slots[pick];
      reserved += grow;  // booked now; account() corrects it to the arena's real size
      s->arena += grow;
      queue.pop_front();
      r->state = RQ_RUNNING;
      r->t_start = Clock::now();
      s->req = r;
      s->phase = SL_RUN;
      admitted++;
      int64_t running = 0;
      for (const Slot& t : slots) running += t.phase == SL_RUN || t.phase == SL_COPY;
      peak_running = std::max(peak_running, running);
    }
  }
  if (!s) return trim_idle(trim_want);  // the budget blocks the head: drop idle arenas, then try again
  // enqueue outside the lock: arena growth, copy in, graph, completion event
  int rc = tpc_reserve(s->ctx, r->n, 1, r->retry_bins, r->retry_tl);
  account(*s);
  if (rc == TPC_OK) rc = launch(*s);
  if (rc != TPC_OK) complete(*s, rc);
  return true;
}

void tpc_server::complete(Slot& s, int rc) {
  Request* r = s.req;
  std::lock_guard<std::mutex> lk(mu);
  r->rc = rc;
  r->state = rc == TPC_OK ? RQ_DONE : RQ_FAILED;
  r->t_done = Clock::now();
  s.req = nullptr;
  s.phase = SL_FREE;
  completed++;
  cv_done.notify_all();
}

// One step of a slot whose event has fired.
void tpc_server::advance(Slot& s) {
  Request* r = s.req;
  if (s.phase == SL_COPY) {
    complete(s, TPC_OK);
    return;
  }
  int64_t nt = -1;
  int rc = tpc_get_tracks_async(s.ctx, r->out, r->cap, &nt, r->cluster_track);
  if (rc == TPC_EOVERFLOW && nt < 0 && !r->retried) {
    // a device capacity (grid bins, tracklets) overflowed: the request goes
    // back to the head of the queue with the worst-case capacities, and is
    // admitted again like any other (budget, free memory)
    int64_t counts[8] = {0};
    tpc_get_counts(s.ctx, counts);
    std::lock_guard<std::mutex> lk(mu);
    r->retried = true;
    r->retry_bins = 2 * std::max<int64_t>(counts[3], 1);
    r->retry_tl = r->n / 3 + 16;
    r->state = RQ_QUEUED;
    s.req = nullptr;
    s.phase = SL_FREE;
    queue.push_front(r);
    return;
  }
  r->n_tracks = nt;
  if (rc != TPC_OK || cudaEventRecord(s.done, s.stream) != cudaSuccess) {
    complete(s, rc != TPC_OK ? rc : TPC_ECUDA);
    return;
  }
  s.phase = SL_COPY;
}

void tpc_server::loop() {
  cudaSetDevice(device);
  while (!stop.load()) {
    bool active = false;
    for (Slot& s : slots) {
      if (s.phase == SL_FREE || s.phase == SL_TRIM) continue;
      active = true;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaSuccess) advance(s);
      else if (q != cudaErrorNotReady) complete(s, TPC_ECUDA);
    }
    while (admit_one()) active = true;
    std::this_thread::sleep_for(std::chrono::microseconds(active ? 10 : 100));
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

int tpc_server_submit(tpc_server* srv, int64_t request_id, const tpc_cluster* clusters, int64_t n,
                      tpc_track* tracks_out, int64_t cap, int32_t* cluster_track_out) {
  if (!srv || n < 0 || (n > 0 && !clusters) || cap < 0 || (cap > 0 && !tracks_out)) return TPC_EINVAL;
  if (srv->budget && tpc_arena_bytes(n, 1) > srv->budget) return TPC_ENOMEM;
  std::lock_guard<std::mutex> lk(srv->mu);
  if ((int32_t)srv->queue.size() >= srv->queue_cap) return TPC_EBUSY;
  if (srv->reqs.count(request_id)) return TPC_EINVAL;
  Request& r = srv->reqs[request_id];
  r.id = request_id;
  r.clusters = clusters;
  r.n = n;
  r.out = tracks_out;
  r.cap = cap;
  r.cluster_track = cluster_track_out;
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

int tpc_server_result(tpc_server* srv, int64_t request_id, int64_t* n_tracks, double times_ms[3]) {
  if (!srv) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return TPC_EINVAL;
  Request& r = it->second;
  if (r.state < RQ_DONE) return TPC_EBUSY;
  if (n_tracks) *n_tracks = r.n_tracks;
  if (times_ms) {
    times_ms[0] = ms_between(r.t_submit, r.t_start);
    times_ms[1] = ms_between(r.t_start, r.t_done);
    times_ms[2] = ms_between(r.t_submit, r.t_done);
  }
  const int rc = r.rc;
  srv->reqs.erase(it);
  return rc;
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
