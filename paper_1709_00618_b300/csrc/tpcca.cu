// libtpcca: C ABI of the B300 sector tracker.  One translation unit: the
// kernels are included from the headers beside this file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "scan.cuh"
#include "grid.cuh"
#include "links.cuh"
#include "kalman.cuh"
#include "follow.cuh"
#include "select.cuh"
#include "probe.cuh"
#include "vertex.cuh"
#include "codec.cuh"
#include "merge.cuh"
#include "reject.cuh"
#include "batch.cuh"

using namespace tpc;

namespace {

constexpr size_t ALIGN = 256;
enum { BATCH_NONE = 0, BATCH_RUNNING = 1, BATCH_COPYING = 2, BATCH_DONE = 3 };
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// Geometry of the reading: X_r = (float)(85.2 + r*((245.8-85.2)/158)),
// Y_r = (float)(that double * tan 10 deg).
void geometry_tables(float* x, float* yhi) {
  for (int r = 0; r < NROW; r++) {
    double xd = 85.2 + r * ((245.8 - 85.2) / 158.0);
    x[r] = (float)xd;
    yhi[r] = (float)(xd * 0.17632698070846498);
  }
  x[NROW] = x[NROW - 1];
  yhi[NROW] = yhi[NROW - 1];
}

// Unique id of the calling thread's current CUDA context (0 when it cannot
// be had).  Device-side state that belongs to the loaded module -- the row
// tables and the allocation-free entry point's scratch array -- lives as
// long as that context: after cudaDeviceReset the runtime creates a new
// primary context with a new id, reloads the module, and the per-device
// set-up below runs again instead of trusting an address of the old one.
unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

std::mutex g_dev_mutex;
std::vector<unsigned long long> g_dev_ready;  // per device: context id the tables were uploaded in

// Uploads the row tables once per device and context; the device must be
// current.
cudaError_t ensure_device_tables(int device) {
  cudaError_t e = cudaSetDevice(device);  // also creates the device's primary context
  if (e != cudaSuccess) return e;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  if ((int)g_dev_ready.size() <= device) g_dev_ready.resize(device + 1, 0);
  if (id != 0 && g_dev_ready[device] == id) return cudaSuccess;
  float x[NROW + 1], y[NROW + 1];
  geometry_tables(x, y);
  e = cudaMemcpyToSymbol(g_row_x, x, sizeof(x));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_row_yhi, y, sizeof(y));
  if (e == cudaSuccess) g_dev_ready[device] = id;
  return e;
}

struct Caps {
  int64_t n = 0;      // clusters
  int32_t req = 0;    // requests
  int64_t bins = 0;   // grid bins
  int64_t tl = 0;     // tracklets
  int64_t tracks = 0; // tracks
  int64_t nrs() const { return (int64_t)req * NSEC * NROW; }
};

Caps default_caps(int64_t n, int32_t req) {
  Caps c;
  c.n = std::max<int64_t>(n, 1024);
  c.req = std::max<int32_t>(req, 1);
  // Grid bins: about n/2 in total plus, per row-sector, a few for an empty
  // one and of order sqrt(n_r dz / 2 wy) for a long drift range; the
  // default holds the measured events, timeframes and batches with room to
  // spare, and an overflow (reported, never truncated) is retried with
  // tpc_reserve.
  c.bins = 2 * c.n + 16 * c.nrs() + 4096;
  // Tracklets: chains are disjoint and hold >= 3 clusters, so n/3 can never
  // overflow; measured events, timeframes and batches give 0.064 per
  // cluster, so the default is n/12 and an overflow is retried the same way.
  c.tl = c.n / 12 + 1024;
  c.tracks = c.tl;  // tracks are a subset of the tracklets
  return c;
}

// Offsets of every device array inside the arena.
struct Layout {
  size_t counts, req_off, req_trk, buckets, starts, in, rs_in, gbin, slot, tmp, perm, yz, rs_of, up, dn, up_m, dn_m, tie, flag, fidx, clen,
      cend, owner, cluster_track, track_clusters;
  size_t rs_cnt, rs_start, zmin, zmax, par, nbins, bin_base;
  size_t bin_cnt, bin_start;
  size_t own_mask, own_rng, fwork, rwork, okey, order, obins, ztail_list, ztail_cov;
  size_t tl_start, tl_len, tl_end, f_n, f_nf, f_nb, f_flags, f_row, hits, hrow, f_par, f_zref, f_cov, f_chi2, keep,
      tidx, nown, tl_track, track_tl, tcount, toff, tracks;
  size_t parts;
  size_t trace;
  size_t total;
};

constexpr int TRACE_RECORDS = 2048;
// Slots per pass of the zone tail lists (follow.cuh): about 10% of the
// zones outlast the zone kernels' in-step rows; a tracklet that finds no
// slot finishes its zone in place.
size_t zone_tail_cap(size_t T) { return T / 4 + 64; }

Layout make_layout(const Caps& c) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t N = (size_t)c.n, R = (size_t)c.req, NRS = (size_t)c.nrs(), B = (size_t)c.bins, T = (size_t)c.tl,
               M = (size_t)c.tracks;
  L.counts = take(sizeof(Counts));
  L.req_off = take(8 * (R + 1));
  L.req_trk = take(8 * R);  // per request: first track, one past its last (tpc_submit_batch)
  L.buckets = take(sizeof(GridBuckets));
  L.in = take(16 * N);
  // Arrays that live only in the grid stage share their space with arrays
  // that are first written after it: rs_in with track_clusters (a8);
  // gbin | slot with flag | fidx (a5); the sorted records (tmp) with owner
  // (a7; cleared in a4) | clen | cend (a5).
  L.rs_in = take(4 * N);
  L.track_clusters = L.rs_in;
  L.gbin = take(8 * (N + 1));
  L.slot = L.gbin + 4 * (N + 1);
  L.flag = L.gbin;
  L.fidx = L.slot;
  L.tmp = take(16 * N);  // records of the grid's counting sort
  L.owner = L.tmp;
  L.clen = L.tmp + 8 * N;
  L.cend = L.tmp + 12 * N;
  L.perm = take(4 * N);
  L.yz = take(8 * N);
  L.rs_of = take(4 * N);
  // up, dn, up_m, dn_m are contiguous: during the grid stage, before the
  // links exist, the 16 N bytes from up on hold the bucketed records
  L.up = take(4 * N);
  L.dn = take(4 * N);
  L.up_m = take(4 * N);
  L.dn_m = take(4 * N);
  L.tie = take(N);
  L.starts = take(4 * (N / 2 + 1));  // chain starts: chains are disjoint and hold >= 2 clusters
  L.cluster_track = take(4 * N);
  L.rs_cnt = take(4 * (NRS + 1));
  L.rs_start = take(4 * (NRS + 1));
  L.zmin = take(4 * NRS);
  L.zmax = take(4 * NRS);
  L.par = take(sizeof(RsParams) * NRS);
  L.nbins = take(4 * (NRS + 1));
  L.bin_base = take(4 * (NRS + 1));
  L.bin_cnt = take(4 * (B + 1));
  L.bin_start = take(4 * (B + 1));
  L.tl_start = take(4 * T);
  L.tl_len = take(4 * T);
  L.tl_end = take(4 * T);
  L.f_n = take(4 * T);
  L.f_nf = take(4 * T);
  L.f_nb = take(4 * T);
  L.f_flags = take(4 * T);
  L.f_row = take(4 * T);
  L.hits = take(4 * T * NROW);
  L.hrow = take(T * NROW);
  L.f_par = take(4 * 5 * T);
  L.f_zref = take(4 * T);
  L.f_cov = take(4 * 15 * T);
  L.f_chi2 = take(8 * T);
  L.keep = take(4 * (T + 1));
  L.tidx = take(4 * (T + 1));
  L.nown = take(4 * T);
  L.own_mask = take(4 * OWN_WORDS * T);
  L.fwork = take(sizeof(FollowWork) * T);
  L.ztail_list = take(4 * 3 * zone_tail_cap(T));  // follow forward, follow backward, refit (M <= T)
  L.ztail_cov = take(8 * 15 * 3 * zone_tail_cap(T));
  L.rwork = take(sizeof(RefitWork) * M);
  L.okey = take(std::max(T, M));
  L.order = take(4 * std::max(T, M));
  L.obins = take(4 * ORD_WORDS);
  L.own_rng = take(4 * T);
  L.tl_track = take(4 * T);
  L.track_tl = take(4 * M);
  L.tcount = take(4 * (M + 1));
  L.toff = take(4 * (M + 1));
  L.tracks = take(sizeof(tpc_track) * M);
  L.parts = take(4 * SCAN_PARTS);
  L.trace = take(4 * TRACE_W * TRACE_RECORDS);
  L.total = off;
  return L;
}

}  // namespace

struct tpc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  tpc_config cfg{};
  KConst kc{};
  Caps caps{};
  Layout L{};
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  size_t budget = 0;
  int n_sm = 148;
  // current batch
  int64_t n = 0;
  int32_t n_req = 0;
  bool loaded = false, found = false, fitted = false;
  Counts* h_counts = nullptr;  // pinned mirror
  int64_t* h_req = nullptr;    // pinned request offsets
  int32_t h_req_cap = 0;
  int32_t* h_req_trk = nullptr;  // pinned: per request first track, one past its last
  // batch submitted with tpc_submit_batch, tracked by tpc_poll
  struct BatchReq {
    tpc_request r;
    int64_t off = 0;  // first cluster of the request in the batch
    int rc = TPC_OK;
    bool done = false;
  };
  std::vector<BatchReq> batch;
  int batch_state = 0;  // BATCH_*
  bool batch_retried = false;
  cudaEvent_t ev_batch = nullptr;
  // tuning
  int block_clusters = 256;
  int block_follow = 128;
  int ctas_zone = 0;     // cap on CTAs per SM of the FP64-zone Kalman kernels (0: by size)
  int ctas_follow = 0;   // cap on CTAs per SM of the refilling Kalman kernels (64: occupancy; 0: by size)
  int refill = 8;        // idle lanes that trigger a warp's refill
  int chunks = 0;        // Kalman-stage chunks (2: zone and FP32 kernels of different chunks overlap; 0: 1)
  int zone_rows = 0;     // zone rows in step before the zone tail kernels (0: by size; NROW or more: no tails)
  int graph_chunks = 0;  // chunks and refilling-kernel CTAs per SM of the captured graph
  int graph_ctas = 0;
  int graph_class = -1;  // the size class (size_class) the graph's kernel variants were chosen for
  cudaStream_t aux = nullptr;       // second stream of the chunked Kalman stage
  // tpc_track_host: the stream of the cluster assignment's copy-out, which
  // overlaps the refit, and its fork and join events (created on first use)
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_sel = nullptr, ev_copied = nullptr;
  // vertex finding (tpc_find_vertices): its own buffer, allocated on first use
  void* vtx_mem = nullptr;
  int64_t vtx_tracks_cap = 0;
  VtxBuf vb{};
  double* vtx_time = nullptr;
  int32_t* vtx_ntr = nullptr;
  int32_t* h_vtx_n = nullptr;  // pinned mirror of vb.n
  bool vtx_valid = false;
  // track-model compression (tpc_compress / tpc_decompress): own buffer
  void* codec_mem = nullptr;
  int64_t codec_tracks_cap = 0, codec_clusters_cap = 0;
  CodecIo cio{};
  int32_t* codec_bad = nullptr;
  bool codec_valid = false;
  // sector merging (tpc_merge_tracks): own buffer
  void* merge_mem = nullptr;
  int64_t merge_tracks_cap = 0, merge_cells_cap = 0;
  MergeBuf mb{};
  int32_t* h_merge_n = nullptr;  // pinned: merged tracks
  bool merge_valid = false;
  // cluster rejection (tpc_reject_clusters): own buffer
  void* reject_mem = nullptr;
  int64_t reject_tracks_cap = 0, reject_clusters_cap = 0;
  RejBuf rb{};
  bool reject_valid = false;
  // fits enqueued so far, and the fit the vertices belong to
  int64_t fit_gen = 0, vtx_gen = -1;
  float vtx_vdrift = 2.5f;
  cudaEvent_t ev_chunk[4] = {};     // fork and join of the chunked follow and refit
  // graph
  cudaGraphExec_t graph = nullptr;
  int32_t trace_t = -1;  // traced tracklet
  // stage events
  bool prof = false;
  bool prof_valid = false;
  cudaEvent_t ev[7] = {};
  // after follow p1, p1t, p2, p3, p3t, p4r; before refit p1; after refit p1, p1t, p2
  cudaEvent_t evk[PH_COUNT] = {};
  int32_t graph_kernels = 0;  // kernel nodes of the captured graph
  std::string err;

  void mark(int i) {
    if (prof) cudaEventRecord(ev[i], stream);
  }
  void mark_k(int i) {
    if (prof) cudaEventRecord(evk[i], stream);
  }

  template <typename T>
  T* ptr(size_t off) const { return reinterpret_cast<T*>(arena + off); }
};

namespace {

int fail(tpc_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, TPC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

KConst make_kconst(const tpc_config& c, const Caps& caps) {
  KConst k{};
  k.inner_steps = 1;
  k.zone_tail_cap = (int64_t)zone_tail_cap((size_t)caps.tl);
  k.K = (float)(0.299792458e-3 * c.bz_kg);
  k.V = (float)(c.sigma * c.sigma);
  k.Vd = c.sigma * c.sigma;
  k.d_max = c.d_max;
  k.wy = (float)(2.0 * ((245.8 - 85.2) / 158.0) + 0.5);
  k.wz = (float)(2.5 * ((245.8 - 85.2) / 158.0) + 0.5);
  k.wy2 = (float)(2 * 2.0 * ((245.8 - 85.2) / 158.0) + 0.5);
  k.wz2 = (float)(2 * 2.5 * ((245.8 - 85.2) / 158.0) + 0.5);
  k.link_skip = c.link_skip;
  k.gate = (float)c.gate;
  for (int i = 0; i < 5; i++) k.c0[i] = (float)c.c0[i];
  k.s_max = (float)c.s_max;
  k.edge = (float)c.edge;
  k.taint = (float)c.taint_rel;
  k.min_chain = c.min_chain;
  k.max_miss = c.max_miss;
  k.n_min_track = c.n_min_track;
  k.fp64_updates = c.fp64_updates;
  k.bins_cap = caps.bins;
  k.tl_cap = caps.tl;
  return k;
}

// Chunks of the Kalman stage: the tuned value, else 1 (measured on B300: the
// overlap gains under 1% on 16 M clusters and loses on 1 M, where launch and
// join costs weigh more; the autotuner tries both).
constexpr int64_t kLargeBatch = int64_t(4) << 20;  // clusters from which the size default switches
constexpr int64_t kZoneTailBwd = int64_t(16) << 20;  // clusters from which the backward zone has a tail kernel
constexpr int64_t kZoneTailFwd = int64_t(48) << 20;  // ... the forward and refit zones
// The input-size class that picks kernel variants and launch shapes.
int size_class(int64_t n) { return (n >= kLargeBatch) + (n >= kZoneTailBwd) + (n >= kZoneTailFwd); }
int effective_chunks(const tpc_ctx* ctx) { return ctx->chunks > 0 ? ctx->chunks : 1; }
// 32-bit ownership keys while every tracklet id fits 24 bits (select.cuh).
bool key32(const tpc_ctx* ctx) { return ctx->caps.tl < (int64_t(1) << 24); }
// CTAs per SM of the refilling Kalman kernels: the tuned value, or by size
// (a small batch is bound by its longest tracklet, a large one by throughput).
int effective_ctas_follow(const tpc_ctx* ctx) {
  if (ctx->ctas_follow > 0) return ctx->ctas_follow;
  return ctx->n >= kLargeBatch ? 64 : 2;
}
// CTAs per SM of the FP64-zone kernels: the tuned value, or by size (a small
// batch's zone kernels end with the tracklets of their last wave, so fewer
// resident warps shorten the tail; on a large batch the FP64 pipe needs as
// many warps as the zone's registers allow, four 128-thread CTAs).
int effective_ctas_zone(const tpc_ctx* ctx) {
  if (ctx->ctas_zone > 0) return ctx->ctas_zone;
  return ctx->n >= kLargeBatch ? 4 : 2;
}

WorkOrder work_order(tpc_ctx* ctx, int phase, int chunk) {
  const Layout& L = ctx->L;
  WorkOrder o;
  o.hist = ctx->ptr<int32_t>(L.obins) + (phase * MAX_CHUNKS + chunk) * 2 * ORD_BINS;
  o.cursor = o.hist + ORD_BINS;
  o.key = ctx->ptr<uint8_t>(L.okey);
  o.order = ctx->ptr<int32_t>(L.order);
  return o;
}

// Blocks of a persistent Kalman kernel: as many as are resident at once
// (one wave), at most ctas_follow per SM.
template <typename Kernel>
int persistent_grid(tpc_ctx* ctx, Kernel kernel, int threads, int cap) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return ctx->n_sm * std::max(1, std::min(per_sm, cap));
}

int grid_for(const tpc_ctx* ctx, int64_t items, int threads, int per_sm = 16) {
  int64_t b = (items + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->n_sm * per_sm;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

// One item per thread, all items in one grid.  For items of uneven work
// (tracklets of 10 to 159 hits) a block ends with its own items and the next
// one starts, where a grid-stride loop would keep every block to its
// slowest thread per stride; for uniform items the capped grid's
// grid-stride loop is faster (no block launch per 256 items).
int grid_lin(int64_t items, int threads) { return (int)std::max<int64_t>(1, (items + threads - 1) / threads); }

int do_reserve(tpc_ctx* ctx, const Caps& want) {
  Caps c = ctx->caps;
  bool grow = want.n > c.n || want.req > c.req || want.bins > c.bins || want.tl > c.tl || want.tracks > c.tracks ||
              ctx->arena == nullptr;
  if (!grow) return TPC_OK;
  c.n = std::max(c.n, want.n);
  c.req = std::max(c.req, want.req);
  c.bins = std::max(c.bins, want.bins);
  c.tl = std::max(c.tl, want.tl);
  c.tracks = std::max(c.tracks, want.tracks);
  Layout L = make_layout(c);
  if (ctx->own_arena) {
    if (ctx->budget && L.total > ctx->budget)
      return fail(ctx, TPC_ENOMEM, "arena of %zu bytes exceeds the HBM budget of %zu bytes", L.total, ctx->budget);
    // stream-ordered: neither the free nor the allocation waits for other
    // streams of the device (contexts of a server keep running meanwhile)
    CK(cudaSetDevice(ctx->device));
    if (ctx->arena) {
      CK(cudaFreeAsync(ctx->arena, ctx->stream));
      ctx->arena = nullptr;
      ctx->arena_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, L.total, ctx->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->caps = Caps{};
      ctx->loaded = ctx->found = ctx->fitted = false;
      return fail(ctx, TPC_ENOMEM, "cudaMallocAsync(%zu): %s", L.total, cudaGetErrorString(e));
    }
    ctx->arena = (char*)p;
    ctx->arena_bytes = L.total;
  } else if (L.total > ctx->arena_bytes) {
    return fail(ctx, TPC_ENOMEM, "caller arena of %zu bytes is smaller than the %zu bytes needed", ctx->arena_bytes,
                L.total);
  }
  ctx->caps = c;
  ctx->L = L;
  ctx->kc = make_kconst(ctx->cfg, c);
  ctx->kc.refill = ctx->refill;
  ctx->kc.trace_t = ctx->trace_t;
  ctx->kc.trace_cap = TRACE_RECORDS;
  ctx->kc.trace = ctx->ptr<float>(L.trace);
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (ctx->h_req_cap < c.req + 1) {
    if (ctx->h_req) cudaFreeHost(ctx->h_req);
    if (ctx->h_req_trk) cudaFreeHost(ctx->h_req_trk);
    ctx->h_req = nullptr;
    ctx->h_req_trk = nullptr;
    ctx->h_req_cap = 0;
    CK(cudaMallocHost(&ctx->h_req, sizeof(int64_t) * (c.req + 1)));
    CK(cudaMallocHost(&ctx->h_req_trk, sizeof(int32_t) * 2 * (c.req + 1)));
    ctx->h_req_cap = c.req + 1;
  }
  return TPC_OK;
}

int create_common(tpc_ctx** out, const tpc_config* cfg, int device, void* stream) {
  if (!out) return TPC_EINVAL;
  *out = nullptr;
  tpc_ctx* ctx = new tpc_ctx();
  if (cfg) ctx->cfg = *cfg;
  else tpc_default_config(&ctx->cfg);
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return TPC_ECUDA;
  }
  e = ensure_device_tables(device);
  if (e != cudaSuccess) {
    delete ctx;
    return TPC_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return TPC_ECUDA;
    }
    ctx->own_stream = true;
  }
  bool ok = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 4 && ok; i++) ok = cudaEventCreateWithFlags(&ctx->ev_chunk[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok || cudaMallocHost(&ctx->h_counts, sizeof(Counts)) != cudaSuccess) {
    for (int i = 0; i < 4; i++)
      if (ctx->ev_chunk[i]) cudaEventDestroy(ctx->ev_chunk[i]);
    if (ctx->vtx_mem) cudaFree(ctx->vtx_mem);
  if (ctx->codec_mem) cudaFree(ctx->codec_mem);
  if (ctx->merge_mem) cudaFree(ctx->merge_mem);
  if (ctx->reject_mem) cudaFree(ctx->reject_mem);
  if (ctx->h_merge_n) cudaFreeHost(ctx->h_merge_n);
  if (ctx->h_vtx_n) cudaFreeHost(ctx->h_vtx_n);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return TPC_ECUDA;
  }
  memset(ctx->h_counts, 0, sizeof(Counts));
  *out = ctx;
  return TPC_OK;
}

// Validate the config (the same bounds the kernels assume).
bool config_ok(const tpc_config& c) {
  return std::isfinite(c.bz_kg) && c.sigma > 0 && c.d_max >= 0 && c.min_chain >= 2 && c.min_chain <= NROW &&
         c.max_miss >= 1 && c.n_min_track >= 1 && c.n_min_track <= NROW && c.gate > 0 && c.s_max > 0 &&
         c.s_max < 1 && c.fp64_updates >= 0 && c.taint_rel >= 0 && (c.link_skip == 0 || c.link_skip == 1);
}

// Exclusive scan of a device-resident length; cap: an upper bound of the
// length (a short array is scanned by one block).
void scan(tpc_ctx* ctx, const int32_t* in, int32_t* out, LenSrc len, int32_t* total_out, int64_t cap = -1) {
  Counts* cn = ctx->ptr<Counts>(ctx->L.counts);
  if (cap >= 0 && cap <= 8 * SCAN_TILE) {
    k_scan_small<<<1, SCAN_THREADS, 0, ctx->stream>>>(in, len, out, total_out, cn);
    return;
  }
  int32_t* parts = ctx->ptr<int32_t>(ctx->L.parts);
  k_scan_reduce<<<SCAN_PARTS, SCAN_THREADS, 0, ctx->stream>>>(in, len, parts, cn);
  k_scan_parts<<<1, 1024, 0, ctx->stream>>>(parts, SCAN_PARTS, total_out, cn);
  k_scan_down<<<SCAN_PARTS, SCAN_THREADS, 0, ctx->stream>>>(in, len, parts, out, cn);
}

GridView grid_view(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  GridView g;
  g.yz = ctx->ptr<float2>(L.yz);
  g.rs_of = ctx->ptr<int32_t>(L.rs_of);
  g.par = ctx->ptr<RsParams>(L.par);
  g.bin_start = ctx->ptr<int32_t>(L.bin_start);
  return g;
}

FollowOut follow_out(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  FollowOut o;
  o.n = ctx->ptr<int32_t>(L.f_n);
  o.nf = ctx->ptr<int32_t>(L.f_nf);
  o.nb = ctx->ptr<int32_t>(L.f_nb);
  o.flags = ctx->ptr<int32_t>(L.f_flags);
  o.row = ctx->ptr<int32_t>(L.f_row);
  o.hits = ctx->ptr<int32_t>(L.hits);
  o.hrow = ctx->ptr<uint8_t>(L.hrow);
  o.par = ctx->ptr<float>(L.f_par);
  o.zref = ctx->ptr<float>(L.f_zref);
  o.cov = ctx->ptr<float>(L.f_cov);
  o.chi2 = ctx->ptr<double>(L.f_chi2);
  return o;
}

// a2..a7 on the context's stream (capacity-sized grids: graph-capturable).
void enqueue_find(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  const Caps& C = ctx->caps;
  cudaStream_t s = ctx->stream;
  Counts* cn = ctx->ptr<Counts>(L.counts);
  const int bc = ctx->block_clusters;
  const int gN = grid_for(ctx, C.n, bc), gR = grid_for(ctx, C.nrs(), bc);
  int gT = grid_for(ctx, C.tl, bc);
  const int gTw = grid_for(ctx, C.tl * 32, bc);  // warp-per-tracklet kernels
  int32_t* rs_cnt = ctx->ptr<int32_t>(L.rs_cnt);
  int32_t* nbins = ctx->ptr<int32_t>(L.nbins);
  int32_t* bin_base = ctx->ptr<int32_t>(L.bin_base);
  int32_t* bin_cnt = ctx->ptr<int32_t>(L.bin_cnt);
  int32_t* bin_start = ctx->ptr<int32_t>(L.bin_start);
  ctx->kc.inner_steps = ctx->n < kLargeBatch ? 16 : 4;  // 10 ms timeframe: 1 step 69.0 ms, 2 68.7, 4 68.6, 8 68.8
  // zone rows in step before a zone goes to the tail kernels (follow.cuh).
  // 10 ms timeframe (90 M clusters): p1 10.06 ms without tails, 9.26 with 9
  // rows (9.65 with 10); p3 11.25 without, 10.03 with 10, 9.92 with 9; refit
  // p1 4.09 without, 3.75 with 10.  A tail kernel costs a launch whose last lanes run alone, so on
  // smaller inputs the tails gain less: 3 ms timeframe (25.5 M) p1 3.06 ->
  // 3.15, p3 3.26 -> 3.09, refit p1 1.28 -> 1.31; 1 ms (8.3 M) all three
  // slower.  Hence the backward pass's tail from 16 Mi clusters, the forward
  // pass's and the refit's from 48 Mi.
  ctx->kc.zone_steps[0] = ctx->n < kZoneTailFwd ? 0 : 9;
  ctx->kc.zone_steps[1] = ctx->n < kZoneTailBwd ? 0 : 9;
  ctx->kc.zone_steps[2] = ctx->n < kZoneTailFwd ? 0 : 10;
  if (ctx->zone_rows > 0)
    for (int i = 0; i < 3; i++) ctx->kc.zone_steps[i] = ctx->zone_rows < NROW ? ctx->zone_rows : 0;
  ctx->mark(0);
  // a2 grid
  k_rs_init<<<gR, bc, 0, s>>>(rs_cnt, ctx->ptr<uint32_t>(L.zmin), ctx->ptr<uint32_t>(L.zmax),
                              ctx->ptr<int32_t>(L.obins), cn);
  k_grid_count<<<gN, bc, 0, s>>>(ctx->ptr<tpc_cluster>(L.in), ctx->ptr<int64_t>(L.req_off), cn,
                                 ctx->ptr<int32_t>(L.rs_in), rs_cnt, ctx->ptr<uint32_t>(L.zmin),
                                 ctx->ptr<uint32_t>(L.zmax));
  k_grid_params<<<gR, bc, 0, s>>>(rs_cnt, ctx->ptr<uint32_t>(L.zmin), ctx->ptr<uint32_t>(L.zmax),
                                  ctx->ptr<RsParams>(L.par), nbins, cn);
  LenSrc lrs{&cn->n_rs, 0, 0};
  scan(ctx, rs_cnt, ctx->ptr<int32_t>(L.rs_start), lrs, nullptr, C.nrs());
  scan(ctx, nbins, bin_base, lrs, nullptr, C.nrs());
  GridBuckets* bk = ctx->ptr<GridBuckets>(L.buckets);
  int4* rec_b = ctx->ptr<int4>(L.up);  // the link arrays' space, free until a3
  k_grid_finish_params<<<gR, bc, 0, s>>>(ctx->ptr<RsParams>(L.par), bin_base, ctx->ptr<int32_t>(L.rs_start), cn,
                                         C.bins, bin_cnt, bk);
  k_grid_bucket<<<grid_for(ctx, (C.n + GRID_TILE_PER_THREAD - 1) / GRID_TILE_PER_THREAD, bc), bc, 0, s>>>(
      ctx->ptr<tpc_cluster>(L.in), ctx->ptr<int32_t>(L.rs_in), ctx->ptr<int32_t>(L.rs_start), bk, rec_b, cn);
  k_grid_bin<<<gN, bc, 0, s>>>(rec_b, ctx->ptr<RsParams>(L.par), bin_cnt, ctx->ptr<int32_t>(L.gbin),
                               ctx->ptr<int32_t>(L.slot), cn);
  LenSrc lb{&cn->n_bins, 0, 0};
  scan(ctx, bin_cnt, bin_start, lb, nullptr);
  int4* rec_s = ctx->ptr<int4>(L.tmp);  // the records in (row-sector, bin) order, arrival order in a bin
  // (one record per thread: measured faster for these 16-byte scattered
  // writes than the capped grid)
  k_grid_scatter<<<grid_lin(C.n, bc), bc, 0, s>>>(rec_b, ctx->ptr<int32_t>(L.gbin), ctx->ptr<int32_t>(L.slot), bin_start, rec_s,
                                   cn);
  k_grid_order<<<gN, bc, 0, s>>>(rec_s, ctx->ptr<RsParams>(L.par), bin_start, ctx->ptr<int32_t>(L.perm),
                                 ctx->ptr<float2>(L.yz), ctx->ptr<int32_t>(L.rs_of),
                                 ctx->ptr<int32_t>(L.cluster_track), cn);
  ctx->mark(1);
  // a3 neighbours: a grid-stride grid of 128 blocks per SM, so that blocks
  // that reach dense regions (longer candidate scans) are outnumbered by
  // blocks still to start (10 ms timeframe: 16 blocks per SM 8.17 ms, 24
  // 7.89, 36 7.64, 64 7.41, 128 7.34; one wave of 6 blocks per SM 9.25)
  k_neighbours<<<grid_for(ctx, C.n, NB_THREADS, 128), NB_THREADS, 0, s>>>(ctx->ptr<float2>(L.yz), ctx->ptr<int32_t>(L.rs_of), ctx->ptr<RsParams>(L.par),
                                  bin_start, ctx->kc, ctx->ptr<int32_t>(L.up), ctx->ptr<int32_t>(L.dn),
                                  ctx->ptr<uint8_t>(L.tie), cn);
  if (ctx->cfg.link_skip)
    k_neighbours_skip<<<gN, bc, 0, s>>>(ctx->ptr<float2>(L.yz), ctx->ptr<int32_t>(L.rs_of),
                                        ctx->ptr<RsParams>(L.par), bin_start, ctx->kc, ctx->ptr<int32_t>(L.up),
                                        ctx->ptr<int32_t>(L.dn), ctx->ptr<uint8_t>(L.tie), cn);
  ctx->mark(2);
  // a4 + a5
  // chain starts flagged in k_clean, listed in sorted order; one walk per
  // start; the kept chains compacted in the same order (flag and fidx hold
  // the per-cluster start flags, then the per-start keep flags)
  int32_t* starts = ctx->ptr<int32_t>(L.starts);
  const int gS = grid_for(ctx, C.n / 2 + 1, bc);
  k_clean<<<gN, bc, 0, s>>>(ctx->ptr<int32_t>(L.up), ctx->ptr<int32_t>(L.dn), ctx->ptr<int32_t>(L.up_m),
                            ctx->ptr<int32_t>(L.dn_m), ctx->ptr<int32_t>(L.flag), ctx->ptr<void>(L.owner), key32(ctx),
                            cn);
  scan(ctx, ctx->ptr<int32_t>(L.flag), ctx->ptr<int32_t>(L.fidx), LenSrc{&cn->n32, 0, 0}, &cn->n_starts);
  k_start_list<<<gN, bc, 0, s>>>(ctx->ptr<int32_t>(L.flag), ctx->ptr<int32_t>(L.fidx), starts, cn);
  k_chains<<<gS, bc, 0, s>>>(ctx->ptr<int32_t>(L.up_m), starts, ctx->kc, ctx->ptr<int32_t>(L.flag),
                             ctx->ptr<int32_t>(L.clen), ctx->ptr<int32_t>(L.cend), cn);
  scan(ctx, ctx->ptr<int32_t>(L.flag), ctx->ptr<int32_t>(L.fidx), LenSrc{&cn->n_starts, 0, 0}, nullptr);
  k_tracklet_compact<<<gS, bc, 0, s>>>(ctx->ptr<int32_t>(L.flag), ctx->ptr<int32_t>(L.fidx), starts,
                                       ctx->ptr<int32_t>(L.clen), ctx->ptr<int32_t>(L.cend),
                                       ctx->ptr<int32_t>(L.tl_start), ctx->ptr<int32_t>(L.tl_len),
                                       ctx->ptr<int32_t>(L.tl_end), cn, C.tl);
  ctx->mark(3);
  // a6 follow: per chunk, zone (p1) -> order -> FP32 (p2) -> zone (p3) ->
  // order -> FP32 refit rows (p4r) -> FP32 extension and outputs (p4).  With two chunks the second runs on the auxiliary
  // stream one kernel behind the first, so that one chunk's FP64 zone shares
  // the SMs with the other's FP32 phase.
  {
    FollowWork* W = ctx->ptr<FollowWork>(L.fwork);
    const ZoneTail zt{ctx->ptr<int32_t>(L.ztail_list), ctx->ptr<double>(L.ztail_cov)};
    const int bf = ctx->block_follow;
    const int nc = ctx->prof ? 1 : effective_chunks(ctx);
    // longest first below kLargeBatch clusters, where the longest tracklet
    // bounds the refilling kernels; index order above (order.cuh)
    const bool longest_first = ctx->n < kLargeBatch;
    int32_t* order = longest_first ? ctx->ptr<int32_t>(L.order) : nullptr;
    auto ord = [&](int phase, int c) { return longest_first ? work_order(ctx, phase, c) : WorkOrder{}; };
    auto follow_chunk = [&](cudaStream_t st, int c, cudaEvent_t after_p1) {
      // profiled runs (one chunk) mark the end of every Kalman kernel (a
      // k_order counts with the kernel before it; a kernel the batch's size
      // does not launch gets an empty interval)
      auto mk = [&](int i) {
        if (nc == 1) ctx->mark_k(i);
      };
      auto order_after = [&](int phase) {
        if (longest_first)
          k_order<<<grid_for(ctx, C.tl, bc), bc, 0, st>>>(work_order(ctx, phase, c), &cn->n_tracklets, c, nc, cn);
      };
      const bool tail1 = ctx->kc.zone_steps[0] > 0, tail3 = ctx->kc.zone_steps[1] > 0;
      k_follow_p1<<<persistent_grid(ctx, k_follow_p1, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
          grid_view(ctx), ctx->ptr<int32_t>(L.tl_start), ctx->ptr<int32_t>(L.tl_len), ctx->ptr<int32_t>(L.tl_end),
          ctx->ptr<int32_t>(L.up_m), ctx->kc, follow_out(ctx), W, zt, ord(0, c), c, nc, cn);
      if (!tail1) order_after(0);
      mk(0);
      if (tail1) {
        k_follow_p1t<<<persistent_grid(ctx, k_follow_p1t, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
            grid_view(ctx), ctx->ptr<int32_t>(L.up_m), ctx->kc, W, zt, ord(0, c), c, nc, cn);
        order_after(0);
      }
      if (after_p1) cudaEventRecord(after_p1, st);
      mk(1);
      auto p2 = ctx->n >= kLargeBatch ? k_follow_p2<7> : k_follow_p2<4>;
      p2<<<persistent_grid(ctx, p2, bf, effective_ctas_follow(ctx)), bf, 0, st>>>(
          grid_view(ctx), ctx->ptr<int32_t>(L.up_m), ctx->kc, follow_out(ctx), W, order, c, nc, cn);
      mk(2);
      k_follow_p3<<<persistent_grid(ctx, k_follow_p3, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
          grid_view(ctx), ctx->kc, follow_out(ctx), W, zt, ord(1, c), c, nc, cn);
      if (!tail3) order_after(1);
      mk(3);
      if (tail3) {
        k_follow_p3t<<<persistent_grid(ctx, k_follow_p3t, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
            grid_view(ctx), ctx->kc, follow_out(ctx), W, zt, ord(1, c), c, nc, cn);
        order_after(1);
      }
      mk(4);
      // large batches: the refit rows (p4r) and the extension (p4) in two
      // kernels, so that no warp mixes them; small ones: both in p4
      if (ctx->n >= kLargeBatch)
        k_follow_p4r<7><<<persistent_grid(ctx, k_follow_p4r<7>, bf, effective_ctas_follow(ctx)), bf, 0, st>>>(
            grid_view(ctx), ctx->kc, follow_out(ctx), W, order, c, nc, cn);
      mk(5);
      auto p4 = ctx->n >= kLargeBatch ? k_follow_p4<7, BW_EXTEND> : k_follow_p4<4, BW_ANY>;
      p4<<<persistent_grid(ctx, p4, bf, effective_ctas_follow(ctx)), bf, 0, st>>>(
          grid_view(ctx), ctx->ptr<int32_t>(L.tl_start), ctx->kc, follow_out(ctx), W, order, c, nc, cn);
    };
    if (nc == 1) {
      follow_chunk(s, 0, nullptr);
    } else {
      follow_chunk(s, 0, ctx->ev_chunk[0]);
      cudaStreamWaitEvent(ctx->aux, ctx->ev_chunk[0], 0);
      follow_chunk(ctx->aux, 1, nullptr);
      cudaEventRecord(ctx->ev_chunk[1], ctx->aux);
      cudaStreamWaitEvent(s, ctx->ev_chunk[1], 0);
    }
  }
  ctx->mark(4);
  // a7 selection
  const bool warp_sel = ctx->n < kLargeBatch;  // warp per tracklet while the owner array stays in L2
  if (!warp_sel) gT = grid_lin(C.tl, bc);  // thread per tracklet: one tracklet per thread
  if (key32(ctx)) {
    uint32_t* owner = ctx->ptr<uint32_t>(L.owner);
    (warp_sel ? k_own<true, uint32_t> : k_own<false, uint32_t>)<<<warp_sel ? gTw : gT, bc, 0, s>>>(
        ctx->ptr<int32_t>(L.f_n), ctx->ptr<int32_t>(L.hits), ctx->kc, owner, cn);
    (warp_sel ? k_keep<true, uint32_t> : k_keep<false, uint32_t>)<<<warp_sel ? gTw : gT, bc, 0, s>>>(
                                        ctx->ptr<int32_t>(L.f_n), ctx->ptr<int32_t>(L.hits),
                                        ctx->ptr<uint8_t>(L.hrow), owner, ctx->kc, ctx->ptr<int32_t>(L.keep),
                                        ctx->ptr<int32_t>(L.nown), ctx->ptr<uint32_t>(L.own_mask),
                                        ctx->ptr<int32_t>(L.own_rng), cn);
  } else {
    uint64_t* owner = ctx->ptr<uint64_t>(L.owner);
    (warp_sel ? k_own<true, uint64_t> : k_own<false, uint64_t>)<<<warp_sel ? gTw : gT, bc, 0, s>>>(
        ctx->ptr<int32_t>(L.f_n), ctx->ptr<int32_t>(L.hits), ctx->kc, owner, cn);
    (warp_sel ? k_keep<true, uint64_t> : k_keep<false, uint64_t>)<<<warp_sel ? gTw : gT, bc, 0, s>>>(
                                        ctx->ptr<int32_t>(L.f_n), ctx->ptr<int32_t>(L.hits),
                                        ctx->ptr<uint8_t>(L.hrow), owner, ctx->kc, ctx->ptr<int32_t>(L.keep),
                                        ctx->ptr<int32_t>(L.nown), ctx->ptr<uint32_t>(L.own_mask),
                                        ctx->ptr<int32_t>(L.own_rng), cn);
  }
  scan(ctx, ctx->ptr<int32_t>(L.keep), ctx->ptr<int32_t>(L.tidx), LenSrc{&cn->n_tracklets, 0, 0}, nullptr);
  (warp_sel ? k_assign<true> : k_assign<false>)<<<warp_sel ? gTw : gT, bc, 0, s>>>(ctx->ptr<int32_t>(L.f_n), ctx->ptr<int32_t>(L.hits), ctx->ptr<uint32_t>(L.own_mask),
                             ctx->ptr<int32_t>(L.keep), ctx->ptr<int32_t>(L.tidx), ctx->ptr<int32_t>(L.perm),
                             ctx->ptr<int32_t>(L.nown), ctx->ptr<int32_t>(L.tl_track), ctx->ptr<int32_t>(L.track_tl),
                             ctx->ptr<int32_t>(L.tcount), ctx->ptr<int32_t>(L.cluster_track), cn);
  ctx->mark(5);
}

RefitIn refit_in(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  RefitIn in;
  in.track_tl = ctx->ptr<int32_t>(L.track_tl);
  in.f_n = ctx->ptr<int32_t>(L.f_n);
  in.f_nf = ctx->ptr<int32_t>(L.f_nf);
  in.f_row = ctx->ptr<int32_t>(L.f_row);
  in.hits = ctx->ptr<int32_t>(L.hits);
  in.hrow = ctx->ptr<uint8_t>(L.hrow);
  in.f_par = ctx->ptr<float>(L.f_par);
  in.f_zref = ctx->ptr<float>(L.f_zref);
  in.f_cov = ctx->ptr<float>(L.f_cov);
  in.f_chi2 = ctx->ptr<double>(L.f_chi2);
  in.own_mask = ctx->ptr<uint32_t>(L.own_mask);
  in.own_rng = ctx->ptr<int32_t>(L.own_rng);
  in.nown = ctx->ptr<int32_t>(L.nown);
  in.toff = ctx->ptr<int32_t>(L.toff);
  return in;
}

// a8 on the context's stream.
void enqueue_fit(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  const Caps& C = ctx->caps;
  cudaStream_t s = ctx->stream;
  Counts* cn = ctx->ptr<Counts>(L.counts);
  const int bc = ctx->block_clusters;
  scan(ctx, ctx->ptr<int32_t>(L.tcount), ctx->ptr<int32_t>(L.toff), LenSrc{&cn->n_tracks, 0, 0},
       &cn->n_track_clusters);
  {
    const int bf = ctx->block_follow;
    RefitIn in = refit_in(ctx);
    RefitWork* RW = ctx->ptr<RefitWork>(L.rwork);
    const int nc = ctx->prof ? 1 : effective_chunks(ctx);
    // longest first below kLargeBatch clusters, index order above (as a6)
    const bool longest_first = ctx->n < kLargeBatch;
    auto refit_chunk = [&](cudaStream_t st, int c, cudaEvent_t after_p1) {
      const ZoneTail zt{ctx->ptr<int32_t>(L.ztail_list), ctx->ptr<double>(L.ztail_cov)};
      const WorkOrder o2 = longest_first ? work_order(ctx, 2, c) : WorkOrder{};
      const bool tail = ctx->kc.zone_steps[2] > 0;
      auto order_after = [&]() {
        if (longest_first)
          k_order<<<grid_for(ctx, C.tracks, bc), bc, 0, st>>>(work_order(ctx, 2, c), &cn->n_tracks, c, nc, cn);
      };
      k_refit_p1<<<persistent_grid(ctx, k_refit_p1, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
          grid_view(ctx), in, ctx->kc, RW, zt, o2, c, nc, cn);
      if (!tail) order_after();
      if (nc == 1) ctx->mark_k(7);
      if (tail) {
        k_refit_p1t<<<persistent_grid(ctx, k_refit_p1t, bf, effective_ctas_zone(ctx)), bf, 0, st>>>(
            grid_view(ctx), ctx->kc, RW, zt, o2, c, nc, cn);
        order_after();
      }
      if (after_p1) cudaEventRecord(after_p1, st);
      if (nc == 1) ctx->mark_k(8);
      k_refit_p2<<<persistent_grid(ctx, k_refit_p2, bf, effective_ctas_follow(ctx)), bf, 0, st>>>(
          grid_view(ctx), in, ctx->kc, RW, longest_first ? ctx->ptr<int32_t>(L.order) : nullptr,
          ctx->ptr<tpc_track>(L.tracks), c, nc, cn);
    };
    ctx->mark_k(6);
    if (nc == 1) {
      refit_chunk(s, 0, nullptr);
    } else {
      refit_chunk(s, 0, ctx->ev_chunk[2]);
      cudaStreamWaitEvent(ctx->aux, ctx->ev_chunk[2], 0);
      refit_chunk(ctx->aux, 1, nullptr);
      cudaEventRecord(ctx->ev_chunk[3], ctx->aux);
      cudaStreamWaitEvent(s, ctx->ev_chunk[3], 0);
    }
    ctx->mark_k(9);
  }
  k_track_clusters<<<grid_for(ctx, C.tracks * 32, bc), bc, 0, s>>>(ctx->ptr<int32_t>(L.track_tl), ctx->ptr<int32_t>(L.f_n),
                                     ctx->ptr<int32_t>(L.f_nf), ctx->ptr<int32_t>(L.hits),
                                     ctx->ptr<uint32_t>(L.own_mask), ctx->ptr<int32_t>(L.toff),
                                     ctx->ptr<int32_t>(L.perm), ctx->ptr<int32_t>(L.track_clusters), cn);
  cudaMemcpyAsync(ctx->h_counts, cn, sizeof(Counts), cudaMemcpyDeviceToHost, s);
  ctx->mark(6);
  ctx->prof_valid = ctx->prof;
}

int32_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  int32_t k = 0;
  for (size_t i = 0; i < n; i++) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
  }
  return k;
}

int check_status(tpc_ctx* ctx) {
  uint32_t st = ctx->h_counts->status;
  if (st & ST_EINVAL) return fail(ctx, TPC_EINVAL, "invalid cluster (row >= 159, sector >= 36 or non-finite y/z)");
  if (st & ST_EOVERFLOW)
    return fail(ctx, TPC_EOVERFLOW, "capacity exceeded (grid bins %d of %lld, tracklets %d of %lld); retry after "
                "tpc_reserve with larger capacities",
                ctx->h_counts->n_bins, (long long)ctx->caps.bins, ctx->h_counts->n_tracklets,
                (long long)ctx->caps.tl);
  if (st & ST_ETIMEOUT) return fail(ctx, TPC_ETIMEOUT, "a bounded device wait ran out");
  return TPC_OK;
}

// parts (optional): request q's clusters are copied from parts[q].clusters
// (host memory) instead of from c + off[q].
int load_common(tpc_ctx* ctx, const tpc_cluster* c, const int64_t* off, int32_t n_req, int on_device,
                const tpc_request* parts = nullptr) {
  if (!ctx) return TPC_EINVAL;
  if (ctx->batch_state == BATCH_RUNNING || ctx->batch_state == BATCH_COPYING)
    return fail(ctx, TPC_EBUSY, "a batch submitted with tpc_submit_batch is still in flight");
  if (n_req < 1 || !off || off[0] != 0) return fail(ctx, TPC_EINVAL, "bad request offsets");
  for (int32_t q = 0; q < n_req; q++)
    if (off[q + 1] < off[q]) return fail(ctx, TPC_EINVAL, "request offsets must be non-decreasing");
  int64_t n = off[n_req];
  if (n < 0 || n >= 0x7FFFFFFF / 2) return fail(ctx, TPC_EINVAL, "cluster count %lld out of range", (long long)n);
  if (n > 0 && !c && !parts) return fail(ctx, TPC_EINVAL, "null cluster pointer");
  if ((int64_t)n_req * NSEC * NROW >= 0x7FFFFFFF / 2) return fail(ctx, TPC_EINVAL, "too many requests");
  Caps want = default_caps(n, n_req);
  want.bins = std::max(want.bins, ctx->caps.bins);
  int rc = do_reserve(ctx, want);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  const Layout& L = ctx->L;
  // host-side scalars of the batch: counts struct + request offsets
  memcpy(ctx->h_req, off, sizeof(int64_t) * (n_req + 1));
  Counts hc{};
  hc.n = n;
  hc.n_req = n_req;
  hc.n_rs = n_req * NSEC * NROW;
  hc.n32 = (int32_t)n;
  CK(cudaStreamSynchronize(ctx->stream));  // the pinned staging buffers are reused
  *ctx->h_counts = hc;
  CK(cudaMemcpyAsync(ctx->ptr<Counts>(L.counts), ctx->h_counts, sizeof(Counts), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->ptr<int64_t>(L.req_off), ctx->h_req, sizeof(int64_t) * (n_req + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  if (parts) {
    for (int32_t q = 0; q < n_req; q++)
      if (off[q + 1] > off[q])
        CK(cudaMemcpyAsync(ctx->ptr<tpc_cluster>(L.in) + off[q], parts[q].clusters,
                           sizeof(tpc_cluster) * (off[q + 1] - off[q]), cudaMemcpyHostToDevice, ctx->stream));
  } else if (n > 0) {
    CK(cudaMemcpyAsync(ctx->ptr<tpc_cluster>(L.in), c, sizeof(tpc_cluster) * n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  }
  ctx->n = n;
  ctx->n_req = n_req;
  ctx->loaded = true;
  ctx->found = ctx->fitted = false;
  return TPC_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int tpc_default_config(tpc_config* c) {
  if (!c) return TPC_EINVAL;
  memset(c, 0, sizeof(*c));
  c->bz_kg = 5.0;
  c->sigma = 0.1;
  c->d_max = 1.0f;
  c->min_chain = 3;
  c->max_miss = 5;
  c->n_min_track = 10;
  c->gate = 16.0;
  c->c0[0] = 100.0;
  c->c0[1] = 100.0;
  c->c0[2] = 1.0;
  c->c0[3] = 1.0;
  c->c0[4] = 100.0;
  c->s_max = 0.95;
  c->edge = 2.0;
  c->taint_rel = 1e-4;
  c->fp64_updates = 10;
  c->link_skip = 0;
  return TPC_OK;
}

int tpc_create(tpc_ctx** out, const tpc_config* cfg, int device, void* cuda_stream, size_t hbm_budget) {
  if (cfg && !config_ok(*cfg)) return TPC_EINVAL;
  int rc = create_common(out, cfg, device, cuda_stream);
  if (rc) return rc;
  (*out)->own_arena = true;
  (*out)->budget = hbm_budget;
  return TPC_OK;
}

int tpc_create_with_arena(tpc_ctx** out, const tpc_config* cfg, int device, void* cuda_stream, void* arena,
                          size_t bytes) {
  if (cfg && !config_ok(*cfg)) return TPC_EINVAL;
  if (!arena || ((uintptr_t)arena % ALIGN) != 0) return TPC_EINVAL;
  int rc = create_common(out, cfg, device, cuda_stream);
  if (rc) return rc;
  (*out)->own_arena = false;
  (*out)->arena = (char*)arena;
  (*out)->arena_bytes = bytes;
  return TPC_OK;
}

void tpc_destroy(tpc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->aux) cudaStreamSynchronize(ctx->aux);
  if (ctx->copy) cudaStreamSynchronize(ctx->copy);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  for (int i = 0; i < 7; i++)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int i = 0; i < PH_COUNT; i++)
    if (ctx->evk[i]) cudaEventDestroy(ctx->evk[i]);
  if (ctx->own_arena && ctx->arena) {
    cudaFreeAsync(ctx->arena, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
  }
  if (ctx->h_counts) cudaFreeHost(ctx->h_counts);
  if (ctx->h_req) cudaFreeHost(ctx->h_req);
  if (ctx->h_req_trk) cudaFreeHost(ctx->h_req_trk);
  if (ctx->ev_batch) cudaEventDestroy(ctx->ev_batch);
  if (ctx->vtx_mem) cudaFree(ctx->vtx_mem);
  if (ctx->codec_mem) cudaFree(ctx->codec_mem);
  if (ctx->merge_mem) cudaFree(ctx->merge_mem);
  if (ctx->reject_mem) cudaFree(ctx->reject_mem);
  if (ctx->h_merge_n) cudaFreeHost(ctx->h_merge_n);
  if (ctx->h_vtx_n) cudaFreeHost(ctx->h_vtx_n);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->copy) cudaStreamDestroy(ctx->copy);
  if (ctx->ev_sel) cudaEventDestroy(ctx->ev_sel);
  if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
  for (int i = 0; i < 4; i++)
    if (ctx->ev_chunk[i]) cudaEventDestroy(ctx->ev_chunk[i]);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* tpc_last_error(tpc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t tpc_arena_bytes(int64_t n_clusters, int32_t n_requests) {
  return make_layout(default_caps(n_clusters, n_requests)).total;
}

size_t tpc_arena_bytes_for(int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets) {
  Caps c = default_caps(n_clusters, n_requests);
  if (n_bins > 0) c.bins = std::max(c.bins, n_bins);
  if (n_tracklets > 0) c.tl = std::max(c.tl, n_tracklets);
  c.tracks = std::max(c.tracks, c.tl);
  return make_layout(c).total;
}

namespace {
Caps reserve_caps(const tpc_ctx* ctx, int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets) {
  Caps want = default_caps(std::max<int64_t>(n_clusters, ctx->caps.n), std::max(n_requests, ctx->caps.req));
  if (n_bins) want.bins = n_bins;
  if (n_tracklets) want.tl = n_tracklets;
  want.tracks = std::max(want.tracks, want.tl);
  return want;
}
}  // namespace

int tpc_reserve(tpc_ctx* ctx, int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets) {
  if (!ctx || n_clusters < 0 || n_requests < 0 || n_bins < 0 || n_tracklets < 0) return TPC_EINVAL;
  return do_reserve(ctx, reserve_caps(ctx, n_clusters, n_requests, n_bins, n_tracklets));
}

int tpc_reserve_bytes(tpc_ctx* ctx, int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets,
                      size_t* bytes) {
  if (!ctx || !bytes || n_clusters < 0 || n_requests < 0 || n_bins < 0 || n_tracklets < 0) return TPC_EINVAL;
  const Caps want = reserve_caps(ctx, n_clusters, n_requests, n_bins, n_tracklets);
  const Caps& c = ctx->caps;
  const bool grow = want.n > c.n || want.req > c.req || want.bins > c.bins || want.tl > c.tl ||
                    want.tracks > c.tracks || ctx->arena == nullptr;
  if (!grow) {
    *bytes = ctx->arena_bytes;
    return TPC_OK;
  }
  Caps m = c;  // do_reserve takes the larger of the current and the wanted capacity
  m.n = std::max(c.n, want.n);
  m.req = std::max(c.req, want.req);
  m.bins = std::max(c.bins, want.bins);
  m.tl = std::max(c.tl, want.tl);
  m.tracks = std::max(c.tracks, want.tracks);
  *bytes = make_layout(m).total;
  return TPC_OK;
}

int tpc_load_clusters(tpc_ctx* ctx, const tpc_cluster* c, int64_t n, int on_device) {
  int64_t off[2] = {0, n};
  return load_common(ctx, c, off, 1, on_device);
}

int tpc_load_batch(tpc_ctx* ctx, const tpc_cluster* c, const int64_t* req_offsets, int32_t n_req, int on_device) {
  return load_common(ctx, c, req_offsets, n_req, on_device);
}

int tpc_find_tracks(tpc_ctx* ctx) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "no clusters loaded");
  CK(cudaSetDevice(ctx->device));
  enqueue_find(ctx);
  CK(cudaGetLastError());
  ctx->found = true;
  return TPC_OK;
}

int tpc_fit_tracks(tpc_ctx* ctx) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->found) return fail(ctx, TPC_EINVAL, "tpc_find_tracks has not run on the loaded clusters");
  CK(cudaSetDevice(ctx->device));
  enqueue_fit(ctx);
  CK(cudaGetLastError());
  ctx->fitted = true;
  ctx->fit_gen++;
  return TPC_OK;
}

int tpc_run_graph(tpc_ctx* ctx) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "no clusters loaded");
  CK(cudaSetDevice(ctx->device));
  if (ctx->graph && (ctx->graph_chunks != effective_chunks(ctx) || ctx->graph_ctas != effective_ctas_follow(ctx) ||
                     ctx->graph_class != size_class(ctx->n))) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (!ctx->graph) {
    if (!ctx->own_stream && ctx->stream == nullptr)
      return fail(ctx, TPC_EINVAL, "graph capture needs a non-default stream");
    cudaGraph_t g = nullptr;
    const bool prof = ctx->prof;
    ctx->prof = false;  // no event nodes in the graph
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_find(ctx);
    enqueue_fit(ctx);
    ctx->prof = prof;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return fail(ctx, TPC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    ctx->graph_kernels = count_kernel_nodes(g);
    ctx->graph_chunks = effective_chunks(ctx);
    ctx->graph_ctas = effective_ctas_follow(ctx);
    ctx->graph_class = size_class(ctx->n);
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      return fail(ctx, TPC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  CK(cudaGraphLaunch(ctx->graph, ctx->stream));
  ctx->found = ctx->fitted = true;
  ctx->fit_gen++;
  return TPC_OK;
}

int tpc_sync(tpc_ctx* ctx) {
  if (!ctx) return TPC_EINVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (!ctx->fitted && ctx->found) {
    CK(cudaMemcpy(ctx->h_counts, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
  }
  return check_status(ctx);
}

int tpc_get_tracks(tpc_ctx* ctx, tpc_track* out, int64_t cap, int64_t* n_out, int32_t* cluster_track,
                   int32_t* track_clusters) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  const Counts& hc = *ctx->h_counts;
  if (n_out) *n_out = hc.n_tracks;
  if (hc.n_tracks > cap) return fail(ctx, TPC_EOVERFLOW, "%d tracks do not fit cap %lld", hc.n_tracks, (long long)cap);
  const Layout& L = ctx->L;
  if (out && hc.n_tracks)
    CK(cudaMemcpyAsync(out, ctx->ptr<tpc_track>(L.tracks), sizeof(tpc_track) * hc.n_tracks, cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (cluster_track && ctx->n)
    CK(cudaMemcpyAsync(cluster_track, ctx->ptr<int32_t>(L.cluster_track), sizeof(int32_t) * ctx->n,
                       cudaMemcpyDeviceToHost, ctx->stream));
  if (track_clusters && hc.n_track_clusters)
    CK(cudaMemcpyAsync(track_clusters, ctx->ptr<int32_t>(L.track_clusters), sizeof(int32_t) * hc.n_track_clusters,
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return TPC_OK;
}

int tpc_get_arena_bytes(tpc_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return TPC_EINVAL;
  *bytes = ctx->arena ? ctx->arena_bytes : 0;
  return TPC_OK;
}

int tpc_track_host(tpc_ctx* ctx, const tpc_cluster* clusters, int64_t n, tpc_track* out, int64_t cap,
                   int64_t* n_out, int32_t* cluster_track) {
  if (!ctx) return TPC_EINVAL;
  int rc = tpc_load_clusters(ctx, clusters, n, 0);
  if (rc) return rc;
  const bool graph_ok = ctx->own_stream || ctx->stream != nullptr;
  if (ctx->n < kLargeBatch && graph_ok) {
    // below kLargeBatch clusters a2-a8 run as the captured graph (one launch
    // for some 45 kernels that each take tens of microseconds here), and both
    // copies follow: a fork and join around the assignment's copy costs more
    // than the copy it would hide (central event: graph 2.64 ms host to host,
    // plain launches 2.75, plain launches with the overlapped copy 2.83)
    rc = tpc_run_graph(ctx);
    if (rc) return rc;
    return tpc_get_tracks(ctx, out, cap, n_out, cluster_track, nullptr);
  }
  if (!ctx->copy) {
    if (cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_sel, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming) != cudaSuccess)
      return fail(ctx, TPC_ECUDA, "copy stream: %s", cudaGetErrorString(cudaGetLastError()));
  }
  enqueue_find(ctx);
  CK(cudaGetLastError());
  ctx->found = true;
  // the assignment is final once a7 has run: its copy runs on the copy
  // stream while a8 runs on the context's stream (10 ms timeframe: 8.5e8 ->
  // 9.0e8 clusters/s host to host)
  const bool ct = cluster_track && ctx->n > 0;
  if (ct) {
    CK(cudaEventRecord(ctx->ev_sel, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy, ctx->ev_sel, 0));
    CK(cudaMemcpyAsync(cluster_track, ctx->ptr<int32_t>(ctx->L.cluster_track), sizeof(int32_t) * ctx->n,
                       cudaMemcpyDeviceToHost, ctx->copy));
    CK(cudaEventRecord(ctx->ev_copied, ctx->copy));
  }
  enqueue_fit(ctx);
  CK(cudaGetLastError());
  ctx->fitted = true;
  ctx->fit_gen++;
  if (ct) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied, 0));  // later work on the stream waits for the copy
  return tpc_get_tracks(ctx, out, cap, n_out, nullptr, nullptr);
}

int tpc_get_tracks_async(tpc_ctx* ctx, tpc_track* out, int64_t cap, int64_t* n_out, int32_t* cluster_track) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  CK(cudaSetDevice(ctx->device));
  const cudaError_t q = cudaStreamQuery(ctx->stream);
  if (q == cudaErrorNotReady) return fail(ctx, TPC_EBUSY, "the run has not completed");
  if (q != cudaSuccess) return fail(ctx, TPC_ECUDA, "stream: %s", cudaGetErrorString(q));
  int rc = check_status(ctx);
  if (rc) return rc;
  const Counts& hc = *ctx->h_counts;
  if (n_out) *n_out = hc.n_tracks;
  if (hc.n_tracks > cap) return fail(ctx, TPC_EOVERFLOW, "%d tracks do not fit cap %lld", hc.n_tracks, (long long)cap);
  const Layout& L = ctx->L;
  if (out && hc.n_tracks)
    CK(cudaMemcpyAsync(out, ctx->ptr<tpc_track>(L.tracks), sizeof(tpc_track) * hc.n_tracks, cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (cluster_track && ctx->n)
    CK(cudaMemcpyAsync(cluster_track, ctx->ptr<int32_t>(L.cluster_track), sizeof(int32_t) * ctx->n,
                       cudaMemcpyDeviceToHost, ctx->stream));
  return TPC_OK;
}

// ---------------------------------------------- batched requests (a1-a9)
namespace {

// After the batch's graph: each request's track range and request-local
// cluster->track indices (into the grid stage's dead per-cluster scratch),
// the ranges copied to the host, and the completion event.
int enqueue_batch_views(tpc_ctx* ctx) {
  const Layout& L = ctx->L;
  cudaStream_t s = ctx->stream;
  Counts* cn = ctx->ptr<Counts>(L.counts);
  const int bc = ctx->block_clusters;
  CK(cudaMemsetAsync(ctx->ptr<int32_t>(L.req_trk), 0, sizeof(int32_t) * 2 * ctx->n_req, s));
  k_req_tracks<<<grid_for(ctx, ctx->caps.tracks, bc), bc, 0, s>>>(ctx->ptr<tpc_track>(L.tracks),
                                                                  ctx->ptr<int32_t>(L.req_trk), cn);
  k_req_rebase<<<grid_for(ctx, std::max<int64_t>(ctx->n, 1), bc), bc, 0, s>>>(
      ctx->ptr<int32_t>(L.cluster_track), ctx->ptr<int64_t>(L.req_off), ctx->ptr<int32_t>(L.req_trk),
      ctx->ptr<int32_t>(L.slot), cn);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_req_trk, ctx->ptr<int32_t>(L.req_trk), sizeof(int32_t) * 2 * ctx->n_req,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev_batch, s));
  return TPC_OK;
}

int launch_batch(tpc_ctx* ctx) {
  const int32_t nq = (int32_t)ctx->batch.size();
  std::vector<int64_t> off(nq + 1, 0);
  std::vector<tpc_request> parts(nq);
  for (int32_t q = 0; q < nq; q++) {
    parts[q] = ctx->batch[q].r;
    off[q + 1] = off[q] + parts[q].n;
  }
  int rc = load_common(ctx, nullptr, off.data(), nq, 0, parts.data());
  if (rc == TPC_OK) rc = tpc_run_graph(ctx);
  if (rc == TPC_OK) rc = enqueue_batch_views(ctx);
  return rc;
}

// Marks every request done; rc is the outcome of those that have no error
// of their own (a request whose cap was too small keeps TPC_EOVERFLOW).
void finish_batch(tpc_ctx* ctx, int rc) {
  for (auto& b : ctx->batch) {
    if (!b.done && b.rc == TPC_OK) b.rc = rc;
    b.done = true;
  }
  ctx->batch_state = BATCH_DONE;
}

// Moves the submitted batch on without waiting: once its graph has run,
// enqueues each request's result copies; once those have landed, marks the
// requests done.  A capacity overflow reruns the batch once with the
// worst-case tracklet capacity.
void advance_batch(tpc_ctx* ctx) {
  if (ctx->batch_state != BATCH_RUNNING && ctx->batch_state != BATCH_COPYING) return;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return finish_batch(ctx, TPC_ECUDA);
  const cudaError_t q = cudaEventQuery(ctx->ev_batch);
  if (q == cudaErrorNotReady) return;
  if (q != cudaSuccess) {
    fail(ctx, TPC_ECUDA, "batch: %s", cudaGetErrorString(q));
    return finish_batch(ctx, TPC_ECUDA);
  }
  if (ctx->batch_state == BATCH_COPYING) return finish_batch(ctx, TPC_OK);
  int rc = check_status(ctx);
  if (rc == TPC_EOVERFLOW && !ctx->batch_retried) {
    ctx->batch_retried = true;
    ctx->batch_state = BATCH_NONE;  // lets load_common run
    const Counts& hc = *ctx->h_counts;
    rc = tpc_reserve(ctx, ctx->n, ctx->n_req, 2 * (int64_t)hc.n_bins, ctx->n / 3 + 16);
    if (rc == TPC_OK) rc = launch_batch(ctx);
    if (rc != TPC_OK) return finish_batch(ctx, rc);
    ctx->batch_state = BATCH_RUNNING;
    return;
  }
  if (rc != TPC_OK) return finish_batch(ctx, rc);
  const Layout& L = ctx->L;
  for (int32_t k = 0; k < (int32_t)ctx->batch.size(); k++) {
    auto& b = ctx->batch[k];
    const int32_t first = ctx->h_req_trk[2 * k], cnt = ctx->h_req_trk[2 * k + 1] - first;
    if (b.r.n_tracks) *b.r.n_tracks = cnt;
    if (cnt > b.r.cap) {
      b.rc = fail(ctx, TPC_EOVERFLOW, "request %lld: %d tracks do not fit cap %lld", (long long)b.r.id, cnt,
                  (long long)b.r.cap);
      continue;
    }
    cudaError_t e = cudaSuccess;
    if (cnt > 0)
      e = cudaMemcpyAsync(b.r.tracks_out, ctx->ptr<tpc_track>(L.tracks) + first, sizeof(tpc_track) * cnt,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && b.r.cluster_track_out && b.r.n > 0)
      e = cudaMemcpyAsync(b.r.cluster_track_out, ctx->ptr<int32_t>(L.slot) + b.off, sizeof(int32_t) * b.r.n,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) {
      fail(ctx, TPC_ECUDA, "batch copy: %s", cudaGetErrorString(e));
      return finish_batch(ctx, TPC_ECUDA);
    }
  }
  if (cudaEventRecord(ctx->ev_batch, ctx->stream) != cudaSuccess) return finish_batch(ctx, TPC_ECUDA);
  ctx->batch_state = BATCH_COPYING;
}

}  // namespace

int tpc_submit_batch(tpc_ctx* ctx, const tpc_request* reqs, int32_t n) {
  if (!ctx) return TPC_EINVAL;
  if (ctx->batch_state == BATCH_RUNNING || ctx->batch_state == BATCH_COPYING) {
    advance_batch(ctx);
    if (ctx->batch_state != BATCH_DONE) return fail(ctx, TPC_EBUSY, "the previous batch is still in flight");
  }
  if (n < 1 || !reqs) return fail(ctx, TPC_EINVAL, "empty batch");
  int64_t total = 0;
  for (int32_t q = 0; q < n; q++) {
    const tpc_request& r = reqs[q];
    if (r.n < 0 || (r.n > 0 && !r.clusters) || r.cap < 0 || (r.cap > 0 && !r.tracks_out))
      return fail(ctx, TPC_EINVAL, "request %d: bad sizes or null buffers", q);
    for (int32_t k = 0; k < q; k++)
      if (reqs[k].id == r.id) return fail(ctx, TPC_EINVAL, "request id %lld appears twice", (long long)r.id);
    total += r.n;
  }
  if (total >= 0x7FFFFFFF / 2) return fail(ctx, TPC_EINVAL, "cluster count %lld out of range", (long long)total);
  CK(cudaSetDevice(ctx->device));
  if (!ctx->ev_batch) CK(cudaEventCreateWithFlags(&ctx->ev_batch, cudaEventDisableTiming));
  ctx->batch.assign(n, tpc_ctx::BatchReq{});
  int64_t off = 0;
  for (int32_t q = 0; q < n; q++) {
    ctx->batch[q].r = reqs[q];
    ctx->batch[q].off = off;
    off += reqs[q].n;
  }
  ctx->batch_state = BATCH_NONE;
  ctx->batch_retried = false;
  const int rc = launch_batch(ctx);
  if (rc != TPC_OK) {
    ctx->batch.clear();
    return rc;
  }
  ctx->batch_state = BATCH_RUNNING;
  return TPC_OK;
}

int tpc_poll(tpc_ctx* ctx, int64_t request_id, int* done) {
  if (!ctx || !done) return TPC_EINVAL;
  int32_t k = -1;
  for (int32_t q = 0; q < (int32_t)ctx->batch.size(); q++)
    if (ctx->batch[q].r.id == request_id) k = q;
  if (k < 0) return fail(ctx, TPC_EINVAL, "unknown request id %lld", (long long)request_id);
  advance_batch(ctx);
  *done = ctx->batch[k].done ? 1 : 0;
  return *done ? ctx->batch[k].rc : TPC_OK;
}

int tpc_get_counts(tpc_ctx* ctx, int64_t counts[8]) {
  if (!ctx || !counts) return TPC_EINVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  Counts hc{};
  if (ctx->loaded) CK(cudaMemcpy(&hc, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
  counts[0] = hc.n;
  counts[1] = hc.n_req;
  counts[2] = hc.n_rs;
  counts[3] = hc.n_bins;
  counts[4] = hc.n_tracklets;
  counts[5] = hc.n_tracks;
  counts[6] = hc.status;
  counts[7] = hc.n_track_clusters;
  return TPC_OK;
}

int tpc_get_stage(tpc_ctx* ctx, int item, void* host_out, int64_t cap_bytes, int64_t* n_bytes) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "nothing loaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  Counts hc{};
  CK(cudaMemcpy(&hc, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
  const Layout& L = ctx->L;
  const int64_t n = hc.n, nrs = hc.n_rs, T = hc.n_tracklets;
  size_t off = 0;
  int64_t bytes = 0;
  switch (item) {
    case TPC_ITEM_PERM: off = L.perm; bytes = 4 * n; break;
    case TPC_ITEM_RS_OF: off = L.rs_of; bytes = 4 * n; break;
    case TPC_ITEM_ROW_START: off = L.rs_start; bytes = 4 * (nrs + 1); break;
    case TPC_ITEM_RS_PARAMS: off = L.par; bytes = (int64_t)sizeof(RsParams) * nrs; break;
    case TPC_ITEM_BIN_START: off = L.bin_start; bytes = 4 * ((int64_t)hc.n_bins + 1); break;
    case TPC_ITEM_UP: off = L.up; bytes = 4 * n; break;
    case TPC_ITEM_DN: off = L.dn; bytes = 4 * n; break;
    case TPC_ITEM_TIE: off = L.tie; bytes = n; break;
    case TPC_ITEM_UP_M: off = L.up_m; bytes = 4 * n; break;
    case TPC_ITEM_DN_M: off = L.dn_m; bytes = 4 * n; break;
    case TPC_ITEM_TL_START: off = L.tl_start; bytes = 4 * T; break;
    case TPC_ITEM_TL_LEN: off = L.tl_len; bytes = 4 * T; break;
    case TPC_ITEM_F_N: off = L.f_n; bytes = 4 * T; break;
    case TPC_ITEM_F_NF: off = L.f_nf; bytes = 4 * T; break;
    case TPC_ITEM_F_NB: off = L.f_nb; bytes = 4 * T; break;
    case TPC_ITEM_F_FLAGS: off = L.f_flags; bytes = 4 * T; break;
    case TPC_ITEM_F_ROW: off = L.f_row; bytes = 4 * T; break;
    case TPC_ITEM_F_HITS: off = L.hits; bytes = 4 * T * NROW; break;
    case TPC_ITEM_F_PAR: off = L.f_par; bytes = 4 * 5 * T; break;
    case TPC_ITEM_F_COV: off = L.f_cov; bytes = 4 * 15 * T; break;
    case TPC_ITEM_F_CHI2: off = L.f_chi2; bytes = 8 * T; break;
    case TPC_ITEM_OWNER: off = L.owner; bytes = 8 * n; break;
    case TPC_ITEM_TL_TRACK: off = L.tl_track; bytes = 4 * T; break;
    case TPC_ITEM_SY:
    case TPC_ITEM_SZ: off = L.yz; bytes = 4 * n; break;
    default: return fail(ctx, TPC_EINVAL, "unknown item %d", item);
  }
  if (n_bytes) *n_bytes = bytes;
  if (!host_out) return TPC_OK;
  if (bytes > cap_bytes) return fail(ctx, TPC_EOVERFLOW, "item needs %lld bytes", (long long)bytes);
  if (bytes == 0) return TPC_OK;
  if (item == TPC_ITEM_SY || item == TPC_ITEM_SZ) {
    std::vector<float> tmp(2 * n);
    CK(cudaMemcpy(tmp.data(), ctx->arena + off, 8 * n, cudaMemcpyDeviceToHost));
    float* o = (float*)host_out;
    for (int64_t i = 0; i < n; i++) o[i] = tmp[2 * i + (item == TPC_ITEM_SZ)];
    return TPC_OK;
  }
  if (item == TPC_ITEM_F_PAR) {
    // z is kept relative to the per-tracklet reference on the device
    std::vector<float> zr(T);
    CK(cudaMemcpy(host_out, ctx->arena + off, bytes, cudaMemcpyDeviceToHost));
    if (T) CK(cudaMemcpy(zr.data(), ctx->arena + L.f_zref, 4 * T, cudaMemcpyDeviceToHost));
    float* o = (float*)host_out;
    for (int64_t t = 0; t < T; t++) o[5 * t + 1] += zr[t];
    return TPC_OK;
  }
  if (item == TPC_ITEM_OWNER && key32(ctx)) {
    // 32-bit keys n << 24 | (2^24 - 1 - t), reported in the 64-bit form
    // n << 32 | (2^32 - 1 - t); 0 (no owner) stays 0
    std::vector<uint32_t> k32(n);
    CK(cudaMemcpy(k32.data(), ctx->arena + off, 4 * n, cudaMemcpyDeviceToHost));
    uint64_t* o = (uint64_t*)host_out;
    for (int64_t i = 0; i < n; i++) {
      const uint32_t k = k32[i];
      const uint64_t t = 0xFFFFFFu - (k & 0xFFFFFFu);
      o[i] = k ? ((uint64_t)(k >> 24) << 32) | (0xFFFFFFFFull - t) : 0ull;
    }
    return TPC_OK;
  }
  CK(cudaMemcpy(host_out, ctx->arena + off, bytes, cudaMemcpyDeviceToHost));
  return TPC_OK;
}

namespace {
void get_tuning(const tpc_ctx* ctx, tpc_tuning* t) {
  t->block_clusters = ctx->block_clusters;
  t->block_follow = ctx->block_follow;
  t->ctas_per_sm_zone = ctx->ctas_zone;
  t->ctas_per_sm_follow = ctx->ctas_follow;
  t->refill = ctx->refill;
  t->chunks = ctx->chunks;
  t->zone_rows = ctx->zone_rows;
}
void apply_tuning(tpc_ctx* ctx, const tpc_tuning* t) {
  if (t->block_clusters > 0) ctx->block_clusters = t->block_clusters;
  if (t->block_follow > 0) ctx->block_follow = t->block_follow;
  if (t->ctas_per_sm_zone > 0) ctx->ctas_zone = t->ctas_per_sm_zone;
  if (t->ctas_per_sm_follow > 0) ctx->ctas_follow = t->ctas_per_sm_follow;
  if (t->refill > 0) ctx->refill = ctx->kc.refill = t->refill;
  if (t->chunks > 0) ctx->chunks = t->chunks;
  if (t->zone_rows > 0) ctx->zone_rows = t->zone_rows;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
}
}  // namespace

int tpc_autotune(tpc_ctx* ctx, int32_t reps, tpc_tuning* best_out, float* best_ms) {
  if (!ctx || reps < 1 || reps > 100) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "load a representative batch before tpc_autotune");
  CK(cudaSetDevice(ctx->device));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->prof;
  ctx->prof = false;
  // median device time of `reps` find + fit runs on the loaded batch
  auto measure = [&](float& ms) -> int {
    std::vector<float> t;
    for (int r = 0; r < reps + 1; r++) {
      CK(cudaEventRecord(e0, ctx->stream));
      enqueue_find(ctx);
      enqueue_fit(ctx);
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float v = 0.0f;
      CK(cudaEventElapsedTime(&v, e0, e1));
      if (r > 0) t.push_back(v);  // the first run warms caches and code
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return check_status(ctx);
  };
  // candidates per field, in the order of tpc_tuning
  static const int kCand[6][4] = {{128, 256, 512, 0}, {64, 96, 128, 0}, {2, 3, 4, 0},
                                  {2, 3, 64, 0},      {1, 4, 8, 16},    {1, 2, 0, 0}};
  static const int kNCand[6] = {3, 3, 3, 3, 4, 2};
  tpc_tuning cur;
  get_tuning(ctx, &cur);
  if (cur.chunks <= 0) cur.chunks = effective_chunks(ctx);
  if (cur.ctas_per_sm_zone <= 0) cur.ctas_per_sm_zone = effective_ctas_zone(ctx);
  if (cur.ctas_per_sm_follow <= 0) cur.ctas_per_sm_follow = effective_ctas_follow(ctx);
  int best[6] = {cur.block_clusters, cur.block_follow, cur.ctas_per_sm_zone, cur.ctas_per_sm_follow, cur.refill,
                 cur.chunks};
  auto as_tuning = [&cur](const int* v) {
    tpc_tuning t = cur;  // fields the autotuner does not vary keep their values
    t.block_clusters = v[0];
    t.block_follow = v[1];
    t.ctas_per_sm_zone = v[2];
    t.ctas_per_sm_follow = v[3];
    t.refill = v[4];
    t.chunks = v[5];
    return t;
  };
  float best_t = 0.0f;
  int rc = measure(best_t);
  for (int dim = 0; dim < 6 && rc == TPC_OK; dim++) {  // coordinate descent
    for (int k = 0; k < kNCand[dim] && rc == TPC_OK; k++) {
      int trial[6];
      for (int i = 0; i < 6; i++) trial[i] = best[i];
      trial[dim] = kCand[dim][k];
      if (trial[dim] == best[dim]) continue;
      const tpc_tuning t = as_tuning(trial);
      apply_tuning(ctx, &t);
      float ms = 0.0f;
      rc = measure(ms);
      if (rc == TPC_OK && ms < best_t) {
        best_t = ms;
        best[dim] = trial[dim];
      }
    }
  }
  const tpc_tuning bt = as_tuning(best);
  apply_tuning(ctx, &bt);
  ctx->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_out) *best_out = bt;
  if (best_ms) *best_ms = best_t;
  return rc;
}

int tpc_set_trace(tpc_ctx* ctx, int32_t tracklet) {
  if (!ctx) return TPC_EINVAL;
  ctx->trace_t = tracklet < 0 ? -1 : tracklet;
  ctx->kc.trace_t = ctx->trace_t;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return TPC_OK;
}

int tpc_get_trace(tpc_ctx* ctx, float* out, int32_t cap_records, int32_t* n_records) {
  if (!ctx || cap_records < 0) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "nothing loaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  Counts hc{};
  CK(cudaMemcpy(&hc, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
  if (n_records) *n_records = hc.trace_n;
  const int32_t n = std::min(std::min(hc.trace_n, (int32_t)TRACE_RECORDS), cap_records);
  if (out && n > 0)
    CK(cudaMemcpy(out, ctx->ptr<float>(ctx->L.trace), sizeof(float) * TRACE_W * n, cudaMemcpyDeviceToHost));
  return TPC_OK;
}

int tpc_set_profiling(tpc_ctx* ctx, int on) {
  if (!ctx) return TPC_EINVAL;
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->ev[0]) {
    for (int i = 0; i < 7; i++) CK(cudaEventCreate(&ctx->ev[i]));
    for (int i = 0; i < PH_COUNT; i++) CK(cudaEventCreate(&ctx->evk[i]));
  }
  ctx->prof = on != 0;
  ctx->prof_valid = false;
  return TPC_OK;
}

int tpc_get_stage_times(tpc_ctx* ctx, float ms[6]) {
  if (!ctx || !ms) return TPC_EINVAL;
  if (!ctx->prof_valid) return fail(ctx, TPC_EINVAL, "no profiled run (tpc_set_profiling, then find + fit)");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 6; i++) CK(cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
  return TPC_OK;
}

int tpc_get_kalman_profile(tpc_ctx* ctx, float ms[TPC_KALMAN_KERNELS], uint64_t work[5 * TPC_KALMAN_KERNELS]) {
  static_assert(TPC_KALMAN_KERNELS == PH_COUNT, "the header's kernel count");
  if (!ctx || (!ms && !work)) return TPC_EINVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ms) {
    if (!ctx->prof_valid) return fail(ctx, TPC_EINVAL, "no profiled run (tpc_set_profiling, then find + fit)");
    const cudaEvent_t* k = ctx->evk;
    const cudaEvent_t b[PH_COUNT] = {ctx->ev[3], k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], k[8]};
    const cudaEvent_t e[PH_COUNT] = {k[0], k[1], k[2], k[3], k[4], k[5], ctx->ev[4], k[7], k[8], k[9]};
    for (int i = 0; i < PH_COUNT; i++) CK(cudaEventElapsedTime(&ms[i], b[i], e[i]));
  }
  if (work) {
    if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "nothing loaded");
    Counts hc{};
    CK(cudaMemcpy(&hc, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
    for (int k = 0; k < PH_COUNT; k++)
      for (int j = 0; j < 5; j++) work[5 * k + j] = hc.phase_work[k][j];
  }
  return TPC_OK;
}

int tpc_graph_kernels(tpc_ctx* ctx, int32_t* n) {
  if (!ctx || !n) return TPC_EINVAL;
  if (!ctx->graph) return fail(ctx, TPC_EINVAL, "no graph captured yet (tpc_run_graph)");
  *n = ctx->graph_kernels;
  return TPC_OK;
}

int tpc_get_work(tpc_ctx* ctx, uint64_t work[5]) {
  if (!ctx || !work) return TPC_EINVAL;
  if (!ctx->loaded) return fail(ctx, TPC_EINVAL, "nothing loaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  Counts hc{};
  CK(cudaMemcpy(&hc, ctx->ptr<Counts>(ctx->L.counts), sizeof(Counts), cudaMemcpyDeviceToHost));
  work[0] = hc.n_prop;
  work[1] = hc.n_upd32;
  work[2] = hc.n_upd64;
  work[3] = hc.n_cand;
  work[4] = hc.n_prop64;
  return TPC_OK;
}

int tpc_get_tuning(tpc_ctx* ctx, tpc_tuning* t) {
  if (!ctx || !t) return TPC_EINVAL;
  get_tuning(ctx, t);
  return TPC_OK;
}

int tpc_set_tuning(tpc_ctx* ctx, const tpc_tuning* t) {
  if (!ctx || !t) return TPC_EINVAL;
  if (t->block_clusters > 0 && (t->block_clusters < 32 || t->block_clusters > 1024 || t->block_clusters % 32))
    return fail(ctx, TPC_EINVAL, "block_clusters must be a multiple of 32 in [32, 1024]");
  if (t->block_follow > 0 && (t->block_follow < 32 || t->block_follow > 128 || t->block_follow % 32))
    return fail(ctx, TPC_EINVAL, "block_follow must be a multiple of 32 in [32, 128]");
  if (t->ctas_per_sm_zone > 64 || t->ctas_per_sm_follow > 64) return fail(ctx, TPC_EINVAL, "ctas_per_sm above 64");
  if (t->refill > 32) return fail(ctx, TPC_EINVAL, "refill must be in [1, 32]");
  if (t->chunks > MAX_CHUNKS) return fail(ctx, TPC_EINVAL, "chunks must be 1 or 2");
  apply_tuning(ctx, t);
  return TPC_OK;
}

int tpc_default_vertex_config(tpc_vertex_config* c) {
  if (!c) return TPC_EINVAL;
  c->vdrift_cm_us = 2.5;
  c->zmax_cm = 250.0;
  c->dca_max_cm = 2.0;
  c->ext_max_cm = 300.0;
  c->gap_us = 0.5;
  c->min_tracks = 3;
  c->min_clusters = 20;
  c->min_pt_gev = 0.0;
  return TPC_OK;
}

namespace {
constexpr int32_t kVtxBins = 1 << 18;  // 65 ms of time range at 0.25 us bins

int vtx_reserve(tpc_ctx* ctx) {
  const int64_t M = std::max<int64_t>(ctx->caps.tracks, 1);
  if (ctx->vtx_mem && ctx->vtx_tracks_cap >= M) return TPC_OK;
  if (ctx->vtx_mem) {
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->vtx_mem);
    ctx->vtx_mem = nullptr;
  }
  const size_t B = kVtxBins;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t o_t = take(4 * M), o_use = take(M), o_vx = take(4 * M), o_z = take(4 * M), o_tgl = take(4 * M);
  const size_t o_bc = take(4 * B), o_bmin = take(4 * B), o_bmax = take(4 * B), o_bvid = take(4 * B);
  const size_t o_vc = take(4 * B), o_vs = take(8 * B), o_vk = take(4 * (B + 1)), o_vi = take(4 * (B + 1));
  const size_t o_rng = take(8), o_n = take(16), o_time = take(8 * B), o_ntr = take(4 * B);
  void* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TPC_ENOMEM, "vertex buffers of %zu bytes", off);
  }
  char* b = (char*)mem;
  ctx->vtx_mem = mem;
  ctx->vtx_tracks_cap = M;
  VtxBuf& v = ctx->vb;
  v.t = (float*)(b + o_t);
  v.use = (uint8_t*)(b + o_use);
  v.vertex = (int32_t*)(b + o_vx);
  v.z = (float*)(b + o_z);
  v.tgl = (float*)(b + o_tgl);
  v.b_cnt = (int32_t*)(b + o_bc);
  v.b_min = (uint32_t*)(b + o_bmin);
  v.b_max = (uint32_t*)(b + o_bmax);
  v.b_vid = (int32_t*)(b + o_bvid);
  v.v_cnt = (int32_t*)(b + o_vc);
  v.v_sum = (unsigned long long*)(b + o_vs);
  v.v_keep = (int32_t*)(b + o_vk);
  v.v_idx = (int32_t*)(b + o_vi);
  v.range = (uint32_t*)(b + o_rng);
  v.n = (int32_t*)(b + o_n);
  ctx->vtx_time = (double*)(b + o_time);
  ctx->vtx_ntr = (int32_t*)(b + o_ntr);
  if (!ctx->h_vtx_n && cudaMallocHost(&ctx->h_vtx_n, 16) != cudaSuccess) return fail(ctx, TPC_ECUDA, "pinned buffer");
  return TPC_OK;
}
}  // namespace

int tpc_find_vertices(tpc_ctx* ctx, const tpc_vertex_config* cfg_in) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  if (ctx->n_req != 1) return fail(ctx, TPC_EINVAL, "vertex finding takes one request (one timeframe) per call");
  tpc_vertex_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else tpc_default_vertex_config(&cfg);
  if (!(cfg.vdrift_cm_us > 0) || !(cfg.gap_us > 0) || cfg.min_tracks < 1 || !(cfg.dca_max_cm >= 0) ||
      !(cfg.ext_max_cm >= 0) || !(cfg.min_pt_gev >= 0 && cfg.min_pt_gev < 1e6))
    return fail(ctx, TPC_EINVAL, "bad vertex configuration");
  CK(cudaSetDevice(ctx->device));
  int rc = vtx_reserve(ctx);
  if (rc) return rc;
  VtxConst vc;
  vc.K = (float)(0.299792458e-3 * ctx->cfg.bz_kg);
  vc.vdrift = (float)cfg.vdrift_cm_us;
  vc.zmax = (float)cfg.zmax_cm;
  vc.dca_max = (float)cfg.dca_max_cm;
  vc.ext_max = (float)cfg.ext_max_cm;
  vc.gap = (float)cfg.gap_us;
  vc.inv_w = (float)(2.0 / cfg.gap_us);
  vc.min_tracks = cfg.min_tracks;
  vc.min_clusters = cfg.min_clusters;
  vc.min_pt = (float)cfg.min_pt_gev;
  vc.bins_cap = kVtxBins;
  const VtxBuf& vb = ctx->vb;
  cudaStream_t s = ctx->stream;
  Counts* cn = ctx->ptr<Counts>(ctx->L.counts);
  const tpc_track* tr = ctx->ptr<tpc_track>(ctx->L.tracks);
  const int bc = ctx->block_clusters;
  const int gM = grid_for(ctx, ctx->caps.tracks, bc), gB = grid_for(ctx, kVtxBins, bc);
  const uint32_t init[2] = {0xFFFFFFFFu, 0u};
  CK(cudaMemcpyAsync(vb.range, init, sizeof(init), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(vb.n, 0, 16, s));
  k_vtx_time<<<gM, bc, 0, s>>>(tr, vc, vb, cn);
  k_vtx_clear<<<gB, bc, 0, s>>>(vc, vb);
  k_vtx_bin<<<gM, bc, 0, s>>>(vc, vb, cn);
  k_vtx_runs<<<1, VTX_RUN_THREADS, 0, s>>>(vc, vb);
  k_vtx_accum<<<gM, bc, 0, s>>>(vc, vb, cn);
  k_vtx_keep<<<gB, bc, 0, s>>>(vc, vb);
  scan(ctx, vb.v_keep, vb.v_idx, LenSrc{vb.n + 1, 0, 0}, nullptr);
  k_vtx_tracks<<<gM, bc, 0, s>>>(tr, vc, vb, cn);
  k_vtx_records<<<gB, bc, 0, s>>>(vc, vb, ctx->vtx_time, ctx->vtx_ntr);
  CK(cudaMemcpyAsync(ctx->h_vtx_n, vb.n, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  ctx->vtx_valid = true;
  ctx->vtx_gen = ctx->fit_gen;
  ctx->vtx_vdrift = vc.vdrift;
  return TPC_OK;
}

int tpc_get_vertices(tpc_ctx* ctx, tpc_vertex* out, int64_t cap, int64_t* n_out, int32_t* track_vertex,
                     float* track_time, float* track_z, float* track_tgl) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->vtx_valid) return fail(ctx, TPC_EINVAL, "tpc_find_vertices has not run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  if (ctx->h_vtx_n[3]) return fail(ctx, TPC_EOVERFLOW, "the tracks' time range needs %d bins, %d reserved",
                                   ctx->h_vtx_n[0], kVtxBins);
  const int32_t nv = ctx->h_vtx_n[2];
  if (n_out) *n_out = nv;
  if (nv > cap && out) return fail(ctx, TPC_EOVERFLOW, "%d vertices do not fit cap %lld", nv, (long long)cap);
  const int32_t M = ctx->h_counts->n_tracks;
  if (out && nv) {
    std::vector<double> t(nv);
    std::vector<int32_t> k(nv);
    CK(cudaMemcpy(t.data(), ctx->vtx_time, sizeof(double) * nv, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(k.data(), ctx->vtx_ntr, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < nv; i++) {
      out[i].time_us = t[i];
      out[i].n_tracks = k[i];
      out[i].request = 0;
    }
  }
  if (track_vertex && M) CK(cudaMemcpy(track_vertex, ctx->vb.vertex, 4 * (size_t)M, cudaMemcpyDeviceToHost));
  if (track_time && M) CK(cudaMemcpy(track_time, ctx->vb.t, 4 * (size_t)M, cudaMemcpyDeviceToHost));
  if (track_z && M) CK(cudaMemcpy(track_z, ctx->vb.z, 4 * (size_t)M, cudaMemcpyDeviceToHost));
  if (track_tgl && M) CK(cudaMemcpy(track_tgl, ctx->vb.tgl, 4 * (size_t)M, cudaMemcpyDeviceToHost));
  return TPC_OK;
}

namespace {
int codec_reserve(tpc_ctx* ctx, int64_t tracks, int64_t clusters) {
  tracks = std::max<int64_t>(tracks, 1);
  clusters = std::max<int64_t>(clusters, 1);
  if (ctx->codec_mem && ctx->codec_tracks_cap >= tracks && ctx->codec_clusters_cap >= clusters) return TPC_OK;
  tracks = std::max(tracks, ctx->codec_tracks_cap);
  clusters = std::max(clusters, ctx->codec_clusters_cap);
  if (ctx->codec_mem) {
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->codec_mem);
    ctx->codec_mem = nullptr;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t o_h = take(sizeof(CodecHeader) * tracks), o_off = take(8 * (tracks + 1)), o_rows = take(clusters);
  const size_t o_qy = take(4 * clusters), o_qz = take(4 * clusters), o_ry = take(4 * clusters),
               o_rz = take(4 * clusters), o_bad = take(4);
  void* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TPC_ENOMEM, "codec buffers of %zu bytes", off);
  }
  char* b = (char*)mem;
  ctx->codec_mem = mem;
  ctx->codec_tracks_cap = tracks;
  ctx->codec_clusters_cap = clusters;
  ctx->cio.head = (CodecHeader*)(b + o_h);
  ctx->cio.off = (const int64_t*)(b + o_off);
  ctx->cio.rows = (uint8_t*)(b + o_rows);
  ctx->cio.qy = (int32_t*)(b + o_qy);
  ctx->cio.qz = (int32_t*)(b + o_qz);
  ctx->cio.ry = (int32_t*)(b + o_ry);
  ctx->cio.rz = (int32_t*)(b + o_rz);
  ctx->codec_bad = (int32_t*)(b + o_bad);
  return TPC_OK;
}

bool codec_unit_ok(double unit) { return unit >= 1e-6 && unit <= 10.0; }
}  // namespace

int tpc_compress(tpc_ctx* ctx, double unit_cm) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  if (!codec_unit_ok(unit_cm)) return fail(ctx, TPC_EINVAL, "fixed-point unit out of range");
  CK(cudaSetDevice(ctx->device));
  int rc = codec_reserve(ctx, ctx->caps.tracks, ctx->caps.n);
  if (rc) return rc;
  Counts* cn = ctx->ptr<Counts>(ctx->L.counts);
  k_codec_encode<<<grid_for(ctx, ctx->caps.tracks, 128, 8), 128, 0, ctx->stream>>>(
      ctx->ptr<tpc_track>(ctx->L.tracks), ctx->ptr<tpc_cluster>(ctx->L.in), refit_in(ctx),
      ctx->ptr<int32_t>(ctx->L.track_clusters), ctx->kc, ctx->cio, (float)unit_cm, cn);
  CK(cudaGetLastError());
  ctx->codec_valid = true;
  return TPC_OK;
}

int tpc_get_compressed(tpc_ctx* ctx, tpc_codec_header* heads, int64_t cap_tracks, uint8_t* rows, int32_t* res_y,
                       int32_t* res_z, int32_t* q_y, int32_t* q_z, int64_t cap_clusters, int64_t* n_tracks,
                       int64_t* n_clusters) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->codec_valid) return fail(ctx, TPC_EINVAL, "tpc_compress has not run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  const int64_t M = ctx->h_counts->n_tracks, N = ctx->h_counts->n_track_clusters;
  if (n_tracks) *n_tracks = M;
  if (n_clusters) *n_clusters = N;
  if ((heads && M > cap_tracks) || ((rows || res_y || res_z || q_y || q_z) && N > cap_clusters))
    return fail(ctx, TPC_EOVERFLOW, "%lld tracks / %lld clusters do not fit", (long long)M, (long long)N);
  if (heads && M) CK(cudaMemcpy(heads, ctx->cio.head, sizeof(CodecHeader) * M, cudaMemcpyDeviceToHost));
  if (rows && N) CK(cudaMemcpy(rows, ctx->cio.rows, N, cudaMemcpyDeviceToHost));
  if (res_y && N) CK(cudaMemcpy(res_y, ctx->cio.ry, 4 * N, cudaMemcpyDeviceToHost));
  if (res_z && N) CK(cudaMemcpy(res_z, ctx->cio.rz, 4 * N, cudaMemcpyDeviceToHost));
  if (q_y && N) CK(cudaMemcpy(q_y, ctx->cio.qy, 4 * N, cudaMemcpyDeviceToHost));
  if (q_z && N) CK(cudaMemcpy(q_z, ctx->cio.qz, 4 * N, cudaMemcpyDeviceToHost));
  return TPC_OK;
}

int tpc_decompress(tpc_ctx* ctx, const tpc_codec_header* heads, int64_t n_tracks, const uint8_t* rows,
                   const int32_t* res_y, const int32_t* res_z, int64_t n_clusters, double unit_cm, int32_t* q_y,
                   int32_t* q_z) {
  if (!ctx || n_tracks < 0 || n_clusters < 0 || (n_tracks && !heads) ||
      (n_clusters && (!rows || !res_y || !res_z || !q_y || !q_z)))
    return TPC_EINVAL;
  if (!codec_unit_ok(unit_cm)) return fail(ctx, TPC_EINVAL, "fixed-point unit out of range");
  std::vector<int64_t> off((size_t)n_tracks + 1, 0);
  for (int64_t m = 0; m < n_tracks; m++) {
    if (heads[m].n_clusters < 0) return fail(ctx, TPC_EINVAL, "negative cluster count in header %lld", (long long)m);
    off[m + 1] = off[m] + heads[m].n_clusters;
  }
  if (off[n_tracks] != n_clusters) return fail(ctx, TPC_EINVAL, "headers count %lld clusters, %lld given",
                                               (long long)off[n_tracks], (long long)n_clusters);
  CK(cudaSetDevice(ctx->device));
  int rc = codec_reserve(ctx, n_tracks, n_clusters);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const CodecIo& io = ctx->cio;
  ctx->codec_valid = false;  // the buffers now hold this decompression
  if (n_tracks) {
    CK(cudaMemcpyAsync(io.head, heads, sizeof(CodecHeader) * n_tracks, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void*)io.off, off.data(), 8 * (n_tracks + 1), cudaMemcpyHostToDevice, s));
  }
  if (n_clusters) {
    CK(cudaMemcpyAsync(io.rows, rows, n_clusters, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(io.ry, res_y, 4 * n_clusters, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(io.rz, res_z, 4 * n_clusters, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(ctx->codec_bad, 0, 4, s));
  if (n_tracks)  // the context's configuration (field, FP64-zone length), whether or not it has loaded data
    k_codec_decode<<<grid_for(ctx, n_tracks, 128, 8), 128, 0, s>>>(make_kconst(ctx->cfg, ctx->caps), io, n_tracks,
                                                                     (float)unit_cm, ctx->codec_bad);
  CK(cudaGetLastError());
  int32_t bad = 0;
  if (n_clusters) {
    CK(cudaMemcpyAsync(q_y, io.qy, 4 * n_clusters, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(q_z, io.qz, 4 * n_clusters, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaMemcpyAsync(&bad, ctx->codec_bad, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return fail(ctx, TPC_EINVAL, "%d tracks could not be decoded (malformed headers or rows)", bad);
  return TPC_OK;
}

int tpc_default_merge_config(tpc_merge_config* c) {
  if (!c) return TPC_EINVAL;
  c->chi2_max = 25.0;
  c->overlap_rows = 10;
  c->min_clusters = 10;
  c->window_cm = 10.0;
  return TPC_OK;
}

namespace {
// z bins per (request, sector) unit: about a quarter of the segments a unit
// can hold, a power of two in [16, 4096].
int64_t merge_zbins(const tpc_ctx* ctx) {
  const int64_t M = std::max<int64_t>(ctx->caps.tracks, 1), U = (int64_t)std::max(ctx->caps.req, 1) * NSEC;
  int64_t nz = 16;
  while (nz < 4096 && nz * 4 * U < M) nz *= 2;
  return nz;
}

int merge_reserve(tpc_ctx* ctx) {
  const int64_t M = std::max<int64_t>(ctx->caps.tracks, 1), U = (int64_t)std::max(ctx->caps.req, 1) * NSEC;
  const int64_t cells = U * merge_zbins(ctx);
  if (ctx->merge_mem && ctx->merge_tracks_cap >= M && ctx->merge_cells_cap >= cells) return TPC_OK;
  if (ctx->merge_mem) {
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->merge_mem);
    ctx->merge_mem = nullptr;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t o_cl = take(4 * M), o_cc = take(4 * cells), o_cs = take(4 * (cells + 1));
  const size_t o_ky = take(sizeof(MergeKey) * M), o_bo = take(4 * M), o_co = take(4 * M), o_so = take(4 * M);
  const size_t o_bi = take(8 * M), o_ln = take(4 * M), o_hi = take(4 * M), o_hd = take(4 * (M + 1));
  const size_t o_ch = take(4 * (M + 1)), o_c = take(4 * M), o_mg = take(sizeof(tpc_track) * M), o_n = take(8);
  void* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TPC_ENOMEM, "merge buffers of %zu bytes", off);
  }
  char* b = (char*)mem;
  ctx->merge_mem = mem;
  ctx->merge_tracks_cap = M;
  ctx->merge_cells_cap = cells;
  MergeBuf& m = ctx->mb;
  m.cell = (int32_t*)(b + o_cl);
  m.cell_cnt = (int32_t*)(b + o_cc);
  m.cell_start = (int32_t*)(b + o_cs);
  m.keys = (MergeKey*)(b + o_ky);
  m.best_out = (int32_t*)(b + o_bo);
  m.chi2_out = (float*)(b + o_co);
  m.second_out = (float*)(b + o_so);
  m.best_in = (unsigned long long*)(b + o_bi);
  m.link = (int32_t*)(b + o_ln);
  m.has_inner = (int32_t*)(b + o_hi);
  m.head = (int32_t*)(b + o_hd);
  m.chain_of_head = (int32_t*)(b + o_ch);
  m.chain = (int32_t*)(b + o_c);
  m.merged = (tpc_track*)(b + o_mg);
  m.n = (int32_t*)(b + o_n);
  if (!ctx->h_merge_n && cudaMallocHost(&ctx->h_merge_n, 8) != cudaSuccess) return fail(ctx, TPC_ECUDA, "pinned buffer");
  return TPC_OK;
}
}  // namespace

int tpc_merge_tracks(tpc_ctx* ctx, const tpc_merge_config* cfg_in) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  tpc_merge_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else tpc_default_merge_config(&cfg);
  if (!(cfg.chi2_max > 0) || cfg.overlap_rows < 0 || cfg.min_clusters < 0 ||
      !(cfg.window_cm >= 1e-3 && cfg.window_cm <= 1e6))
    return fail(ctx, TPC_EINVAL, "bad merge configuration");
  CK(cudaSetDevice(ctx->device));
  int rc = merge_reserve(ctx);
  if (rc) return rc;
  MergeConst mc;
  mc.chi2_max = (float)cfg.chi2_max;
  mc.overlap = cfg.overlap_rows;
  mc.min_clusters = cfg.min_clusters;
  mc.window = (float)cfg.window_cm;
  mc.inv_window = 1.0f / mc.window;
  const int64_t nz = merge_zbins(ctx);
  mc.nz_mask = (int32_t)(nz - 1);
  const MergeBuf& mb = ctx->mb;
  cudaStream_t s = ctx->stream;
  Counts* cn = ctx->ptr<Counts>(ctx->L.counts);
  const tpc_track* tr = ctx->ptr<tpc_track>(ctx->L.tracks);
  const int64_t M = ctx->caps.tracks, U = (int64_t)ctx->caps.req * NSEC;
  const int bc = ctx->block_clusters, gM = grid_for(ctx, M, bc);
  const int64_t cells = U * nz;
  CK(cudaMemsetAsync(mb.cell_cnt, 0, 4 * cells, s));
  CK(cudaMemsetAsync(mb.best_in, 0xFF, 8 * M, s));
  CK(cudaMemsetAsync(mb.has_inner, 0, 4 * M, s));
  CK(cudaMemsetAsync(mb.n, 0, 8, s));
  k_merge_cells<<<gM, bc, 0, s>>>(tr, mc, mb, cn);
  scan(ctx, mb.cell_cnt, mb.cell_start, LenSrc{nullptr, cells, 0}, nullptr);
  k_merge_scatter<<<gM, bc, 0, s>>>(tr, mb, cn);
  k_merge_pairs<<<grid_for(ctx, M * 32, 256, 8), 256, 0, s>>>(tr, ctx->kc, mc, mb, cn);
  k_merge_links<<<gM, bc, 0, s>>>(mb, cn);
  k_merge_heads<<<gM, bc, 0, s>>>(mb, cn);
  scan(ctx, mb.head, mb.chain_of_head, LenSrc{&cn->n_tracks, 0, 0}, mb.n);
  // a thread per segment, so that the chains of a warp start together
  k_merge_refit<<<(int)((M + 127) / 128), 128, 0, s>>>(tr, ctx->ptr<tpc_cluster>(ctx->L.in), refit_in(ctx),
                                                      ctx->ptr<int32_t>(ctx->L.track_clusters), ctx->kc, mb, cn);
  CK(cudaMemcpyAsync(ctx->h_merge_n, mb.n, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaGetLastError());
  ctx->merge_valid = true;
  return TPC_OK;
}

int tpc_get_merged(tpc_ctx* ctx, tpc_track* out, int64_t cap, int64_t* n_out, int32_t* track_link,
                   int32_t* track_chain, float* pair_chi2, float* pair_second) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->merge_valid) return fail(ctx, TPC_EINVAL, "tpc_merge_tracks has not run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  const int32_t nm = ctx->h_merge_n[0];
  const int64_t M = ctx->h_counts->n_tracks;
  if (n_out) *n_out = nm;
  if (out && nm > cap) return fail(ctx, TPC_EOVERFLOW, "%d merged tracks do not fit cap %lld", nm, (long long)cap);
  if (out && nm) CK(cudaMemcpy(out, ctx->mb.merged, sizeof(tpc_track) * nm, cudaMemcpyDeviceToHost));
  if (track_link && M) CK(cudaMemcpy(track_link, ctx->mb.link, 4 * M, cudaMemcpyDeviceToHost));
  if (track_chain && M) CK(cudaMemcpy(track_chain, ctx->mb.chain, 4 * M, cudaMemcpyDeviceToHost));
  if (pair_chi2 && M) CK(cudaMemcpy(pair_chi2, ctx->mb.chi2_out, 4 * M, cudaMemcpyDeviceToHost));
  if (pair_second && M) CK(cudaMemcpy(pair_second, ctx->mb.second_out, 4 * M, cudaMemcpyDeviceToHost));
  return TPC_OK;
}

int tpc_default_reject_config(tpc_reject_config* c) {
  if (!c) return TPC_EINVAL;
  c->p_min_gev = 0.05;
  c->tgl_max = 2.0;
  c->dz_leg_cm = 10.0;
  c->z_ref_cm = 0.0;
  c->use_vertices = 0;
  c->reserved = 0;
  return TPC_OK;
}

namespace {
int reject_reserve(tpc_ctx* ctx) {
  const int64_t M = std::max<int64_t>(ctx->caps.tracks, 1), N = std::max<int64_t>(ctx->caps.n, 1);
  if (ctx->reject_mem && ctx->reject_tracks_cap >= M && ctx->reject_clusters_cap >= N) return TPC_OK;
  if (ctx->reject_mem) {
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->reject_mem);
    ctx->reject_mem = nullptr;
  }
  const size_t o_cnt = 0, o_cls = align_up(32), o_keep = align_up(o_cls + M), total = align_up(o_keep + N);
  void* mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TPC_ENOMEM, "rejection buffers of %zu bytes", total);
  }
  char* b = (char*)mem;
  ctx->reject_mem = mem;
  ctx->reject_tracks_cap = M;
  ctx->reject_clusters_cap = N;
  ctx->rb.count = (unsigned long long*)(b + o_cnt);
  ctx->rb.cls = (uint8_t*)(b + o_cls);
  ctx->rb.keep = (uint8_t*)(b + o_keep);
  return TPC_OK;
}
}  // namespace

int tpc_reject_clusters(tpc_ctx* ctx, const tpc_reject_config* cfg_in) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->fitted) return fail(ctx, TPC_EINVAL, "tpc_fit_tracks has not run");
  tpc_reject_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else tpc_default_reject_config(&cfg);
  if (!(cfg.p_min_gev >= 0) || !(cfg.tgl_max >= 0) || !(cfg.dz_leg_cm >= 0) || !std::isfinite(cfg.z_ref_cm) ||
      (cfg.use_vertices != 0 && cfg.use_vertices != 1))
    return fail(ctx, TPC_EINVAL, "bad rejection configuration");
  if (cfg.use_vertices && !(ctx->vtx_valid && ctx->vtx_gen == ctx->fit_gen))
    return fail(ctx, TPC_EINVAL, "use_vertices needs tpc_find_vertices on the current fit");
  CK(cudaSetDevice(ctx->device));
  int rc = reject_reserve(ctx);
  if (rc) return rc;
  RejConst c;
  c.p_min = (float)cfg.p_min_gev;
  c.tgl_max = (float)cfg.tgl_max;
  c.dz_leg = (float)cfg.dz_leg_cm;
  c.z_ref = (float)cfg.z_ref_cm;
  c.K = (float)(0.299792458e-3 * ctx->cfg.bz_kg);
  c.x_out = (float)(85.2 + (NROW - 1) * ((245.8 - 85.2) / 158.0));
  c.vdrift = ctx->vtx_vdrift;
  c.use_vertices = cfg.use_vertices;
  cudaStream_t s = ctx->stream;
  const int64_t M = ctx->caps.tracks;
  CK(cudaMemsetAsync(ctx->rb.count, 0, 32, s));
  if (ctx->n) CK(cudaMemsetAsync(ctx->rb.keep, 1, ctx->n, s));
  k_reject<<<grid_for(ctx, M, 256), 256, 0, s>>>(ctx->ptr<tpc_track>(ctx->L.tracks),
                                                ctx->ptr<int32_t>(ctx->L.track_clusters), c,
                                                cfg.use_vertices ? ctx->vtx_time : nullptr,
                                                cfg.use_vertices ? ctx->vb.n + 2 : nullptr,
                                                cfg.use_vertices ? ctx->vb.t : nullptr, ctx->rb,
                                                ctx->ptr<Counts>(ctx->L.counts));
  CK(cudaGetLastError());
  ctx->reject_valid = true;
  return TPC_OK;
}

int tpc_get_rejection(tpc_ctx* ctx, uint8_t* track_class, uint8_t* cluster_keep, int64_t* counts) {
  if (!ctx) return TPC_EINVAL;
  if (!ctx->reject_valid) return fail(ctx, TPC_EINVAL, "tpc_reject_clusters has not run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  const int64_t M = ctx->h_counts->n_tracks;
  if (track_class && M) CK(cudaMemcpy(track_class, ctx->rb.cls, M, cudaMemcpyDeviceToHost));
  if (cluster_keep && ctx->n) CK(cudaMemcpy(cluster_keep, ctx->rb.keep, ctx->n, cudaMemcpyDeviceToHost));
  if (counts) {
    unsigned long long c[4];
    CK(cudaMemcpy(c, ctx->rb.count, sizeof(c), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; i++) counts[i] = (int64_t)c[i];
  }
  return TPC_OK;
}

int tpc_measure_alu_peaks(int device, double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops && !fp64_tflops) return TPC_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return TPC_ECUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TPC_ECUDA;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* out = nullptr;
  int rc = TPC_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&out, sizeof(double)) != cudaSuccess)
    rc = TPC_ECUDA;
  const int threads = 256, blocks = n_sm * 8;
  auto run = [&](bool dbl, int iters, double* tflops) {
    if (rc != TPC_OK || !tflops) return;
    float best = 0.0f;
    for (int r = 0; r < 3; r++) {  // the first run warms up, the best of the rest counts
      cudaEventRecord(e0, st);
      if (dbl) k_fma_probe<double><<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
      else k_fma_probe<float><<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = TPC_ECUDA;
        return;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    const double flop = 2.0 * PROBE_CHAINS * (double)iters * threads * blocks;
    *tflops = flop / (best * 1e-3) / 1e12;
  };
  run(false, 1 << 12, fp32_tflops);
  run(true, 1 << 7, fp64_tflops);
  if (cudaGetLastError() != cudaSuccess) rc = TPC_ECUDA;
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return rc;
}

}  // extern "C"

// =========================================================== no-alloc variant
//
// tpc_row_params_noalloc: the per-row-sector pass of the grid stage (cluster
// count, exact z range, bin parameters and bin bases of every (request,
// sector, row)) for callers that cannot allocate device memory -- code that
// runs inside a host-side memory budget it does not own, an allocator hook,
// or a process whose CUDA allocations are forbidden once it is serving.  It
// writes the same RsParams records as the grid stage of tpc_find_tracks,
// but its counters live in the file-scope array below instead of an arena.
namespace {

constexpr int NOALLOC_MAX_REQ = 8;
constexpr int NOALLOC_MAX_RS = NOALLOC_MAX_REQ * NSEC * NROW;  // 45,792 row-sectors

struct NoallocScratch {
  uint32_t status;
  uint32_t pad[63];
  int64_t req_off[NOALLOC_MAX_REQ + 1];
  int64_t pad2[7];
  int32_t cnt[NOALLOC_MAX_RS];
  uint32_t zmin[NOALLOC_MAX_RS];
  uint32_t zmax[NOALLOC_MAX_RS];
  int32_t nbins[NOALLOC_MAX_RS];
};

}  // namespace

// About 0.73 MB on every GPU that loads the library, kept until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

namespace {

__global__ void k_na_clear(NoallocScratch* s, int nrs) {
  for (int64_t i = gtid(); i < nrs; i += gstride()) {
    s->cnt[i] = 0;
    s->zmin[i] = 0xFFFFFFFFu;
    s->zmax[i] = 0u;
  }
  if (gtid() == 0) s->status = 0u;
}

__global__ void k_na_count(const tpc_cluster* __restrict__ in, int64_t n, int n_req, NoallocScratch* s) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int4 raw = __ldg(reinterpret_cast<const int4*>(in) + i);
    const float z = __int_as_float(raw.y), y = __int_as_float(raw.x);
    const uint32_t row = (uint32_t)raw.z & 0xFFFFu, sec = (uint32_t)raw.z >> 16;
    if (row >= NROW || sec >= NSEC || !isfinite(y) || !isfinite(z)) {
      atomicOr(&s->status, ST_EINVAL);
      continue;
    }
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s->req_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const int rs = (lo * NSEC + (int)sec) * NROW + (int)row;
    atomicAdd(&s->cnt[rs], 1);
    const uint32_t zo = f2ord(z);
    atomicMin(&s->zmin[rs], zo);
    atomicMax(&s->zmax[rs], zo);
  }
}

// Bin parameters, the same binary32 operation sequence as the grid stage.
__global__ void k_na_params(NoallocScratch* s, int nrs, RsParams* __restrict__ out) {
  for (int64_t rs = gtid(); rs < nrs; rs += gstride()) {
    const int row = (int)(rs % NROW);
    const int n = s->cnt[rs];
    const float zl = n ? ord2f(s->zmin[rs]) : 0.0f, zh = n ? ord2f(s->zmax[rs]) : 0.0f;
    const float yh = g_row_yhi[row], yl = -yh;
    const float wy = __fsub_rn(yh, yl);
    const float dz = __fsub_rn(zh, zl);
    const float area = __fmul_rn(wy, fmaxf(dz, 1.0f));
    float sz = __fsqrt_rn(__fdiv_rn(__fmul_rn(area, 2.0f), __int2float_rn(n > 1 ? n : 1)));
    sz = fminf(fmaxf(sz, 1.0f), 64.0f);
    int ny = __float2int_rz(__fdiv_rn(wy, sz)) + 1;
    int nz = __float2int_rz(__fdiv_rn(dz, sz)) + 1;
    if (ny > 256) ny = 256;
    if (nz > 4096) nz = 4096;
    RsParams p;
    p.z_lo = zl;
    p.z_hi = zh;
    p.inv_y = __fdiv_rn(__int2float_rn(ny), wy);
    p.inv_z = __fdiv_rn(__int2float_rn(nz), fmaxf(dz, 1e-3f));
    p.n_y = ny;
    p.n_z = nz;
    p.bin_base = 0;
    p.count = n;
    out[rs] = p;
    s->nbins[rs] = ny * nz;
  }
}

// Exclusive prefix sum of the bin counts into bin_base (one block).
__global__ void __launch_bounds__(1024) k_na_binbase(const NoallocScratch* s, int nrs, RsParams* __restrict__ out) {
  __shared__ int ws[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nrs; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nrs ? s->nbins[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += t;
      }
      ws[lane] = w;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? ws[warp - 1] : 0);
    if (i < nrs) out[i].bin_base = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += ws[31];
    __syncthreads();
  }
}

std::mutex g_na_mutex;
struct NaAddr {
  unsigned long long ctx_id = 0;  // context the address belongs to
  void* addr = nullptr;           // device address of g_noalloc_scratch there
};
std::vector<NaAddr> g_na_addr;  // per device

}  // namespace

extern "C" int tpc_row_params_noalloc(const tpc_cluster* d_clusters, int64_t n, const int64_t* req_offsets,
                                      int32_t n_req, void* d_params_out, void* cuda_stream) {
  if (n_req < 1 || n_req > NOALLOC_MAX_REQ || !req_offsets || req_offsets[0] != 0 || req_offsets[n_req] != n ||
      n < 0 || n >= 0x7FFFFFFF || (n > 0 && !d_clusters) || !d_params_out)
    return TPC_EINVAL;
  for (int32_t q = 0; q < n_req; q++)
    if (req_offsets[q + 1] < req_offsets[q]) return TPC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPC_ECUDA;
  void* addr = nullptr;
  {
    // once per device, with that device current: the device address of the
    // scratch array (its name is only a host-side stand-in in host code)
    // (again after the context was replaced, e.g. by cudaDeviceReset)
    if (ensure_device_tables(dev) != cudaSuccess) return TPC_ECUDA;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if ((int)g_na_addr.size() <= dev) g_na_addr.resize(dev + 1);
    if (!g_na_addr[dev].addr || id == 0 || g_na_addr[dev].ctx_id != id) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TPC_ECUDA;
      g_na_addr[dev].addr = p;
      g_na_addr[dev].ctx_id = id;
    }
    addr = g_na_addr[dev].addr;
  }
  NoallocScratch* s = reinterpret_cast<NoallocScratch*>(addr);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nrs = n_req * NSEC * NROW;
  RsParams* out = reinterpret_cast<RsParams*>(d_params_out);
  int64_t off_host[NOALLOC_MAX_REQ + 1];
  memcpy(off_host, req_offsets, sizeof(int64_t) * (n_req + 1));
  if (cudaMemcpyAsync(s->req_off, off_host, sizeof(int64_t) * (n_req + 1), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return TPC_ECUDA;
  k_na_clear<<<(nrs + 255) / 256, 256, 0, st>>>(s, nrs);
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_na_count<<<blocks, 256, 0, st>>>(d_clusters, n, n_req, s);
  }
  k_na_params<<<(nrs + 255) / 256, 256, 0, st>>>(s, nrs, out);
  k_na_binbase<<<1, 1024, 0, st>>>(s, nrs, out);
  if (cudaGetLastError() != cudaSuccess) return TPC_ECUDA;
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, &s->status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TPC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TPC_ECUDA;
  return (status & ST_EINVAL) ? TPC_EINVAL : TPC_OK;
}
