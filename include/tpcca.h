/*
 * tpcca.h -- C ABI of the B300 sector tracker (libtpcca.so).
 *
 * Per-sector TPC track finding as described in Sec. 2 of "Tracking
 * performance in high multiplicities environment at ALICE" (arXiv
 * 1709.00618): the TPC is split into 36 sectors tracked independently; a
 * cellular automaton links adjacent hits close to a straight line (Fig. 1a)
 * and concatenates the links into short candidates (Fig. 1b); track following
 * fits each candidate and extends it row by row with a simplified Kalman
 * filter (Fig. 1c); a final selection gives each cluster to at most one track.
 * The field model is uniform Bz (Sec. 2: Bx and By are not used online).
 * Several independent requests (events or timeframes) can be processed in one
 * batch, as Sec. 2 does to fill a GPU.
 *
 * Conventions for every function:
 *  - Return value: TPC_OK (0) or one of the TPC_E* codes; tpc_last_error()
 *    gives a one-line description of the last failure on that context.
 *  - Host pointers are owned by the caller and only read/written during the
 *    call (tpc_load_* copies its input before returning when on_device == 0;
 *    with on_device != 0 the device buffer must stay valid until the copy on
 *    the context's stream has run, i.e. until the next tpc_sync/tpc_get_*).
 *  - Device memory used by the pipeline belongs to the context (its arena).
 *  - All work is enqueued on the context's CUDA stream in call order;
 *    tpc_find_tracks / tpc_fit_tracks return without waiting.  Errors raised
 *    on the device (bad input, capacity overflow, a bounded wait that ran
 *    out) are reported by the next tpc_sync or tpc_get_* call.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef TPCCA_H
#define TPCCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
enum {
  TPC_OK = 0,
  TPC_EINVAL = 1,    /* bad argument or bad cluster (row >= 159, sector >= 36, non-finite y/z) */
  TPC_ENOMEM = 2,    /* the request does not fit the context's HBM budget / arena */
  TPC_ECUDA = 3,     /* a CUDA runtime call failed */
  TPC_ETIMEOUT = 4,  /* a bounded device-side wait ran out (no GPU hang; the context stays usable) */
  TPC_EOVERFLOW = 5, /* an output or internal capacity was too small; nothing was truncated silently,
                        the call can be retried with a larger capacity (see tpc_reserve) */
  TPC_EBUSY = 6      /* the serving queue is full */
};

/* ----------------------------------------------------------------- records */
/* One cluster, 16 bytes.  (row, sector) address the pad row (0..158, radii
 * linearly spaced 85.2..245.8 cm) and the sector (0..35; 0..17 z >= 0 side,
 * 18..35 z < 0 side, centre angle (s mod 18)*20+10 degrees).  y and z are the
 * local sector coordinates in cm (z may be a drift-time coordinate for
 * continuous read-out, Sec. 5).  id is opaque and ignored. */
typedef struct {
  float y, z;
  uint16_t row, sector;
  uint32_t id;
} tpc_cluster;

/* One fitted sector track, 128 bytes.  par = (y, z, sin phi, dz/ds_T, q/pT)
 * at local x (the radius of first_row); cov = packed lower triangle of the
 * symmetric 5x5 covariance in row-major order ((0,0),(1,0),(1,1),(2,0),...).
 * cluster_offset indexes the optional track_clusters output of
 * tpc_get_tracks.  flags: TPC_TF_* bits. */
typedef struct {
  float x;
  float par[5];
  float cov[15];
  int32_t reserved;
  double chi2;
  int32_t ndf, n_clusters, sector, request, first_row, last_row, cluster_offset, flags;
} tpc_track;

enum {
  TPC_TF_TAINT_TIE = 1,   /* a pick had a second candidate within the divergence margin */
  TPC_TF_TAINT_GATE = 2,  /* a candidate lay within the margin of the chi2 gate */
  TPC_TF_TAINT_EDGE = 4,  /* a sector-edge stop test was within the margin */
  TPC_TF_TAINT_SLIM = 8,  /* a |sin phi| limit test was within the margin */
  TPC_TF_SEED_FAIL = 16,
  TPC_TF_BACK_FAIL = 32,
  TPC_TF_REFIT_FAIL = 64
};

/* Algorithm constants.  The paper prints none of them; the defaults are the
 * documented reading (tpc_default_config). */
typedef struct {
  double bz_kg;        /* uniform field (kG); default 5 */
  double sigma;        /* cluster resolution in y and z (cm); default 0.1 */
  float d_max;         /* accepted squared straight-line deviation of a link (cm^2); 1.0 */
  int32_t min_chain;   /* clusters of the shortest tracklet; 3 */
  int32_t max_miss;    /* consecutive empty rows that end an extension; 5 */
  int32_t n_min_track; /* clusters a selected track must own; 10 */
  double gate;         /* chi2 gate of the pick-up; 16 */
  double c0[5];        /* seed covariance diagonal; 100, 100, 1, 1, 100 */
  double s_max;        /* |sin phi| limit of the propagation; 0.95 */
  double edge;         /* cm beyond the sector edge that end an extension; 2 */
  double taint_rel;    /* divergence margin for the taint flags; 1e-4: a pick whose second-best
                          chi2 is within taint_rel (1 + best), or a candidate within
                          taint_rel (1 + gate) of the gate, flags its tracklet */
  int32_t fp64_updates;/* Kalman updates after each seed done in FP64; 10.
                          Outside the forward pass, up to as many again while
                          the last one still more than halved the variance of
                          sin phi, dz/ds_T or q/pT */
  int32_t link_skip;   /* 0 (default): links join rows r-1 and r+1 only.  1: the
                          next-row variant against duplicate tracklets -- a
                          cluster on rows 2..156 without an accepted r-1/r+1 pair
                          takes the best pair skipping one row on one or both
                          sides, (r-2, r+1), (r-1, r+2) or (r-2, r+2), with windows
                          scaled by the row distance; chains then cross the
                          skipped rows and track following only propagates
                          through them */
} tpc_config;

/* Fills cfg with the defaults above. */
int tpc_default_config(tpc_config *cfg);

/* --------------------------------------------------------------- contexts */
typedef struct tpc_ctx tpc_ctx;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * enqueue on (NULL: the context creates its own non-blocking stream).
 * hbm_budget: bytes the context may allocate for its arena (0: no limit
 * beyond free memory).  cfg NULL: defaults. */
int tpc_create(tpc_ctx **out, const tpc_config *cfg, int device, void *cuda_stream, size_t hbm_budget);

/* Same, but the arena is caller-provided device memory (e.g. a PyTorch
 * tensor) of `bytes` bytes, aligned to 256 bytes, that must outlive the
 * context.  The context never allocates device memory beyond it. */
int tpc_create_with_arena(tpc_ctx **out, const tpc_config *cfg, int device, void *cuda_stream, void *arena,
                          size_t bytes);

void tpc_destroy(tpc_ctx *ctx);
const char *tpc_last_error(tpc_ctx *ctx);

/* Arena bytes needed for batches of up to n_clusters clusters in up to
 * n_requests requests (0 = library defaults for the internal capacities). */
size_t tpc_arena_bytes(int64_t n_clusters, int32_t n_requests);

/* The same for explicit grid-bin and tracklet capacities (0: the default,
 * which is also the least), e.g. the arena of a retry after TPC_EOVERFLOW. */
size_t tpc_arena_bytes_for(int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets);

/* Size the context for at least n_clusters / n_requests (and, when nonzero,
 * the given grid-bin and tracklet capacities).  Called implicitly by the
 * load functions; call it explicitly to retry after TPC_EOVERFLOW. */
int tpc_reserve(tpc_ctx *ctx, int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets);

/* Device bytes the context's arena holds now (0 before the first load). */
int tpc_get_arena_bytes(tpc_ctx *ctx, size_t *bytes);

/* Device bytes the context's arena would hold after tpc_reserve with these
 * arguments (its current size when that reserve would not grow it).  Host
 * arithmetic only: allocates nothing and does not touch the device. */
int tpc_reserve_bytes(tpc_ctx *ctx, int64_t n_clusters, int32_t n_requests, int64_t n_bins, int64_t n_tracklets,
                      size_t *bytes);

/* ------------------------------------------------------------ the hot path */
/* a1: copy n clusters (host or device pointer) into the context as one
 * request.  Validation of each cluster happens on the device; a bad cluster
 * makes the next tpc_sync / tpc_get_* return TPC_EINVAL. */
int tpc_load_clusters(tpc_ctx *ctx, const tpc_cluster *clusters, int64_t n, int on_device);

/* Same for a batch of n_req independent requests: request q is clusters
 * [req_offsets[q], req_offsets[q+1]) (host array of n_req+1 entries,
 * req_offsets[0] = 0, non-decreasing).  Requests never share tracks. */
int tpc_load_batch(tpc_ctx *ctx, const tpc_cluster *clusters, const int64_t *req_offsets, int32_t n_req,
                   int on_device);

/* a2-a7: grid, CA neighbours, link cleaning, tracklets, Kalman following,
 * selection and cluster assignment (Sec. 2 phase 1).  Asynchronous. */
int tpc_find_tracks(tpc_ctx *ctx);

/* a8: Kalman refit of every selected track on the clusters it owns (the
 * final fit on the GPU of Sec. 2).  Asynchronous. */
int tpc_fit_tracks(tpc_ctx *ctx);

/* Both of the above as one CUDA-graph launch (captured on first use for the
 * context's current capacity, then replayed).  Equivalent results. */
int tpc_run_graph(tpc_ctx *ctx);

/* a9: wait for the stream and copy the results out.  out: room for cap
 * tracks; *n_out receives the number of tracks (also when cap is too small,
 * in which case nothing is copied and TPC_EOVERFLOW is returned).
 * cluster_track (optional, n entries): track index of every loaded cluster
 * in load order, -1 when unassigned.  track_clusters (optional, sum of
 * n_clusters entries): the load-order indices of each track's clusters at
 * tracks[i].cluster_offset, innermost row first. */
int tpc_get_tracks(tpc_ctx *ctx, tpc_track *out, int64_t cap, int64_t *n_out, int32_t *cluster_track,
                   int32_t *track_clusters);

/* One request host to host (a1-a9 in one call): copies n clusters from host
 * memory in (page-locked memory lets the copy run at full speed), finds and
 * fits the tracks, and copies the tracks into out (room for cap) and the
 * cluster assignment into cluster_track (optional, n entries, as
 * tpc_get_tracks).  From 4 Mi clusters on, the assignment's copy, which is
 * final after the selection (a7), runs on a stream of its own while the
 * refit (a8) computes (with a page-locked cluster_track; a pageable one makes
 * the copy wait for the host); below that a2-a8 run as the context's CUDA
 * graph (tpc_run_graph, unless the context was created on the legacy default
 * stream) and both copies follow.  The call returns when both copies have
 * landed.  Same results and errors as
 * tpc_load_clusters + tpc_find_tracks + tpc_fit_tracks + tpc_get_tracks;
 * after an error the contents of cluster_track are undefined. */
int tpc_track_host(tpc_ctx *ctx, const tpc_cluster *clusters, int64_t n, tpc_track *out, int64_t cap,
                   int64_t *n_out, int32_t *cluster_track);

/* Non-blocking form of tpc_get_tracks for a run that has completed (the
 * caller has seen its stream idle, e.g. through an event recorded after
 * tpc_run_graph): reports device-side errors and *n_out as tpc_get_tracks,
 * then enqueues the copies of the tracks and of cluster_track (either may
 * be NULL) on the context's stream and returns.  The copies have landed
 * once the stream is idle again; with page-locked destinations they run
 * without holding up the calling thread.  TPC_EBUSY: the run is still
 * going.  TPC_EOVERFLOW: device capacities overflowed (*n_out untouched)
 * or cap < *n_out (nothing copied). */
int tpc_get_tracks_async(tpc_ctx *ctx, tpc_track *out, int64_t cap, int64_t *n_out, int32_t *cluster_track);

/* ------------------------------------------------------ batched requests */
/* Several independent requests (events or timeframes) tracked as one batch
 * on one context, the way Sec. 2 processes several events at once to fill a
 * GPU: the requests' clusters are copied from their own host buffers into
 * the context (one copy per request), a2-a8 run as one CUDA-graph launch
 * over the whole batch (tpc_run_graph), and each request's tracks and
 * cluster assignment are copied into its own buffers.  Requests never share
 * tracks, so each request's result equals the one it gets alone. */
typedef struct {
  int64_t id;                  /* caller-chosen, unique within the batch */
  const tpc_cluster *clusters; /* host memory, n records; page-locked memory lets the copy run
                                  asynchronously.  Must stay valid and unchanged until tpc_poll
                                  reports the request done */
  int64_t n;
  tpc_track *tracks_out;       /* host memory, room for cap tracks (a track owns at least
                                  n_min_track clusters, so n / n_min_track + 1 always suffices);
                                  tracks as tpc_get_tracks writes them for the whole batch
                                  (request = the request's position in the batch) */
  int64_t cap;
  int32_t *cluster_track_out;  /* host memory, n entries or NULL: index into this request's
                                  tracks_out of every cluster's track (input order), -1 when
                                  unassigned */
  int64_t *n_tracks;           /* NULL, or receives the request's track count when it is done
                                  (also when cap was too small) */
} tpc_request;

/* Enqueue the batch reqs[0..n) on the context's stream and return without
 * waiting.  Buffers are owned by the caller and must stay valid until
 * tpc_poll reports each request done.  TPC_EBUSY: the previous batch of
 * this context is still in flight (its requests are forgotten once a new
 * batch is accepted).  TPC_EINVAL: n < 1, bad sizes, null buffers or an id
 * used twice.  TPC_ENOMEM: the batch does not fit the context's budget.
 * While a batch is in flight the context's tpc_load_* calls return
 * TPC_EBUSY; once it is done, tpc_get_tracks and tpc_get_stage show the
 * whole batch. */
int tpc_submit_batch(tpc_ctx *ctx, const tpc_request *reqs, int32_t n);

/* Never waits.  *done = 1 once the request's results are in its buffers
 * (the call then returns the request's status: TPC_OK, TPC_EOVERFLOW when
 * its cap was too small -- nothing copied, *n_tracks set -- or the batch's
 * error, e.g. TPC_EINVAL for a cluster that failed validation); *done = 0
 * while it runs (TPC_OK).  A device capacity overflow reruns the batch once
 * with the worst-case tracklet capacity.  TPC_EINVAL for an id that is not
 * in the context's current batch. */
int tpc_poll(tpc_ctx *ctx, int64_t request_id, int *done);

/* Wait for the context's stream and report device-side errors. */
int tpc_sync(tpc_ctx *ctx);

/* Counters of the last run: [0] clusters, [1] requests, [2] row-sectors,
 * [3] grid bins, [4] tracklets, [5] tracks, [6] device status word. */
int tpc_get_counts(tpc_ctx *ctx, int64_t counts[8]);

/* Intermediate results of the last run, for stage-by-stage parity checks:
 * copies item `item` (TPC_ITEM_*) to host_out if cap_bytes suffices and
 * stores its size in *n_bytes.  Waits for the stream. */
enum {
  TPC_ITEM_PERM = 1,       /* int32[n]   sorted position -> load index */
  TPC_ITEM_RS_OF = 2,      /* int32[n]   sorted position -> row-sector (request*36+sector)*159+row */
  TPC_ITEM_ROW_START = 3,  /* int32[nrs+1] */
  TPC_ITEM_RS_PARAMS = 4,  /* nrs x {float z_lo, z_hi, inv_y, inv_z; int32 n_y, n_z, bin_base, count} */
  TPC_ITEM_BIN_START = 5,  /* int32[n_bins+1] */
  TPC_ITEM_UP = 6, TPC_ITEM_DN = 7, TPC_ITEM_TIE = 8, /* int32[n], int32[n], uint8[n] (sorted indexing) */
  TPC_ITEM_UP_M = 9, TPC_ITEM_DN_M = 10,
  TPC_ITEM_TL_START = 11, TPC_ITEM_TL_LEN = 12,       /* int32[n_tracklets] */
  TPC_ITEM_F_N = 13, TPC_ITEM_F_NF = 14, TPC_ITEM_F_NB = 15, TPC_ITEM_F_FLAGS = 16, TPC_ITEM_F_ROW = 17,
  TPC_ITEM_F_HITS = 18,    /* int32[n_tracklets*159] */
  TPC_ITEM_F_PAR = 19,     /* float[n_tracklets*5], z absolute */
  TPC_ITEM_F_COV = 20,     /* float[n_tracklets*15] */
  TPC_ITEM_F_CHI2 = 21,    /* double[n_tracklets] */
  TPC_ITEM_OWNER = 22,     /* uint64[n] */
  TPC_ITEM_TL_TRACK = 23,  /* int32[n_tracklets] */
  TPC_ITEM_SY = 24, TPC_ITEM_SZ = 25 /* float[n] sorted positions */
};
int tpc_get_stage(tpc_ctx *ctx, int item, void *host_out, int64_t cap_bytes, int64_t *n_bytes);

/* ------------------------------------------------------------ measurement */
/* With profiling on, tpc_find_tracks / tpc_fit_tracks record CUDA events on
 * the context's stream between stages (not inside tpc_run_graph).
 * tpc_get_stage_times waits for the stream and returns the device time in ms
 * of [0] a2 grid, [1] a3 neighbours, [2] a4+a5 links and tracklets,
 * [3] a6 follow, [4] a7 selection, [5] a8 refit of the last such run. */
int tpc_set_profiling(tpc_ctx *ctx, int on);
int tpc_get_stage_times(tpc_ctx *ctx, float ms[6]);

/* Work counters of the last run (waits for the stream): [0] propagations
 * with covariance transport, [1] FP32 Kalman updates, [2] FP64-zone updates,
 * [3] candidate clusters examined by the pick-up, [4] propagations done with
 * the FP64 covariance. */
int tpc_get_work(tpc_ctx *ctx, uint64_t work[5]);

/* Per Kalman kernel, in launch order -- [0] follow seed + forward FP64 zone,
 * [1] its zone tail, [2] follow forward FP32, [3] follow backward re-seed +
 * FP64 zone, [4] its zone tail, [5] follow backward FP32 refit rows, [6]
 * follow backward FP32 (extension) + output, [7] refit FP64 zone, [8] its
 * zone tail, [9] refit FP32 + output -- ms[k]: device time of the last
 * profiled run (events between the launches; a work-order pass counts with
 * the kernel before it; a kernel the batch's size does not launch has
 * about 0; ms may be NULL), work[5k..5k+4]: that kernel's share of the
 * counters of tpc_get_work in the same order (work may be NULL).  Waits for
 * the stream. */
#define TPC_KALMAN_KERNELS 10
int tpc_get_kalman_profile(tpc_ctx *ctx, float ms[TPC_KALMAN_KERNELS], uint64_t work[5 * TPC_KALMAN_KERNELS]);

/* Measured issue rates of the FP32 and FP64 fused multiply-add pipes of
 * device `device` (TFLOP/s, an FMA counting 2): 8 independent FMA chains
 * per thread over 8 blocks of 256 threads per SM, best of two timed runs
 * after a warm-up.  Either pointer may be NULL.  The denominators of the
 * Kalman kernels' ALU rooflines. */
int tpc_measure_alu_peaks(int device, double *fp32_tflops, double *fp64_tflops);

/* Number of kernel launches in one tpc_run_graph (kernel nodes of the
 * captured graph); TPC_EINVAL before the first capture. */
int tpc_graph_kernels(tpc_ctx *ctx, int32_t *n);

/* Debug trace of one tracklet's Kalman updates (a6): after
 * tpc_set_trace(ctx, t) every following tpc_find_tracks records, for each
 * update of tracklet t (numbered as in TPC_ITEM_TL_START), 16 floats: pass
 * (0 forward, 1 backward), row, updates since the (re)seed, y, z, sin phi,
 * dz/ds_T, q/pT, C_yy, C_zz, C_ss, C_tt, C_qq, chi2, residual y, residual z
 * (the residuals before the update).  t < 0 switches it off.  At most 2048
 * records are kept; *n_records reports how many were produced. */
int tpc_set_trace(tpc_ctx *ctx, int32_t tracklet);
int tpc_get_trace(tpc_ctx *ctx, float *out, int32_t cap_records, int32_t *n_records);

/* ------------------------------------------------- allocation-free variant */
/* The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory (code running under a memory budget owned
 * by someone else, inside an allocator hook, or in a server that forbids
 * CUDA allocations once running).  It computes the per-row-sector records
 * of the grid stage -- the same 32-byte {z_lo, z_hi, inv_y, inv_z, n_y, n_z,
 * bin_base, count} records as TPC_ITEM_RS_PARAMS -- for the clusters at
 * d_clusters (device memory, n records in load order, requests as in
 * tpc_load_batch with host req_offsets), writing n_req*36*159 records to
 * d_params_out (device memory, caller-allocated).  Its counters live in one
 * file-scope device array of about 0.73 MB that every GPU loading the
 * library keeps until exit; no call allocates or frees device memory.
 * Limits: 1 <= n_req <= 8 (TPC_EINVAL beyond), n < 2^31 - 1.
 * The first call on a device looks up the array's device address and
 * uploads the row geometry with that device current; make that first call
 * before any stream capture.  Work is enqueued on cuda_stream (NULL: the
 * default stream) and the call waits for it: it returns TPC_EINVAL when a
 * cluster fails validation, TPC_ECUDA on a CUDA error, TPC_OK otherwise.
 * Every call clears and reuses the same array, so calls that overlap on the
 * GPU (other streams, other host threads) race with each other. */
int tpc_row_params_noalloc(const tpc_cluster *d_clusters, int64_t n, const int64_t *req_offsets, int32_t n_req,
                           void *d_params_out, void *cuda_stream);

/* ------------------------------------------------------ tuning (autotuner) */
/* Launch shapes of a context.  Results do not depend on them. */
typedef struct {
  int32_t block_clusters;     /* threads per block of the cluster-, row-sector- and tracklet-parallel kernels
                                 (multiple of 32, at most 1024) */
  int32_t block_follow;       /* threads per block of the Kalman kernels (multiple of 32, at most 128) */
  int32_t ctas_per_sm_zone;   /* most CTAs per SM of the Kalman kernels running FP64 zones; their grids are
                                 one wave of resident CTAs (64: as many as fit); reported as 0 while the
                                 default applies: 4 from 4 Mi loaded clusters on, else 2 */
  int32_t ctas_per_sm_follow; /* the same for the Kalman kernels that refill lanes (FP32 phases); reported
                                 as 0 while the default applies: 64 from 4 Mi loaded clusters on, else 2 */
  int32_t refill;             /* idle lanes of a warp of a refilling kernel that trigger the warp's common
                                 fetch of new work (1..32; 1: each lane refills at once) */
  int32_t chunks;             /* 1, or 2: the Kalman stage splits its items in two halves whose kernels run
                                 on two streams, one kernel apart, so that one half's FP64 zone shares the
                                 SMs with the other half's FP32 phase (profiled runs use 1); reported as 0
                                 while the default (1) applies */
  int32_t zone_rows;          /* row steps the FP64-zone kernels take with a warp's 32 tracklets (tracks) in
                                 step before a zone still open goes on in a zone tail kernel, 32 such items to
                                 a warp (follow forward and backward passes and refit; 159 or more: no tail
                                 kernels); reported as 0 while the default applies: 9 backward from 16 Mi
                                 loaded clusters on, 9 forward and 10 in the refit from 48 Mi on, else none */
} tpc_tuning;

int tpc_get_tuning(tpc_ctx *ctx, tpc_tuning *t);

/* Fields <= 0 keep their current value.  TPC_EINVAL for out-of-range
 * values.  Invalidates a captured graph. */
int tpc_set_tuning(tpc_ctx *ctx, const tpc_tuning *t);

/* Autotuner: with a representative batch loaded, times tpc_find_tracks +
 * tpc_fit_tracks (median of reps runs, CUDA events on the context's stream)
 * over block_clusters {128, 256, 512}, block_follow {64, 96, 128},
 * ctas_per_sm_zone {2, 3, 4}, ctas_per_sm_follow {2, 3, 64}, refill
 * {1, 4, 8, 16} and chunks {1, 2} by coordinate descent from the current
 * shapes, keeps the fastest and reports it in *best and *best_ms (either
 * may be NULL).  The results of the loaded batch are overwritten (rerun
 * tpc_find_tracks before get). */
int tpc_autotune(tpc_ctx *ctx, int32_t reps, tpc_tuning *best, float *best_ms);

/* --------------------------------------------- vertices in the drift time */
/* Continuous read-out (Sec. 5): the collision time is unknown before
 * tracking, so a timeframe is tracked with z replaced by the drift
 * coordinate z_t = v_d (t_collision - t_frame) + z_max - |z|, the collision
 * times are estimated from the tracks, and z_t is then converted to space.
 * Reading: a track extrapolated to its closest approach to the beam axis
 * gives t = (z_t - z_max) / v_d; tracks with |distance| <= dca_max, at least
 * min_clusters clusters, a z_t change of at most ext_max in the
 * extrapolation and a pT of at least min_pt_gev (0: no cut; above the
 * looping momentum it keeps the further legs of loopers out) take part; sorted in t they are cut wherever neighbours are
 * more than gap apart; runs of at least min_tracks tracks are vertices with
 * the mean t of their tracks; their tracks get z = side (z_max - (z_t -
 * v_d t_vertex)) at the innermost row (side +1 for sectors 0..17, -1 for
 * 18..35) and dz/ds_T = -side t. */
typedef struct {
  double vdrift_cm_us;  /* drift velocity; 2.5 */
  double zmax_cm;       /* drift length; 250 */
  double dca_max_cm;    /* largest transverse distance to the beam axis; 2 */
  double ext_max_cm;    /* largest z_t change of the extrapolation; 300 */
  double gap_us;        /* time gap that separates vertices; 0.5 */
  int32_t min_tracks;   /* tracks of a vertex; 3 */
  int32_t min_clusters; /* clusters of a participating track; 20 */
  double min_pt_gev;    /* smallest pT of a participating track; 0 (none) */
} tpc_vertex_config;

typedef struct {
  double time_us;   /* mean time estimate of its tracks (frame time, us) */
  int32_t n_tracks; /* tracks assigned */
  int32_t request;  /* request index (0) */
} tpc_vertex;

int tpc_default_vertex_config(tpc_vertex_config *cfg);

/* On the fitted tracks of the loaded request (one request per call;
 * TPC_EINVAL otherwise or before tpc_fit_tracks).  cfg NULL: defaults.
 * Asynchronous; results with tpc_get_vertices. */
int tpc_find_vertices(tpc_ctx *ctx, const tpc_vertex_config *cfg);

/* Waits and copies: vertices in time order (out: room for cap; *n_out the
 * count; TPC_EOVERFLOW without copying when cap is too small, or when the
 * tracks' time range exceeds the reserved 2^18 bins of gap/2), and per track
 * (optional, n_tracks entries each): vertex index or -1, time estimate (us),
 * spatial z (cm; NaN without a vertex) and spatial dz/ds_T. */
int tpc_get_vertices(tpc_ctx *ctx, tpc_vertex *out, int64_t cap, int64_t *n_out, int32_t *track_vertex,
                     float *track_time, float *track_z, float *track_tgl);

/* ------------------------------------------------ track-model compression */
/* The compression section's track-model coding: each selected track is
 * refitted over its own clusters, outermost first; at each cluster the
 * residual between the fixed-point cluster (rint(v / unit), binary32) and
 * the rounded extrapolated track position is stored, and the fit is updated
 * with the fixed-point value; decompression repeats the same fit from the
 * same header and adds the residuals back, which restores every fixed-point
 * cluster exactly.  The paper's distortion transform is the identity here.
 * A track whose fit stops at the |sin phi| limit (ok = 0) carries its
 * fixed-point clusters in the residual streams instead. */
typedef struct {
  float par[5];        /* y, z, sin phi, dz/ds_T, q/pT where the fit starts (the outermost cluster's row) */
  int32_t row_out;     /* that row */
  int32_t n_clusters;  /* the track's clusters */
  int32_t ok;          /* 1: residuals; 0: fixed-point clusters */
} tpc_codec_header;

/* Encode the fitted tracks of the loaded batch (after tpc_fit_tracks).
 * Asynchronous; results with tpc_get_compressed. */
int tpc_compress(tpc_ctx *ctx, double unit_cm);

/* Waits and copies: per track its header (tpc_get_tracks order); per cluster
 * (tracks in that order, each outermost first) its row, residuals and --
 * optional -- the fixed-point coordinates that were encoded.  Any pointer
 * may be NULL; *n_tracks and *n_clusters receive the sizes (TPC_EOVERFLOW
 * without copying when a capacity is too small). */
int tpc_get_compressed(tpc_ctx *ctx, tpc_codec_header *heads, int64_t cap_tracks, uint8_t *rows, int32_t *res_y,
                       int32_t *res_z, int32_t *q_y, int32_t *q_z, int64_t cap_clusters, int64_t *n_tracks,
                       int64_t *n_clusters);

/* Decode n_tracks tracks (host headers and streams, the layout of
 * tpc_get_compressed) into fixed-point clusters q_y, q_z (host, n_clusters
 * each), on the context's device with its configuration (the field and the
 * FP64-zone length must be the encoder's).  Synchronous.  TPC_EINVAL when
 * the headers' counts do not add up to n_clusters or a track's rows do not
 * lie at or below its row_out. */
int tpc_decompress(tpc_ctx *ctx, const tpc_codec_header *heads, int64_t n_tracks, const uint8_t *rows,
                   const int32_t *res_y, const int32_t *res_z, int64_t n_clusters, double unit_cm, int32_t *q_y,
                   int32_t *q_z);

/* ------------------------------------- merging sector segments (phase 2) */
/* Sec. 2's second phase: the segments the sector tracker found in different
 * sectors are merged into final tracks and refitted.  Reading: an inner
 * segment A and an outer segment B in neighbouring sectors of one side
 * (A's first row below B's, A's last row at most overlap_rows past B's first)
 * are compared at B's first row -- A's fitted state and covariance turned
 * into B's frame and carried there; if their z there differ by at most
 * window_cm (a bound that lets the search visit only segments near the
 * predicted z), chi2 = d^T (C_A + C_B)^-1 d over the five parameters; a pair
 * within chi2_max that is the best choice of both is merged.  Chains of merges are refitted from the outermost segment's refit
 * seed inward over all their clusters, the frame turned between segments
 * (the FP64 zone as in the refit); a merged track is given at its innermost
 * cluster in the innermost segment's frame.  Segments with a failed refit or
 * fewer than min_clusters clusters take no part. */
typedef struct {
  double chi2_max;      /* 25 */
  int32_t overlap_rows; /* 10 */
  int32_t min_clusters; /* 10 */
  double window_cm;     /* 10; 1e-3 .. 1e6 */
} tpc_merge_config;

int tpc_default_merge_config(tpc_merge_config *cfg);

/* On the fitted tracks of the loaded batch (after tpc_fit_tracks); cfg NULL:
 * defaults.  Asynchronous; results with tpc_get_merged. */
int tpc_merge_tracks(tpc_ctx *ctx, const tpc_merge_config *cfg);

/* Waits and copies the merged tracks (tpc_track records, in the order of
 * their innermost segments: par/cov/chi2/ndf/n_clusters of the merged fit,
 * sector/request and first_row of the innermost segment, last_row of the
 * outermost, reserved = segments, cluster_offset = index of the innermost
 * segment among the tracks of tpc_get_tracks, flags TPC_TF_REFIT_FAIL if
 * the merged fit stopped); and per segment (optional, n_tracks entries
 * each): its merged outer partner or -1, its merged track or -1, the chi2 of
 * its best outer candidate and the second-best chi2 (infinity: none). */
int tpc_get_merged(tpc_ctx *ctx, tpc_track *out, int64_t cap, int64_t *n_out, int32_t *track_link,
                   int32_t *track_chain, float *pair_chi2, float *pair_second);

/* ------------------------------------------------------- cluster rejection */
/* The compression section: before compression, the clusters of tracks that
 * physics does not use are dropped (about half of all clusters in the
 * paper's data).  Reading, per fitted sector track (its state at the
 * innermost row): class TPC_RJ_LOW_P if its momentum sqrt(1 + t^2)/|q/pT|
 * is below p_min_gev; TPC_RJ_INCLINED if |dz/ds_T| is above tgl_max;
 * TPC_RJ_LOOPER_LEG if it is a looper (its circle's farthest point from the
 * beam axis inside the outermost row radius) and its z at its closest
 * approach to the beam axis lies more than dz_leg_cm from the collision --
 * z_ref_cm for an event, or (use_vertices = 1, continuous read-out) the
 * nearest vertex found by tpc_find_vertices on the current fit, the
 * distance then being v_drift |t_track - t_vertex|.  Every leg of a helix
 * from the collision passes the axis again after each full turn with z
 * moved by 2 pi R dz/ds_T, so only a first leg points back to the collision.
 * A track with any class is rejected, and so are its clusters; clusters of
 * no track are kept. */
typedef struct {
  double p_min_gev;     /* 0.05 */
  double tgl_max;       /* 2.0 */
  double dz_leg_cm;     /* 10 */
  double z_ref_cm;      /* 0 */
  int32_t use_vertices; /* 0 */
  int32_t reserved;
} tpc_reject_config;

enum { TPC_RJ_LOW_P = 1, TPC_RJ_INCLINED = 2, TPC_RJ_LOOPER_LEG = 4 };

int tpc_default_reject_config(tpc_reject_config *cfg);

/* On the fitted tracks of the loaded batch (after tpc_fit_tracks); cfg NULL:
 * defaults.  TPC_EINVAL before a fit, for a bad configuration, or for
 * use_vertices without vertices of the current fit.  Asynchronous; results
 * with tpc_get_rejection. */
int tpc_reject_clusters(tpc_ctx *ctx, const tpc_reject_config *cfg);

/* Waits and copies (each optional): per track its class bits (n_tracks
 * entries, the order of tpc_get_tracks), per loaded cluster its keep flag
 * (1: stays; n_clusters entries, input order), and counts[4] = clusters
 * rejected in all, of class LOW_P, INCLINED, LOOPER_LEG (a cluster of a
 * track with several classes counts in each of them). */
int tpc_get_rejection(tpc_ctx *ctx, uint8_t *track_class, uint8_t *cluster_keep, int64_t *counts);

/* ------------------------------------------------------ serving (requests) */
/* Continuous-batching request loop: the serving form of tracking several
 * events or continuous-readout timeframes (Sec. 2, Sec. 5) as they arrive.
 * A server owns max_slots tracker contexts, each on its own CUDA stream of
 * device `device`, and one worker thread.  Requests wait in submission
 * order; the worker admits the head of the queue as soon as a slot is free
 * and that slot's arena for the request (tpc_arena_bytes(n, 1)) fits both
 * hbm_budget (bytes summed over all slots; 0: no budget) and the device's
 * free memory, so requests admitted while others run overlap on the GPU.
 * Slots keep their arenas (grid, links, tracklets, tracks) across requests
 * and only grow them; idle slots drop theirs when the budget would block the
 * head of the queue.  Each request runs the same graph as tpc_run_graph, so
 * its result equals the one it gets alone.  queue_cap: requests that may
 * wait (admitted ones excluded).  Errors: TPC_EINVAL for bad arguments,
 * TPC_ECUDA when a stream or context cannot be created. */
typedef struct tpc_server tpc_server;
int tpc_server_create(tpc_server **out, const tpc_config *cfg, int device, int32_t max_slots, size_t hbm_budget,
                      int32_t queue_cap);

/* Queue n clusters (host memory, one request) under a caller-chosen id that
 * no pending request uses.  Results go straight to the caller's buffers:
 * tracks_out (room for cap tracks; a track owns at least n_min_track
 * clusters, so n / n_min_track + 1 always suffices) and cluster_track_out
 * (n entries, or NULL), as tpc_get_tracks writes them.  All three buffers
 * must stay valid, and the input unchanged, until tpc_server_poll reports
 * the request finished or failed; page-locked buffers let the copies run
 * while other requests compute.  TPC_EBUSY: the queue is full (retry
 * later).  TPC_ENOMEM: the request alone exceeds the budget.  TPC_EINVAL:
 * bad argument or an id in use. */
int tpc_server_submit(tpc_server *srv, int64_t request_id, const tpc_cluster *clusters, int64_t n,
                      tpc_track *tracks_out, int64_t cap, int32_t *cluster_track_out);

/* *state: 0 queued, 1 running, 2 finished, 3 failed, -1 unknown id. */
int tpc_server_poll(tpc_server *srv, int64_t request_id, int *state);

/* Outcome of a finished or failed request, which is then forgotten:
 * *n_tracks (tracks written to tracks_out; the number found when cap was
 * too small), times_ms (optional): [0] queue wait, [1] admission to results
 * in the caller's buffers, [2] submission to results.  Returns the
 * request's status (TPC_OK, or its error: TPC_EOVERFLOW when cap was too
 * small, ...), TPC_EBUSY while it is queued or running (nothing changes),
 * TPC_EINVAL for an unknown id. */
int tpc_server_result(tpc_server *srv, int64_t request_id, int64_t *n_tracks, double times_ms[3]);

/* Wait until no request is queued or running (timeout_s <= 0: no limit);
 * TPC_ETIMEOUT when the limit ran out. */
int tpc_server_drain(tpc_server *srv, double timeout_s);

/* [0] admitted, [1] completed, [2] queued now, [3] arena bytes held by the
 * slots, [4] most requests that ran at the same time. */
int tpc_server_stats(tpc_server *srv, int64_t stats[5]);

/* Stops the worker after its current step (requests still queued are
 * dropped), waits for the slots' streams and frees everything. */
void tpc_server_destroy(tpc_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* TPCCA_H */
