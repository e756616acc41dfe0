// Shared device definitions of the sector tracker kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tpcca.h"

namespace tpc {

constexpr int NROW = 159;
constexpr int NSEC = 36;

// Device status word bits (host reads them at tpc_sync / tpc_get_*).
enum : uint32_t {
  ST_EINVAL = 1u,     // a cluster failed validation
  ST_EOVERFLOW = 2u,  // a capacity was exceeded (grid bins, tracklets)
  ST_ETIMEOUT = 4u,   // a bounded wait ran out
};

// Per row-sector grid parameters, 32 bytes (one sector-sized load).
struct __align__(16) RsParams {
  float z_lo, z_hi, inv_y, inv_z;
  int32_t n_y, n_z, bin_base, count;
};

// Hint: bring the line holding p into L1 ahead of its use (no register, no
// fault on any address).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Read-only 32-byte load of a row-sector's parameters.
__device__ __forceinline__ RsParams load_params(const RsParams* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
  RsParams r;
  r.z_lo = a.x;
  r.z_hi = a.y;
  r.inv_y = a.z;
  r.inv_z = a.w;
  r.n_y = b.x;
  r.n_z = b.y;
  r.bin_base = b.z;
  r.count = b.w;
  return r;
}

constexpr int PH_COUNT_MAX = 10;  // Kalman kernels with work counters (PH_*, below)

// Scalars of a run that live in device memory so that graph-captured
// kernels read the sizes of whatever batch is loaded.
struct Counts {
  int64_t n;          // clusters
  int32_t n_req;      // requests
  int32_t n_rs;       // row-sectors = n_req * 36 * 159
  int32_t n_bins;     // total grid bins
  int32_t n_tracklets;
  int32_t n_tracks;
  uint32_t status;    // ST_* bits
  int32_t n_track_clusters;
  int32_t n32;         // clusters as int32 (length source of the per-cluster scans)
  int32_t work_next[20];  // work counters of the persistent Kalman kernels, [fetch phase x chunk]
  int32_t zone_pend[6];   // items deferred to a zone tail kernel, [pass x chunk] (follow.cuh)
  // work counters of the follow (a6) and refit (a8) kernels
  unsigned long long n_prop;    // helix propagations with covariance transport
  unsigned long long n_upd32;   // FP32 Kalman updates
  unsigned long long n_upd64;   // FP64-zone Kalman updates
  unsigned long long n_cand;    // candidate clusters examined by the gated pick-up
  unsigned long long n_prop64;  // propagations done with the FP64 covariance
  int32_t trace_n;              // trace records written
  int32_t n_starts;             // chain starts (clusters with a kept upward link and none downward)
  unsigned long long pad2[2];
  // the same counters per Kalman kernel (PH_*): {prop, upd32, upd64, cand, prop64}
  unsigned long long phase_work[PH_COUNT_MAX][5];
};

// Kalman kernels, in launch order: their work counters (one per chunk) and
// their tallies.  A kernel that a batch's size does not launch (the zone
// tails, phase 4r) keeps zero work.
enum {
  PH_FOLLOW_P1 = 0,
  PH_FOLLOW_P1T,
  PH_FOLLOW_P2,
  PH_FOLLOW_P3,
  PH_FOLLOW_P3T,
  PH_FOLLOW_P4R,
  PH_FOLLOW_P4,
  PH_REFIT_P1,
  PH_REFIT_P1T,
  PH_REFIT_P2,
  PH_COUNT
};
constexpr int PH_FETCH = PH_COUNT;  // work counters per chunk

// The Kalman stage may split its items into chunks whose zone and FP32
// kernels run concurrently on two streams (the FP64 pipe of one chunk's
// zone beside the other's FP32 work); chunk c of nc covers [begin, end).
constexpr int MAX_CHUNKS = 2;
static_assert(PH_FETCH * MAX_CHUNKS <= (int)(sizeof(((Counts*)nullptr)->work_next) / sizeof(int32_t)),
              "a work counter per Kalman kernel and chunk");
static_assert(PH_COUNT == PH_COUNT_MAX,
              "tallies per Kalman kernel");
struct Chunk {
  int32_t begin, end;
};
__device__ __forceinline__ Chunk chunk_range(int32_t n, int c, int nc) {
  return {(int32_t)((int64_t)n * c / nc), (int32_t)((int64_t)n * (c + 1) / nc)};
}
__device__ __forceinline__ int32_t* work_counter(Counts* cn, int phase, int c) {
  return &cn->work_next[phase * MAX_CHUNKS + c];
}

// Per-thread work tallies, flushed once per thread into Counts.
struct Tally {
  unsigned long long prop = 0, upd32 = 0, upd64 = 0, cand = 0, prop64 = 0;
  __device__ __forceinline__ void flush(Counts* cn, int phase) {
    unsigned long long* w = cn->phase_work[phase];
    if (prop) atomicAdd(&cn->n_prop, prop), atomicAdd(&w[0], prop);
    if (upd32) atomicAdd(&cn->n_upd32, upd32), atomicAdd(&w[1], upd32);
    if (upd64) atomicAdd(&cn->n_upd64, upd64), atomicAdd(&w[2], upd64);
    if (cand) atomicAdd(&cn->n_cand, cand), atomicAdd(&w[3], cand);
    if (prop64) atomicAdd(&cn->n_prop64, prop64), atomicAdd(&w[4], prop64);
  }
};

// Algorithm constants passed by value to every kernel (kernel parameter
// space is read through the constant cache).
struct KConst {
  float K;          // 0.299792458e-3 * Bz[kG]
  float V;          // sigma^2
  double Vd;
  float d_max;
  float wy, wz;     // link windows (one row)
  float wy2, wz2;   // link windows two rows away (link_skip)
  int32_t link_skip;
  float gate;
  float c0[5];
  float s_max;
  float edge;
  float taint;      // divergence margin
  int32_t min_chain, max_miss, n_min_track, fp64_updates;
  int64_t bins_cap, tl_cap;
  // per-update trace of one tracklet (trace_t < 0: off)
  int32_t trace_t;
  int32_t trace_cap;
  float* trace;  // trace_cap records of TRACE_W floats
  // lanes of a warp of a refilling Kalman kernel that must be idle before
  // the warp fetches new work for them together (1: refill at once)
  int32_t refill;
  // row steps a refilling Kalman kernel's lanes take between the warp's
  // refill checks (16 on inputs bound by the longest tracklet: fewer
  // warp-wide votes; 4 on large inputs, where lanes idle until the check)
  int32_t inner_steps;
  // row steps the zone kernels take with a warp's 32 tracklets in step,
  // [follow forward, follow backward, refit]; a zone still open after them
  // goes on in the zone tail kernel (0: no limit), whose list holds up to
  // zone_tail_cap items per pass
  int32_t zone_steps[3];
  int64_t zone_tail_cap;
};

// Trace record: pass (0 forward, 1 backward), row, updates since seed, then
// y, z (absolute), sin phi, dz/ds, q/pT, C_yy, C_zz, C_ss, C_tt, C_qq, chi2,
// residual y, residual z.
constexpr int TRACE_W = 16;

// Row radii X_r and active half-widths Y_r in binary32 (set once per device;
// the library is a single translation unit).
__device__ float g_row_x[NROW + 1];
__device__ float g_row_yhi[NROW + 1];

__device__ __forceinline__ bool fatal(const Counts* cn) {
  return (*(volatile const uint32_t*)&cn->status) & (ST_EINVAL | ST_EOVERFLOW | ST_ETIMEOUT);
}

// Monotone map float -> uint32 so that unsigned min/max order equals float order.
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// Grid-stride helper bounds.
__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

}  // namespace tpc
