// Longest-first work order of the refilling Kalman kernels.  A refilling
// kernel ends when the last tracklet it fetched ends, so tracklets are
// handed out in decreasing order of the rows they can still cross: the
// producing kernel files each item under its remaining-row class (a
// warp-aggregated histogram), k_order turns the classes into positions, and
// the refilling kernel fetches order[0], order[1], ...  Every item is
// independent, so the order changes no result.  On inputs that fill the GPU
// the follow kernels take tracklets in index order instead (no order[]):
// indices follow the clusters' (request, sector, row) order, so the
// tracklets in flight share a few sectors' clusters, which then stay in L2,
// and the tail of the kernel is short against its length.
#pragma once
#include "common.cuh"

namespace tpc {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int ORD_BINS = NROW + 1;           // remaining-row classes (0: longest)
constexpr int ORD_PHASES = 3;                // follow p2, follow p4, refit p2
constexpr int ORD_WORDS = ORD_PHASES * MAX_CHUNKS * 2 * ORD_BINS;

struct WorkOrder {
  int32_t* hist;    // [ORD_BINS] items per class
  int32_t* cursor;  // [ORD_BINS] items placed per class
  uint8_t* key;     // [items] class of each item
  int32_t* order;   // [items] item indices, longest first
};

// Files item i (lanes with valid) under the class of `rem` remaining rows.
// All lanes of `mask` make the call.
__device__ __forceinline__ void order_count(const WorkOrder& o, int64_t i, bool valid, int rem,
                                            unsigned mask = FULL_MASK) {
  if (!o.key) return;  // index order
  const int b = NROW - 1 - min(max(rem, 0), NROW - 1);
  if (valid) o.key[i] = (uint8_t)b;
  const unsigned peers = __match_any_sync(mask, valid ? b : -1);
  if (valid && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&o.hist[b], __popc(peers));
}

// Positions of the items of chunk c of nc: the exclusive prefix of the
// chunk's class histogram plus a warp-aggregated running count per class,
// within the chunk's own range of order[].
__global__ void k_order(WorkOrder o, const int32_t* __restrict__ n_items, int c, int nc, const Counts* cn) {
  // after an overflow the item count exceeds the capacities: do nothing, as
  // every kernel of the pipeline
  if (fatal(cn)) return;
  __shared__ int32_t pre[ORD_BINS];
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int b = 0; b < ORD_BINS; b++) {
      pre[b] = s;
      s += o.hist[b];
    }
  }
  __syncthreads();
  const Chunk ch = chunk_range(*n_items, c, nc);
  const int32_t N = ch.end - ch.begin;
  const int lane = threadIdx.x & 31;
  for (int64_t base = gtid() - lane; base < N; base += gstride()) {
    const int64_t i = ch.begin + base + lane;
    const bool valid = base + lane < N;
    const int b = valid ? o.key[i] : -1;
    const unsigned peers = __match_any_sync(FULL_MASK, b);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (valid && lane == leader) pos = atomicAdd(&o.cursor[b], __popc(peers));
    pos = __shfl_sync(FULL_MASK, pos, leader);
    if (valid) o.order[ch.begin + pre[b] + pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

}  // namespace tpc
