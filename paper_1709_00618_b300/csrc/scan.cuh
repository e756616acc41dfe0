// Device-wide exclusive prefix sum of int32 counts (reduce, scan partials,
// down-sweep).  The length is read from device memory so the same launches
// serve any batch inside a captured graph.  out[len] receives the total.
#pragma once
#include "common.cuh"

namespace tpc {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SCAN_PARTS = 296;  // 2 per SM on 148 SMs

struct LenSrc {
  const int32_t* dev;  // if non-null: length = *dev + add
  int64_t host;        // otherwise: length = host
  int32_t add;
  __device__ __forceinline__ int64_t get() const { return dev ? (int64_t)(*dev) + add : host; }
};

// Inclusive scan over a block of SCAN_THREADS threads; returns the inclusive
// prefix of this thread's value and the block total.
__device__ __forceinline__ int block_incl_scan(int v, int* warp_sums, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_sums[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (SCAN_THREADS / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += t;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  total = warp_sums[SCAN_THREADS / 32 - 1];
  int r = v + (warp > 0 ? warp_sums[warp - 1] : 0);
  __syncthreads();
  return r;
}

__device__ __forceinline__ void chunk_of(int64_t len, int64_t& a, int64_t& b) {
  int64_t per = (len + gridDim.x - 1) / gridDim.x;
  per = (per + SCAN_TILE - 1) / SCAN_TILE * SCAN_TILE;
  a = (int64_t)blockIdx.x * per;
  b = a + per < len ? a + per : len;
  if (a > len) a = len;
}

// The whole scan in one block, tile after tile with a running carry: for
// short arrays (a few tiles), where the three-kernel scan's launches cost
// more than the work.  out may alias in; out[len] = total.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_small(const int32_t* in, LenSrc L, int32_t* out,
                                                             int32_t* total_out, const Counts* cn) {
  __shared__ int ws[32];
  if (fatal(cn)) return;
  const int64_t len = L.get();
  int carry = 0;
  for (int64_t base = 0; base < len; base += SCAN_TILE) {
    int v[SCAN_ITEMS], sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      const int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
      v[k] = i < len ? in[i] : 0;
      sum += v[k];
    }
    int tot;
    int run = carry + block_incl_scan(sum, ws, tot) - sum;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      const int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
      if (i < len) out[i] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    out[len] = carry;
    if (total_out) *total_out = carry;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t* __restrict__ in, LenSrc L,
                                                              int32_t* __restrict__ part, const Counts* cn) {
  __shared__ int ws[32];
  if (fatal(cn)) return;
  int64_t len = L.get(), a, b;
  chunk_of(len, a, b);
  int acc = 0;
  for (int64_t i = a + threadIdx.x; i < b; i += SCAN_THREADS) acc += in[i];
  int tot;
  block_incl_scan(acc, ws, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_parts(int32_t* part, int n_parts, int32_t* total_out,
                                                     const Counts* cn) {
  __shared__ int ws[32];
  if (fatal(cn)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int v = threadIdx.x < n_parts ? part[threadIdx.x] : 0, x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += t;
    }
    ws[lane] = w;
  }
  __syncthreads();
  int incl = x + (warp > 0 ? ws[warp - 1] : 0);
  if (threadIdx.x < n_parts) part[threadIdx.x] = incl - v;
  if (threadIdx.x == 0 && total_out) *total_out = ws[31];
}

// out may alias in.  out[len] = total (written by the block owning the end).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int32_t* in, LenSrc L,
                                                            const int32_t* __restrict__ part, int32_t* out,
                                                            const Counts* cn) {
  __shared__ int ws[32];
  if (fatal(cn)) return;
  int64_t len = L.get(), a, b;
  chunk_of(len, a, b);
  int carry = part[blockIdx.x];
  for (int64_t base = a; base < b; base += SCAN_TILE) {
    int64_t i0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      v[k] = (i0 + k < b) ? in[i0 + k] : 0;
      s += v[k];
    }
    int tot;
    int incl = block_incl_scan(s, ws, tot);
    int run = carry + incl - s;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
      if (i0 + k < b) out[i0 + k] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (b == len && a < b) out[len] = carry;
  if (len == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

}  // namespace tpc
