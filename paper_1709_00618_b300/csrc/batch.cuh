// Per-request views of a batch's results (tpc_submit_batch / tpc_poll).
// Tracks are numbered in the order of their tracklets, which follow the
// sorted (request, sector, row, bin, input index) order, so the tracks of
// one request are contiguous; these kernels find each request's range and
// turn the batch's cluster->track indices into request-local ones.
#pragma once
#include "common.cuh"

namespace tpc {

// req_trk[2q] = first track of request q, req_trk[2q+1] = one past its last
// (both 0 for a request without tracks; the caller clears the array).
__global__ void k_req_tracks(const tpc_track* __restrict__ tracks, int32_t* __restrict__ req_trk,
                             const Counts* __restrict__ cn) {
  if (fatal(cn)) return;
  const int32_t m = cn->n_tracks;
  for (int64_t t = gtid(); t < m; t += gstride()) {
    const int32_t q = tracks[t].request;
    if (t == 0 || tracks[t - 1].request != q) req_trk[2 * q] = (int32_t)t;
    if (t == m - 1 || tracks[t + 1].request != q) req_trk[2 * q + 1] = (int32_t)t + 1;
  }
}

// out[i] = the request-local track index of cluster i (load order), -1 when
// it is unassigned.
__global__ void k_req_rebase(const int32_t* __restrict__ cluster_track, const int64_t* __restrict__ req_off,
                             const int32_t* __restrict__ req_trk, int32_t* __restrict__ out,
                             const Counts* __restrict__ cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  const int n_req = cn->n_req;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {  // the last request whose first cluster is at or before i
      const int mid = (lo + hi + 1) >> 1;
      if (req_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const int32_t k = cluster_track[i];
    out[i] = k >= 0 ? k - req_trk[2 * lo] : -1;
  }
}

}  // namespace tpc
