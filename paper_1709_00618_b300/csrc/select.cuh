// a7 selection of good tracks and final cluster assignment (Sec. 2: "the
// selection of good tracks and final assignment of clusters to tracks
// dissolving ambiguities"), and a8 the Kalman refit of every selected track
// on the clusters it owns.
#pragma once
#include "follow.cuh"

namespace tpc {

__device__ __forceinline__ uint64_t track_key(int n, int t) {
  return ((uint64_t)(uint32_t)n << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
}

__global__ void k_zero64(uint64_t* __restrict__ a, const Counts* cn) {
  const int64_t n = cn->n;
  for (int64_t i = gtid(); i < n; i += gstride()) a[i] = 0ull;
}

__global__ void k_fill32(int32_t* __restrict__ a, int32_t v, const Counts* cn) {
  const int64_t n = cn->n;
  for (int64_t i = gtid(); i < n; i += gstride()) a[i] = v;
}

// owner[c] = max key over the tracklets holding c.
__global__ void k_own(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits, KConst kc,
                      uint64_t* __restrict__ owner, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  for (int64_t t = gtid(); t < T; t += gstride()) {
    const int n = f_n[t];
    if (n < kc.n_min_track) continue;
    const uint64_t key = track_key(n, (int)t);
    const int32_t* h = hits + t * NROW;
    for (int i = 0; i < n; i++) atomicMax((unsigned long long*)(owner + h[i]), (unsigned long long)key);
  }
}

// keep[t] = 1 when tracklet t owns at least n_min_track of its clusters.
__global__ void k_keep(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits,
                       const uint64_t* __restrict__ owner, KConst kc, int32_t* __restrict__ keep,
                       int32_t* __restrict__ nown, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  for (int64_t t = gtid(); t < T; t += gstride()) {
    const int n = f_n[t];
    int kept = 0;
    if (n >= kc.n_min_track) {
      const uint64_t key = track_key(n, (int)t);
      const int32_t* h = hits + t * NROW;
      for (int i = 0; i < n; i++) kept += __ldg((const unsigned long long*)owner + h[i]) == key;
    }
    const int k = kept >= kc.n_min_track;
    keep[t] = k;
    nown[t] = k ? kept : 0;
  }
}

// Track numbering in tracklet order; per-cluster assignment in load order.
__global__ void k_assign(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits,
                         const uint64_t* __restrict__ owner, const int32_t* __restrict__ keep,
                         const int32_t* __restrict__ tidx, const int32_t* __restrict__ perm,
                         int32_t* __restrict__ tl_track, int32_t* __restrict__ track_tl,
                         int32_t* __restrict__ cluster_track, Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  if (gtid() == 0) cn->n_tracks = tidx[T];
  for (int64_t t = gtid(); t < T; t += gstride()) {
    if (!keep[t]) {
      tl_track[t] = -1;
      continue;
    }
    const int idx = tidx[t];
    tl_track[t] = idx;
    track_tl[idx] = (int32_t)t;
    const int n = f_n[t];
    const uint64_t key = track_key(n, (int)t);
    const int32_t* h = hits + t * NROW;
    for (int i = 0; i < n; i++)
      if (__ldg((const unsigned long long*)owner + h[i]) == key) cluster_track[__ldg(perm + h[i])] = idx;
  }
}

// Scatter the owned counts of the tracks (in track order) for the offset scan.
__global__ void k_track_counts(const int32_t* __restrict__ track_tl, const int32_t* __restrict__ nown,
                               int32_t* __restrict__ tcount, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t i = gtid(); i < M; i += gstride()) tcount[i] = nown[track_tl[i]];
}

// a8: refit of each kept track over its owned clusters, outermost to
// innermost, seeded by the follow state carried to the outermost owned row.
__global__ void __launch_bounds__(128) k_refit(GridView g, const int32_t* __restrict__ track_tl,
                                               const int32_t* __restrict__ f_n, const int32_t* __restrict__ f_nf,
                                               const int32_t* __restrict__ f_row, const int32_t* __restrict__ hits,
                                               const uint8_t* __restrict__ hrow, const float* __restrict__ f_par,
                                               const float* __restrict__ f_zref, const float* __restrict__ f_cov,
                                               const double* __restrict__ f_chi2,
                                               const uint64_t* __restrict__ owner,
                                               const int32_t* __restrict__ toff, const int32_t* __restrict__ perm,
                                               KConst kc, tpc_track* __restrict__ out,
                                               int32_t* __restrict__ track_clusters, Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  Tally tally;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const int t = track_tl[m];
    const int n = f_n[t], nf = f_nf[t];
    const uint64_t key = track_key(n, t);
    const int32_t* h = hits + (int64_t)t * NROW;
    const uint8_t* hr = hrow + (int64_t)t * NROW;
    // owned list in update order (outermost first): forward hits descending,
    // then backward-extension hits in stored (descending-row) order
    int order_cnt = 0;
    int r_out = -1, r_in = NROW;
    for (int i = nf - 1; i >= 0; i--)
      if (__ldg((const unsigned long long*)owner + h[i]) == key) {
        r_out = max(r_out, (int)hr[i]);
        r_in = min(r_in, (int)hr[i]);
        order_cnt++;
      }
    for (int i = nf; i < n; i++)
      if (__ldg((const unsigned long long*)owner + h[i]) == key) {
        r_out = max(r_out, (int)hr[i]);
        r_in = min(r_in, (int)hr[i]);
        order_cnt++;
      }
    const int rs_any = __ldg(g.rs_of + h[0]);
    const int unit = rs_any / NROW;
    uint32_t flags = 0;
    Filter f;
    f.tally = &tally;
    f.seed(f_row[t], sX[f_row[t]], f_par[t * 5 + 0], f_zref[t], f_par[t * 5 + 2], f_par[t * 5 + 3],
           f_par[t * 5 + 4]);
    f.p.z = f_par[t * 5 + 1];
    f.reset_cov(kc);
    bool ok = true;
    const int step = r_out >= f.p.row ? 1 : -1;
    for (int r = f.p.row + step; ok && (step > 0 ? r <= r_out : r >= r_out); r += step)
      ok = f.propagate(r, sX[r], kc, flags, false);
    if (ok) {
      f.reset_cov(kc);
      // update order j = 0..n-1 visits slot nf-1-j for j < nf (forward hits,
      // rows descending) and slot j after that (backward hits, rows
      // descending); rows strictly decrease along it
      int j = 0, cur = -1;
      for (; j < n; j++) {
        const int slot = j < nf ? nf - 1 - j : j;
        if (__ldg((const unsigned long long*)owner + h[slot]) == key) {
          cur = slot;
          break;
        }
      }
      for (int r = r_out; ok && r >= r_in; r--) {
        if (r != r_out) ok = f.propagate(r, sX[r], kc, flags);
        if (ok && cur >= 0 && hr[cur] == r) {
          const float2 P = __ldg(g.yz + h[cur]);
          f.update(P.x, P.y, kc);
          cur = -1;
          for (j++; j < n; j++) {
            const int slot = j < nf ? nf - 1 - j : j;
            if (__ldg((const unsigned long long*)owner + h[slot]) == key) {
              cur = slot;
              break;
            }
          }
        }
      }
    }
    tpc_track tr;
    if (ok) {
      tr.x = sX[r_in];
      tr.par[0] = f.p.y + f.p.yl;
      tr.par[1] = f.p.zref + (f.p.z + f.p.zl);
      tr.par[2] = f.p.s + f.p.sl;
      tr.par[3] = f.p.t;
      tr.par[4] = f.p.q;
      f.cov_out(tr.cov);
      tr.chi2 = f.chi2;
      tr.first_row = r_in;
    } else {
      const int fr = f_row[t];
      tr.x = sX[fr];
      tr.par[0] = f_par[t * 5 + 0];
      tr.par[1] = f_zref[t] + f_par[t * 5 + 1];
      tr.par[2] = f_par[t * 5 + 2];
      tr.par[3] = f_par[t * 5 + 3];
      tr.par[4] = f_par[t * 5 + 4];
      for (int j = 0; j < 15; j++) tr.cov[j] = f_cov[t * 15 + j];
      tr.chi2 = f_chi2[t];
      tr.first_row = fr;
      flags = TF_REFIT_FAIL;
    }
    tr.reserved = 0;
    tr.ndf = 2 * order_cnt - 5;
    tr.n_clusters = order_cnt;
    tr.sector = unit % NSEC;
    tr.request = unit / NSEC;
    tr.last_row = r_out;
    tr.cluster_offset = toff[m];
    tr.flags = (int32_t)flags;
    out[m] = tr;
    // owned clusters in load order, innermost row first: backward list from
    // its end, then forward list from its start
    if (track_clusters) {
      int w = toff[m];
      for (int j = n - 1; j >= nf; j--)
        if (__ldg((const unsigned long long*)owner + h[j]) == key) track_clusters[w++] = __ldg(perm + h[j]);
      for (int j = 0; j < nf; j++)
        if (__ldg((const unsigned long long*)owner + h[j]) == key) track_clusters[w++] = __ldg(perm + h[j]);
    }
  }
  tally.flush(cn);
}

}  // namespace tpc
