// a7 selection of good tracks and final cluster assignment (Sec. 2: "the
// selection of good tracks and final assignment of clusters to tracks
// dissolving ambiguities"), and a8 the Kalman refit of every selected track
// on the clusters it owns.
#pragma once
#include "follow.cuh"

namespace tpc {

// Ownership key of tracklet t with n clusters: the larger key wins a
// cluster, i.e. more clusters first, then the lower tracklet id.  64-bit:
// n << 32 | (2^32 - 1 - t).  32-bit, while the tracklet capacity is below
// 2^24 (n <= 159 < 2^8): n << 24 | (2^24 - 1 - t) -- the same order, half
// the bytes and atomics of half the width.
template <typename Key>
__device__ __forceinline__ Key track_key(int n, int t);
template <>
__device__ __forceinline__ uint64_t track_key<uint64_t>(int n, int t) {
  return ((uint64_t)(uint32_t)n << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
}
template <>
__device__ __forceinline__ uint32_t track_key<uint32_t>(int n, int t) {
  return ((uint32_t)n << 24) | (0xFFFFFFu - (uint32_t)t);
}

__device__ __forceinline__ void key_max(uint64_t* a, uint64_t k) {
  atomicMax((unsigned long long*)a, (unsigned long long)k);
}
__device__ __forceinline__ void key_max(uint32_t* a, uint32_t k) { atomicMax((unsigned int*)a, (unsigned int)k); }

// Hits a thread-per-tracklet selection kernel (k_keep, k_assign) loads at
// once: SEL_BATCH independent loads in flight instead of one dependent chain.
constexpr int SEL_BATCH = 8;

// owner[c] = max key over the tracklets holding c.  W: one warp per
// tracklet, the lanes over its hits (coalesced hit loads, 32 atomics in
// flight; faster while the owner array is L2-resident); else one thread per
// tracklet (a warp's 32 atomics then fall on neighbouring tracklets' rows:
// better DRAM locality on inputs far larger than L2).
template <bool W, typename Key>
__global__ void k_own(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits, KConst kc,
                      Key* __restrict__ owner, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  const int lane = W ? (int)(threadIdx.x & 31) : 0, step = W ? 32 : 1;
  for (int64_t t = W ? gtid() >> 5 : gtid(); t < T; t += W ? gstride() >> 5 : gstride()) {
    const int n = f_n[t];
    if (n < kc.n_min_track) continue;
    const Key key = track_key<Key>(n, (int)t);
    const int32_t* h = hits + t * NROW;
    // owner keys only grow, so a read through the non-coherent cache that
    // already shows a key at least ours (possibly an older, smaller one would
    // only cost an atomic) means this tracklet cannot win that cluster
    for (int i = lane; i < n; i += step) {
      Key* o = owner + h[i];
      if (__ldg(o) < key) key_max(o, key);
    }
  }
}

// keep[t] = 1 when tracklet t owns at least n_min_track of its clusters;
// for kept tracklets also the bit mask of owned hit slots (5 words) and the
// owned row range (r_in | r_out << 16), so that the refit and the output
// stage need no ownership loads.
constexpr int OWN_WORDS = 5;
// W: one warp per tracklet, lanes over its hits (below 4 Mi clusters);
// else one thread per tracklet, so that a warp's loads of hit i of 32
// consecutive tracklets fall on one row, close together (as k_own).
template <bool W, typename Key>
__global__ void k_keep(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits,
                       const uint8_t* __restrict__ hrow, const Key* __restrict__ owner, KConst kc,
                       int32_t* __restrict__ keep, int32_t* __restrict__ nown, uint32_t* __restrict__ own_mask,
                       int32_t* __restrict__ own_rng, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  if (!W) {
    for (int64_t t = gtid(); t < T; t += gstride()) {
      const int n = f_n[t];
      int kept = 0;
      unsigned r_in = NROW, r_out = 0;
      if (n >= kc.n_min_track) {
        const Key key = track_key<Key>(n, (int)t);
        const int32_t* h = hits + t * NROW;
        const uint8_t* hr = hrow + t * NROW;
        uint32_t* m = own_mask + t * OWN_WORDS;
        for (int w = 0; w < OWN_WORDS; w++) {  // 32 hit slots per mask word
          uint32_t word = 0;
          const int i1 = min(n, 32 * (w + 1));
          for (int i0 = 32 * w; i0 < i1; i0 += SEL_BATCH) {  // SEL_BATCH keys in flight, as k_own
            int c[SEL_BATCH];
            bool own[SEL_BATCH];
#pragma unroll
            for (int k = 0; k < SEL_BATCH; k++) c[k] = i0 + k < i1 ? h[i0 + k] : -1;
#pragma unroll
            for (int k = 0; k < SEL_BATCH; k++) own[k] = c[k] >= 0 && __ldg(owner + c[k]) == key;
#pragma unroll
            for (int k = 0; k < SEL_BATCH; k++) {
              if (own[k]) {
                const int i = i0 + k;
                word |= 1u << (i & 31);
                kept++;
                const unsigned r = hr[i];
                r_in = min(r_in, r);
                r_out = max(r_out, r + 1);
              }
            }
          }
          m[w] = word;
        }
      }
      const int k = kept >= kc.n_min_track;
      keep[t] = k;
      nown[t] = k ? kept : 0;
      if (k) own_rng[t] = (int)r_in | (((int)r_out - 1) << 16);
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  for (int64_t t = gtid() >> 5; t < T; t += gstride() >> 5) {  // one warp per tracklet, lanes over hits
    const int n = f_n[t];
    int kept = 0;
    unsigned r_in = NROW, r_out = 0;  // r_out: one past the outermost owned row
    uint32_t mw = 0;                  // lane w < OWN_WORDS: mask word w
    if (n >= kc.n_min_track) {
      const Key key = track_key<Key>(n, (int)t);
      const int32_t* h = hits + t * NROW;
      const uint8_t* hr = hrow + t * NROW;
      for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool own = i < n && __ldg(owner + h[i]) == key;
        const uint32_t b = __ballot_sync(FULL_MASK, own);
        if (lane == (i0 >> 5)) mw = b;
        kept += __popc(b);
        if (own) {
          const unsigned r = hr[i];
          r_in = min(r_in, r);
          r_out = max(r_out, r + 1);
        }
      }
      r_in = __reduce_min_sync(FULL_MASK, r_in);
      r_out = __reduce_max_sync(FULL_MASK, r_out);
    }
    const int k = kept >= kc.n_min_track;
    if (lane == 0) {
      keep[t] = k;
      nown[t] = k ? kept : 0;
      if (k) own_rng[t] = (int)r_in | (((int)r_out - 1) << 16);
    }
    if (k && lane < OWN_WORDS) own_mask[t * OWN_WORDS + lane] = mw;
  }
}

// Load-order indices of each track's owned clusters, innermost row first
// (backward-extension hits from the last stored, then forward hits).
__global__ void k_track_clusters(const int32_t* __restrict__ track_tl, const int32_t* __restrict__ f_n,
                                 const int32_t* __restrict__ f_nf, const int32_t* __restrict__ hits,
                                 const uint32_t* __restrict__ own_mask, const int32_t* __restrict__ toff,
                                 const int32_t* __restrict__ perm, int32_t* __restrict__ track_clusters,
                                 const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const int lane = threadIdx.x & 31;
  for (int64_t m = gtid() >> 5; m < M; m += gstride() >> 5) {  // one warp per track, lanes over slots
    const int t = track_tl[m];
    const int n = f_n[t], nf = f_nf[t];
    const uint32_t mw = lane < OWN_WORDS ? own_mask[t * OWN_WORDS + lane] : 0u;
    const int32_t* h = hits + (int64_t)t * NROW;
    int wpos = toff[m];
    // output position j: slots n-1 .. nf (backward extension, innermost first), then 0 .. nf-1
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const int slot = j < n - nf ? n - 1 - j : j - (n - nf);
      const uint32_t word = __shfl_sync(FULL_MASK, mw, j < n ? slot >> 5 : 0);
      const bool own = j < n && ((word >> (slot & 31)) & 1u);
      const uint32_t b = __ballot_sync(FULL_MASK, own);
      if (own) track_clusters[wpos + __popc(b & ((1u << lane) - 1u))] = __ldg(perm + h[slot]);
      wpos += __popc(b);
    }
  }
}

// Track numbering in tracklet order; per-cluster assignment in load order
// (W: one warp per tracklet, as k_own).  The owned hits are read from the
// bit masks k_keep stored, so the owner keys are not read again.
template <bool W>
__global__ void k_assign(const int32_t* __restrict__ f_n, const int32_t* __restrict__ hits,
                         const uint32_t* __restrict__ own_mask, const int32_t* __restrict__ keep,
                         const int32_t* __restrict__ tidx, const int32_t* __restrict__ perm,
                         const int32_t* __restrict__ nown, int32_t* __restrict__ tl_track,
                         int32_t* __restrict__ track_tl, int32_t* __restrict__ tcount,
                         int32_t* __restrict__ cluster_track, Counts* cn) {
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  if (gtid() == 0) cn->n_tracks = tidx[T];
  const int lane = W ? (int)(threadIdx.x & 31) : 0;
  for (int64_t t = W ? gtid() >> 5 : gtid(); t < T; t += W ? gstride() >> 5 : gstride()) {
    if (!keep[t]) {
      if (lane == 0) tl_track[t] = -1;
      continue;
    }
    const int idx = tidx[t];
    if (lane == 0) {
      tl_track[t] = idx;
      track_tl[idx] = (int32_t)t;
      tcount[idx] = nown[t];  // owned clusters per track, for the offsets of the refit's output
    }
    const int n = f_n[t];
    const int32_t* h = hits + t * NROW;
    if (W) {  // lanes over the hits, the mask words shuffled from the first lanes
      const uint32_t mw = lane < OWN_WORDS ? own_mask[t * OWN_WORDS + lane] : 0u;
      for (int i0 = 0; i0 < n; i0 += 32) {
        const uint32_t word = __shfl_sync(FULL_MASK, mw, i0 >> 5);
        const int i = i0 + lane;
        if (i < n && ((word >> lane) & 1u)) cluster_track[__ldg(perm + h[i])] = idx;
      }
    } else {  // SEL_BATCH owned hits at a time: their indices, then their load-order positions
      for (int w = 0; w < OWN_WORDS; w++) {
        uint32_t word = own_mask[t * OWN_WORDS + w];
        while (word) {
          int c[SEL_BATCH];
#pragma unroll
          for (int k = 0; k < SEL_BATCH; k++) {
            c[k] = -1;
            if (word) {
              c[k] = h[w * 32 + __ffs(word) - 1];
              word &= word - 1;
            }
          }
          int d[SEL_BATCH];
#pragma unroll
          for (int k = 0; k < SEL_BATCH; k++) d[k] = c[k] >= 0 ? __ldg(perm + c[k]) : -1;
#pragma unroll
          for (int k = 0; k < SEL_BATCH; k++)
            if (d[k] >= 0) cluster_track[d[k]] = idx;
        }
      }
    }
  }
}

// a8: refit of each kept track over its owned clusters, outermost to
// innermost, seeded by the follow state carried (state only) to the
// outermost owned row.  The owned hits are visited in update order: forward
// hits from the last to the first, then the backward-extension hits as
// stored; rows strictly decrease along it.
struct RefitLane {
  const int32_t* h;
  const uint8_t* hr;
  int n, nf, j, r_in;
  int cur_row;      // row of the next owned hit (-1: none)
  float2 cur_yz;    // its position
  int nn_row, nn_c; // row (-1: none) and index of the owned hit after it
  uint32_t m[OWN_WORDS];
  const float2* yz;
  __device__ __forceinline__ bool owned(int slot) const {
    uint32_t w = m[0];
#pragma unroll
    for (int k = 1; k < OWN_WORDS; k++)
      if ((slot >> 5) == k) w = m[k];
    return (w >> (slot & 31)) & 1u;
  }
  // The next owned hit in update order (row and position) is loaded ahead
  // of its use.  The FP64 zone (phase 1), bound by its FP64 pipe, loads it
  // in one stage (take: index, then position); the binary32 phase 2, whose
  // row steps wait on their loads, in two (advance): taking a hit issues its
  // successor's position load from an index loaded one take earlier
  // (nn_*), so that no take waits for a load it issues.
  // next_owned: the next owned slot at or after j (-1: none), j past it.
  __device__ __forceinline__ int next_owned() {
    for (; j < n; j++) {
      const int slot = j < nf ? nf - 1 - j : j;
      if (owned(slot)) {
        j++;
        return slot;
      }
    }
    return -1;
  }
  __device__ __forceinline__ void load_after() {
    const int slot = next_owned();
    if (slot >= 0) {
      nn_row = hr[slot];
      nn_c = h[slot];
    } else {
      nn_row = -1;
    }
  }
  // one stage: the next owned hit into cur_*
  __device__ __forceinline__ void take() {
    const int slot = next_owned();
    if (slot >= 0) {
      cur_row = hr[slot];
      cur_yz = __ldg(yz + h[slot]);
    } else {
      cur_row = -1;
    }
  }
  // two stages: the hit in nn_* into cur_*, the one after it into nn_*
  // (after load_after has primed nn_*)
  __device__ __forceinline__ void advance() {
    cur_row = nn_row;
    if (cur_row >= 0) cur_yz = __ldg(yz + nn_c);
    load_after();
  }
};

template <bool Z>
__device__ __forceinline__ bool refit_step(const GridView& g, const KConst& kc, const float* sX, RefitLane& w,
                                           TrkState& p, double* D, float* C, Chi2Acc& chi2, int& nupd, bool& ok,
                                           uint32_t& flags, LocalTally& tl, int& zend, bool& dg) {
  const int r = p.row - 1;
  if (r < w.r_in) return false;
  const bool zone = Z && nupd < zend;
  if (!propagate_any(p, zone, D, C, r, sX[r], kc, flags, Z && dg)) {
    ok = false;
    return false;
  }
  dg = false;
  tl.prop++;
  tl.prop64 += zone;
  if (w.cur_row == r) {
    const float2 P = w.cur_yz;
    chi2.add(zone_update(p, zone, D, C, P.x, P.y, kc, nupd, zend, 2 * kc.fp64_updates));
    if (zone) tl.upd64++;
    else tl.upd32++;
    if (Z) w.take();
    else w.advance();
  }
  return true;
}

// Refit state parked between the two refit phases.
struct RefitWork {
  RefitLane w;
  TrkState p;
  float C[15];
  Chi2Acc chi2;
  int32_t nupd, ok, go, flags, r_out, nown, unit, t, zend;
};

struct RefitIn {
  const int32_t* track_tl;
  const int32_t* f_n;
  const int32_t* f_nf;
  const int32_t* f_row;
  const int32_t* hits;
  const uint8_t* hrow;
  const float* f_par;
  const float* f_zref;
  const float* f_cov;
  const double* f_chi2;
  const uint32_t* own_mask;
  const int32_t* own_rng;
  const int32_t* nown;
  const int32_t* toff;
};

// Zone row steps of one refit lane: up to cap (0: until the zone or the
// refit ends).  True while the refit goes on.
__device__ __forceinline__ bool refit_zone(const GridView& g, const KConst& kc, const float* sX, RefitLane& w,
                                           TrkState& p, double* D, float* C, Chi2Acc& chi2, int& nupd, bool& ok,
                                           uint32_t& flags, LocalTally& tl, int& zend, bool& dg, int cap) {
  bool go = true;
  for (int k = 0; go && nupd < zend && (cap == 0 || k < cap); k++)
    go = refit_step<true>(g, kc, sX, w, p, D, C, chi2, nupd, ok, flags, tl, zend, dg);
  return go;
}

// Phase 1 of the refit: carry the follow state to the outermost owned row
// (state only), then the updates with the covariance in FP64 (the zone's
// first kc.zone_steps[2] rows with a warp's 32 tracks in step, the rest of
// an open zone in the zone tail kernel k_refit_p1t, as the follow stage's
// zone kernels do).
__global__ void __launch_bounds__(128, 4) k_refit_p1(GridView g, RefitIn in, KConst kc, RefitWork* RW, ZoneTail zt,
                                                  WorkOrder next, int chunk, int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const int ZONE = kc.fp64_updates;
  LocalTally tl;
  double D[15];
  float C[15];
  // a warp takes 32 consecutive tracks at a time (lanes past the end idle),
  // so that it can be reconverged before the FP64 zone
  const Chunk ch = chunk_range(M, chunk, nchunk);
  for (;;) {
    const int64_t m = ch.begin + warp_fetch(work_counter(cn, PH_REFIT_P1, chunk), FULL_MASK);
    const int64_t base = __shfl_sync(FULL_MASK, m, 0);
    if (base >= ch.end) break;
    const bool valid = m < ch.end;
    const int t = valid ? in.track_tl[m] : in.track_tl[base];
    RefitLane w;
    w.n = in.f_n[t];
    w.nf = in.f_nf[t];
    w.h = in.hits + (int64_t)t * NROW;
    w.hr = in.hrow + (int64_t)t * NROW;
    w.yz = g.yz;
#pragma unroll
    for (int k = 0; k < OWN_WORDS; k++) w.m[k] = in.own_mask[t * OWN_WORDS + k];
    const int rng = in.own_rng[t];
    const int r_out = rng >> 16;
    w.r_in = rng & 0xFFFF;
    uint32_t flags = 0;
    TrkState p;
    seed_state(p, in.f_row[t], sX[in.f_row[t]], in.f_par[t * 5 + 0], in.f_zref[t], in.f_par[t * 5 + 2],
               in.f_par[t * 5 + 3], in.f_par[t * 5 + 4]);
    p.z = in.f_par[t * 5 + 1];
    bool ok = valid;
    const int step = r_out >= p.row ? 1 : -1;
    for (int r = p.row + step; ok && (step > 0 ? r <= r_out : r >= r_out); r += step)
      ok = prop_state(p, r, sX[r], kc, flags, nullptr);
    Chi2Acc chi2;
    chi2.reset();
    int nupd = 0, zend = ZONE;
    bool go = false, dg = false;
    const bool run = ok;
    __syncwarp();  // start the FP64 zone with the whole warp
    if (run) {
      w.j = 0;
      w.take();  // the outermost owned hit, on row r_out
      cov_seed<double>(D, kc);
      cov_seed<float>(C, kc);
      const bool zone0 = ZONE > 0;
      chi2.add(zone_update(p, zone0, D, C, w.cur_yz.x, w.cur_yz.y, kc, nupd, zend, 2 * ZONE, true));  // diagonal seed
      dg = zone0;
      if (zone0) tl.upd64++;
      else tl.upd32++;
      w.take();
      go = true;
    }
    // round 0: the in-step rows; round 1: the rest of a zone that found no
    // tail slot (one copy of the row step in the code)
    int64_t slot = -1;
#pragma unroll 1
    for (int round = 0; round < 2; round++) {
      if (go && slot < 0)
        go = refit_zone(g, kc, sX, w, p, D, C, chi2, nupd, ok, flags, tl, zend, dg, round ? 0 : kc.zone_steps[2]);
      if (round) break;
      slot = tail_claim(kc, cn, 2, chunk, nchunk, go && nupd < zend);
    }
    if (slot >= 0) {
      tail_park(zt, slot, m, D);
    } else if (run && nupd < zend) {
#pragma unroll
      for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
    }
    order_count(next, m, valid && slot < 0, go && ok ? p.row - w.r_in : 0);  // rows left inward
    if (!valid) continue;
    RefitWork& s = RW[m];
    s.w = w;
    s.p = p;
#pragma unroll
    for (int i = 0; i < 15; i++) s.C[i] = C[i];
    s.chi2 = chi2;
    s.nupd = nupd;
    s.ok = ok;
    s.go = go && ok;
    s.flags = (int32_t)flags;
    s.r_out = r_out;
    s.nown = in.nown[t];
    s.unit = __ldg(g.rs_of + w.h[0]) / NROW;
    s.t = t;
    s.zend = zend;
  }
  tl.flush(cn, PH_REFIT_P1);
}

// Zone tail of refit phase 1: the zones phase 1 parked, lanes refilling as
// in the follow stage's zone tail kernels.
__global__ void __launch_bounds__(128, 4) k_refit_p1t(GridView g, KConst kc, RefitWork* RW, ZoneTail zt,
                                                   WorkOrder next, int chunk, int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int64_t n = min((int64_t)cn->zone_pend[2 * MAX_CHUNKS + chunk], tail_size(kc, chunk, nchunk));
  const int64_t base = tail_base(kc, 2, chunk, nchunk);
  LocalTally tl;
  double D[15];
  float C[15];
  RefitLane w;
  TrkState p;
  Chi2Acc chi2;
  int nupd = 0, zend = 0;
  bool ok = false, dg = false;
  uint32_t flags = 0;
  int64_t m = -1;
  bool zgo = false, pass = false, live = true;
  for (;;) {
    const unsigned need = refill_mask(live && !zgo, zgo, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (m >= 0) {
        if (nupd < zend) {
#pragma unroll
          for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
        }
        RefitWork& s = RW[m];
        s.w = w;
        s.p = p;
#pragma unroll
        for (int i = 0; i < 15; i++) s.C[i] = C[i];
        s.chi2 = chi2;
        s.nupd = nupd;
        s.ok = ok;
        s.go = pass && ok;
        s.flags = (int32_t)flags;
        s.zend = zend;
      }
      order_count(next, m, m >= 0, pass && ok ? p.row - w.r_in : 0, need);  // rows left inward
      const int64_t k = warp_fetch(work_counter(cn, PH_REFIT_P1T, chunk), need);
      m = -1;
      live = k < n;
      if (live) {
        m = zt.list[base + k];
        const RefitWork& s = RW[m];
        w = s.w;
        p = s.p;
        chi2 = s.chi2;
        nupd = s.nupd;
        zend = s.zend;
        flags = (uint32_t)s.flags;
        ok = true;
        dg = false;
#pragma unroll
        for (int i = 0; i < 15; i++) D[i] = zt.cov[(base + k) * 15 + i];
        pass = true;
        zgo = nupd < zend;
      }
    }
    if (!__any_sync(FULL_MASK, zgo)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    if (zgo) {
      pass = refit_step<true>(g, kc, sX, w, p, D, C, chi2, nupd, ok, flags, tl, zend, dg);
      zgo = pass && nupd < zend;
    }
  }
  tl.flush(cn, PH_REFIT_P1T);
}

__device__ __forceinline__ void write_track(const RefitIn& in, const float* sX, int64_t m, const RefitWork& s,
                                            const TrkState& p, const float* C, const Chi2Acc& chi2, bool ok,
                                            uint32_t flags, tpc_track* __restrict__ out) {
  const int t = s.t;
  tpc_track tr;
  if (ok) {
    tr.x = sX[s.w.r_in];
    tr.par[0] = p.y + p.yl;
    tr.par[1] = p.zref + (p.z + p.zl);
    tr.par[2] = p.s + p.sl;
    tr.par[3] = p.t;
    tr.par[4] = p.q;
#pragma unroll
    for (int j = 0; j < 15; j++) tr.cov[j] = C[j];
    tr.chi2 = chi2.value();
    tr.first_row = s.w.r_in;
  } else {
    const int fr = in.f_row[t];
    tr.x = sX[fr];
    tr.par[0] = in.f_par[t * 5 + 0];
    tr.par[1] = in.f_zref[t] + in.f_par[t * 5 + 1];
    tr.par[2] = in.f_par[t * 5 + 2];
    tr.par[3] = in.f_par[t * 5 + 3];
    tr.par[4] = in.f_par[t * 5 + 4];
    for (int j = 0; j < 15; j++) tr.cov[j] = in.f_cov[t * 15 + j];
    tr.chi2 = in.f_chi2[t];
    tr.first_row = fr;
    flags = TF_REFIT_FAIL;
  }
  tr.reserved = 0;
  tr.ndf = 2 * s.nown - 5;
  tr.n_clusters = s.nown;
  tr.sector = s.unit % NSEC;
  tr.request = s.unit / NSEC;
  tr.last_row = s.r_out;
  tr.cluster_offset = in.toff[m];
  tr.flags = (int32_t)flags;
  out[m] = tr;
}

// Phase 2 of the refit: the remaining updates in FP32; lanes refill.
__global__ void __launch_bounds__(128) k_refit_p2(GridView g, RefitIn in, KConst kc, RefitWork* RW,
                                                  const int32_t* __restrict__ order, tpc_track* __restrict__ out,
                                                  int chunk, int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const Chunk ch = chunk_range(M, chunk, nchunk);
  LocalTally tl;
  double D[15];  // unused in this phase
  float C[15];
  RefitLane w;
  TrkState p;
  Chi2Acc chi2;
  int nupd = 0;
  bool ok = true, go = false, live = true;
  uint32_t flags = 0;
  int64_t m = -1;
  auto load = [&](int64_t mm) {
    const RefitWork& s = RW[mm];
    w = s.w;
    p = s.p;
#pragma unroll
    for (int i = 0; i < 15; i++) C[i] = s.C[i];
    chi2 = s.chi2;
    nupd = s.nupd;
    ok = s.ok != 0;
    go = s.go != 0;
    flags = (uint32_t)s.flags;
    if (go) w.load_after();  // phase 1 loaded the next hit in one stage
  };
  // lanes refill together once kc.refill of them are idle (as the follow
  // phases 2 and 4)
  for (;;) {
    const unsigned need = refill_mask(live && !go, go, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (m >= 0) write_track(in, sX, m, RW[m], p, C, chi2, ok, flags, out);
      const int64_t idx = ch.begin + warp_fetch(work_counter(cn, PH_REFIT_P2, chunk), need);
      m = idx < ch.end ? (order ? order[idx] : idx) : M;
      if (m < M) load(m);
      else live = false;
    }
    if (!__any_sync(FULL_MASK, go)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    int zend = 0;  // the zone is over
    bool dg = false;  // no FP64 zone in this phase
    if (go) go = refit_step<false>(g, kc, sX, w, p, D, C, chi2, nupd, ok, flags, tl, zend, dg);
  }
  tl.flush(cn, PH_REFIT_P2);
}

}  // namespace tpc
