// a6 track following (Fig. 1c): one thread per tracklet, whole state in
// registers.  Seed from the chain chord, forward pass over the chain and
// outward with gated pick-up, fresh backward pass refitting the forward
// clusters and extending inward.
//
// The first `fp64_updates` Kalman updates after each (re)seed keep the
// covariance in FP64 (in the backward pass a few more while it is still
// converging, zone_update); only the zone kernels (phases 1 and 3) instantiate that
// path, so the binary32 kernels keep their registers.  The lanes of a
// warp are consecutive tracklets, which start on neighbouring rows, so their
// FP64 zones overlap.
#pragma once
#include "kalman.cuh"
#include "order.cuh"

namespace tpc {

struct FollowOut {
  int32_t* n;      // [T] clusters
  int32_t* nf;     // forward clusters
  int32_t* nb;     // backward-extension clusters
  int32_t* flags;
  int32_t* row;    // row of the output state
  int32_t* hits;   // [T*NROW] sorted indices: forward (rows ascending) then backward (rows descending)
  uint8_t* hrow;   // [T*NROW] their rows
  float* par;      // [T*5] z relative to zref
  float* zref;     // [T]
  float* cov;      // [T*15]
  double* chi2;    // [T]
};

struct GridView {
  const float2* yz;
  const int32_t* rs_of;
  const RsParams* par;
  const int32_t* bin_start;
};

__device__ __forceinline__ bool outside_sector(const TrkState& p, const KConst& kc, uint32_t& flags) {
  const float lim = p.x * 0.17632698070846498f + kc.edge;
  const float y = p.y + p.yl;
  if (fabsf(fabsf(y) - lim) <= 1e-3f) flags |= TF_EDGE;
  return fabsf(y) > lim;
}

// Index range of the bins of one row-sector axis covering [v - w, v + w];
// the window is widened by a margin far above the binary32 rounding of its
// edges, and the caller applies the exact test to every candidate.
__device__ __forceinline__ void axis_range(float v, float w, float lo, float inv, int nb, int& i0, int& i1) {
  const float m = w + 1e-3f + 2e-6f * fabsf(v);
  const float f0 = floorf((v - m - lo) * inv), f1 = floorf((v + m - lo) * inv);
  const float top = (float)(nb - 1);
  i0 = !(f0 >= 0.0f) ? 0 : (f0 > top ? nb - 1 : (int)f0);
  i1 = !(f1 >= 0.0f) ? 0 : (f1 > top ? nb - 1 : (int)f1);
}

constexpr int PICK_BATCH = 4;  // candidate loads a pick issues together
// Best cluster of row-sector rs for the predicted state: minimum chi2 =
// dy^2/Syy + dz^2/Szz within the gate, ties to the lower sorted index.
// Near-ties and near-gate candidates raise the taint flags.
template <bool BATCH>
__device__ __forceinline__ int pick(const GridView& g, int rs, int row, const TrkState& p, float cyy, float czz,
                                    const KConst& kc, const float* sYH, uint32_t& flags, unsigned& ncand) {
  const RsParams P = load_params(g.par + rs);
  if (P.count == 0) return -1;
  const float Syy = cyy + kc.V, Szz = czz + kc.V;
  const float wy = ksqrt(kc.gate * Syy), wz = ksqrt(kc.gate * Szz);
  const float iSyy = kinv(Syy), iSzz = kinv(Szz);
  int iy0, iy1, iz0, iz1;
  axis_range(p.y + p.yl, wy, -sYH[row], P.inv_y, P.n_y, iy0, iy1);
  axis_range(p.zref + (p.z + p.zl), wz, P.z_lo, P.inv_z, P.n_z, iz0, iz1);
  const float gate = kc.gate, eps = kc.taint;
  float b1v = __int_as_float(0x7F800000), b2v = b1v;
  int best = -1;
  auto consider = [&](float2 q, int c) {
    const float dy = (q.x - p.y) - p.yl;
    const float dz = ((q.y - p.zref) - p.z) - p.zl;
    const float chi = dy * dy * iSyy + dz * dz * iSzz;
    if (fabsf(chi - gate) <= eps * (1.0f + gate)) flags |= TF_GATE;
    if (!(chi <= gate)) return;
    if (chi < b1v || (chi == b1v && c < best)) {
      b2v = b1v;
      b1v = chi;
      best = c;
    } else if (chi < b2v) {
      b2v = chi;
    }
  };
  // The pick does not depend on the order in which candidates are taken, so
  // (BATCH) a window of up to three z-rows of bins loads the three bin
  // ranges in one round and then its candidates PICK_BATCH at a time across
  // the z-rows (one round per batch instead of one per z-row and candidate
  // pair: a binary32 row step waited on up to six dependent rounds to L2).
  // The FP64-zone kernels, bound by their FP64 pipe, keep the z-row loop and
  // its registers.
  if (BATCH && iz1 - iz0 < 3) {
    int a0, n0, a1 = 0, n1 = 0, a2 = 0, n2 = 0;
    {
      const int base = P.bin_base + iz0 * P.n_y;
      a0 = __ldg(g.bin_start + base + iy0);
      n0 = __ldg(g.bin_start + base + iy1 + 1);
      if (iz1 > iz0) {
        a1 = __ldg(g.bin_start + base + P.n_y + iy0);
        n1 = __ldg(g.bin_start + base + P.n_y + iy1 + 1);
      }
      if (iz1 > iz0 + 1) {
        a2 = __ldg(g.bin_start + base + 2 * P.n_y + iy0);
        n2 = __ldg(g.bin_start + base + 2 * P.n_y + iy1 + 1);
      }
      n0 -= a0;
      n1 -= a1;
      n2 -= a2;
    }
    const int tot = n0 + n1 + n2;
    ncand += (unsigned)tot;
    for (int j0 = 0; j0 < tot; j0 += PICK_BATCH) {
      int c[PICK_BATCH];
      float2 q[PICK_BATCH];
#pragma unroll
      for (int k = 0; k < PICK_BATCH; k++) {
        const int j = j0 + k;
        c[k] = j < n0 ? a0 + j : (j < n0 + n1 ? a1 + (j - n0) : a2 + (j - n0 - n1));
        if (j < tot) q[k] = __ldg(g.yz + c[k]);
      }
#pragma unroll
      for (int k = 0; k < PICK_BATCH; k++)
        if (j0 + k < tot) consider(q[k], c[k]);
    }
  } else {
    for (int iz = iz0; iz <= iz1; iz++) {
      const int base = P.bin_base + iz * P.n_y;
      const int a = __ldg(g.bin_start + base + iy0), b = __ldg(g.bin_start + base + iy1 + 1);
      ncand += (unsigned)(b - a);
      int c = a;  // two candidates' loads in flight at a time
      for (; c + 1 < b; c += 2) {
        const float2 q0 = __ldg(g.yz + c), q1 = __ldg(g.yz + c + 1);
        consider(q0, c);
        consider(q1, c + 1);
      }
      if (c < b) consider(__ldg(g.yz + c), c);
    }
  }
  if (best >= 0 && b2v != __int_as_float(0x7F800000) && b2v - b1v <= eps * (1.0f + b1v)) flags |= TF_TIE;
  return best;
}

// Per-lane bookkeeping of one tracklet.
struct Lane {
  int32_t* hits;
  uint8_t* hrow;
  int ubase, r0, L;
  int nf, nb;
  int k;        // current chain cluster (forward)
  int nk;       // next chain cluster, loaded a step ahead (-1: none)
  int i;        // next chain index (forward)
  int r_last;   // row of the last forward update
  int kf;       // next forward hit to refit (backward)
  int misses;
  int nupd;     // updates since the last (re)seed
  int zend;     // update count that ends the FP64 zone (zone_update)
  int nx_row;   // backward: row of forward hit kf (-1: none), its index and position, loaded a step ahead
  int nx_c;
  float2 nx_yz;
  uint32_t flags;
  bool seed_fail;
  bool tr;       // this tracklet is traced
  bool snap;     // backward zone: the output covariance is pending in the FP64 snapshot (zone_snap_take)
  bool dg;       // zone: the FP64 covariance is the diagonal one the seed's first update left (until a propagation)
  Counts* cn;
  TrkState fwd;  // forward state after its last update
};

// Loads forward hit kf for the backward refit, one step before its use.
__device__ __forceinline__ void next_fwd_hit(Lane& w, const GridView& g) {
  if (w.kf >= 0) {
    w.nx_row = w.hrow[w.kf];
    w.nx_c = w.hits[w.kf];
    w.nx_yz = __ldg(g.yz + w.nx_c);
  } else {
    w.nx_row = -1;
  }
}

// Trace line of one Kalman update (out of line: executed for one tracklet).
__device__ __noinline__ void trace_line(Counts* cn, float* trace, int cap, float pass, float row, float nupd,
                                        float y, float z, float s, float t, float q, float cyy, float czz,
                                        float css, float ctt, float cqq, float chi2, float r0, float r1) {
  const int k = atomicAdd(&cn->trace_n, 1);
  if (k >= cap) return;
  float* o = trace + (size_t)k * TRACE_W;
  const float v[TRACE_W] = {pass, row, nupd, y, z, s, t, q, cyy, czz, css, ctt, cqq, chi2, r0, r1};
#pragma unroll
  for (int i = 0; i < TRACE_W; i++) o[i] = v[i];
}

// Kalman update of the lane's state (covariance in D during the zone, else
// in C); records a trace line when the lane is traced.
template <bool Z>
__device__ __forceinline__ void lane_update(Lane& w, const KConst& kc, TrkState& p, bool zone, double* D, float* C,
                                            float2 P, Chi2Acc& chi2, int pass, bool diag = false) {
  zone = Z && zone;
  const float r0 = residual_y(p, P.x), r1 = residual_z(p, P.y);
  chi2.add(zone_update(p, zone, D, C, P.x, P.y, kc, w.nupd, w.zend, pass ? 2 * kc.fp64_updates : kc.fp64_updates,
                       diag));
  if (w.tr)
    trace_line(w.cn, kc.trace, kc.trace_cap, (float)pass, (float)p.row, (float)w.nupd, p.y + p.yl,
               p.zref + (p.z + p.zl), p.s + p.sl, p.t, p.q, zone ? (float)D[0] : C[0], zone ? (float)D[2] : C[2],
               zone ? (float)D[5] : C[5], zone ? (float)D[9] : C[9], zone ? (float)D[14] : C[14],
               (float)chi2.value(), r0, r1);
}

// Output snapshot of the backward pass: the state after its last update,
// kept in the lane's shared-memory output slot (out_put) by every backward
// kernel and parked with the tracklet between them (FollowWork::out), so
// that it takes no registers.  Inside the FP64 zone the covariance is kept
// as FP64 in shared memory (element i of a lane at snap[i * SNAP_STRIDE]) and
// rounded to binary32 into the slot once, by zone_snap_take, instead of at
// every update: the FP64 pipe, which bounds the zone, then does no
// conversions for updates that a later one replaces.
constexpr int SNAP_STRIDE = 128;  // the largest block of the follow kernels
constexpr int OUT_WORDS = 25;     // words of a lane's output snapshot (out_put)
// Shared-memory output slot of a phase-4 lane (word i at so[i * SNAP_STRIDE],
// OUT_WORDS words): row, y, z, sin phi, dz/ds_T, q/pT (the compensated
// sums), zref, the 15 covariance entries, the chi2 total (two words) and its
// binary32 part.
__device__ __forceinline__ void out_put_state(float* so, const TrkState& p, const Chi2Acc& chi2) {
  so[0] = __int_as_float(p.row);
  so[1 * SNAP_STRIDE] = p.y + p.yl;
  so[2 * SNAP_STRIDE] = p.z + p.zl;
  so[3 * SNAP_STRIDE] = p.s + p.sl;
  so[4 * SNAP_STRIDE] = p.t;
  so[5 * SNAP_STRIDE] = p.q;
  so[6 * SNAP_STRIDE] = p.zref;
  so[22 * SNAP_STRIDE] = __int_as_float(__double2hiint(chi2.total));
  so[23 * SNAP_STRIDE] = __int_as_float(__double2loint(chi2.total));
  so[24 * SNAP_STRIDE] = chi2.part;
}
__device__ __forceinline__ void out_put(float* so, const TrkState& p, const float* C, const Chi2Acc& chi2) {
  out_put_state(so, p, chi2);
#pragma unroll
  for (int i = 0; i < 15; i++) so[(7 + i) * SNAP_STRIDE] = C[i];
}
// A state in a lane's shared-memory slot (word i at s[i * SNAP_STRIDE]):
// phase 2 keeps the forward state after its last update there.
constexpr int TRK_WORDS = 11;
__device__ __forceinline__ void trk_put(float* s, const TrkState& p) {
  s[0] = p.x;
  s[1 * SNAP_STRIDE] = __int_as_float(p.row);
  s[2 * SNAP_STRIDE] = p.y;
  s[3 * SNAP_STRIDE] = p.z;
  s[4 * SNAP_STRIDE] = p.s;
  s[5 * SNAP_STRIDE] = p.t;
  s[6 * SNAP_STRIDE] = p.q;
  s[7 * SNAP_STRIDE] = p.yl;
  s[8 * SNAP_STRIDE] = p.zl;
  s[9 * SNAP_STRIDE] = p.sl;
  s[10 * SNAP_STRIDE] = p.zref;
}
__device__ __forceinline__ TrkState trk_get(const float* s) {
  TrkState p;
  p.x = s[0];
  p.row = __float_as_int(s[1 * SNAP_STRIDE]);
  p.y = s[2 * SNAP_STRIDE];
  p.z = s[3 * SNAP_STRIDE];
  p.s = s[4 * SNAP_STRIDE];
  p.t = s[5 * SNAP_STRIDE];
  p.q = s[6 * SNAP_STRIDE];
  p.yl = s[7 * SNAP_STRIDE];
  p.zl = s[8 * SNAP_STRIDE];
  p.sl = s[9 * SNAP_STRIDE];
  p.zref = s[10 * SNAP_STRIDE];
  return p;
}
template <bool Z>
__device__ __forceinline__ void keep_output(Lane& w, const TrkState& p, bool zone, const double* D, const float* C,
                                            const Chi2Acc& chi2, double* snap, float* so) {
  if (Z && zone) {
    out_put_state(so, p, chi2);
#pragma unroll
    for (int i = 0; i < 15; i++) snap[i * SNAP_STRIDE] = D[i];
    w.snap = true;
    return;
  }
  out_put(so, p, C, chi2);
  if (Z) w.snap = false;
}
__device__ __forceinline__ void zone_snap_take(Lane& w, const double* snap, float* so) {
  if (w.snap) {
#pragma unroll
    for (int i = 0; i < 15; i++) so[(7 + i) * SNAP_STRIDE] = narrow(snap[i * SNAP_STRIDE]);
    w.snap = false;
  }
}

// One forward row step; false ends the pass.  The covariance is in D while
// fewer than fp64_updates updates have been made since the seed.  PB: the
// pick loads its candidates in batches (pick); phase 2's build for inputs
// that fill the GPU keeps the z-row loop (in its register budget the
// batches spilled: 8.22 -> 8.81 ms on the 10 ms timeframe).
template <bool Z, bool PB = false>
__device__ __forceinline__ bool fwd_step(const GridView& g, const int32_t* __restrict__ up_m, const KConst& kc,
                                         const float* sX, const float* sYH, Lane& w, TrkState& p, double* D,
                                         float* C, Chi2Acc& chi2, LocalTally& tl, float* sf) {
  const int r = p.row + 1;
  if (r >= NROW) return false;
  if (r + 1 < NROW) prefetch_l1(g.par + w.ubase + r + 1);  // the next step's row-sector parameters
  const bool chain = w.i < w.L;
  const bool zone = Z && w.nupd < w.zend;
  float2 Pc;
  int c = -1;
  bool cross = false;  // a row the chain's links skipped (link_skip): crossed without an update
  if (chain) {  // the chain's cluster and the one after it are loaded while the state propagates
    c = w.nk;
    if (kc.link_skip) cross = __ldg(g.rs_of + c) % NROW != r;
    if (!cross) {
      Pc = __ldg(g.yz + c);
      w.nk = w.i + 1 < w.L ? __ldg(up_m + c) : -1;
    }
  }
  if (!propagate_any(p, zone, D, C, r, sX[r], kc, w.flags, Z && w.dg)) {
    if (chain) w.seed_fail = true;
    return false;
  }
  if (Z) w.dg = false;
  tl.prop++;
  tl.prop64 += zone;
  if (cross) return true;
  if (chain) {
    w.k = c;
    w.i++;
  } else {
    if (outside_sector(p, kc, w.flags)) return false;
    c = pick<PB>(g, w.ubase + r, r, p, zone ? narrow(D[0]) : C[0], zone ? narrow(D[2]) : C[2], kc, sYH, w.flags,
             tl.cand);
    if (c < 0) return ++w.misses < kc.max_miss;
  }
  const float2 P = chain ? Pc : __ldg(g.yz + c);
  lane_update<Z>(w, kc, p, zone, D, C, P, chi2, 0);
  if (zone) tl.upd64++;
  else tl.upd32++;
  w.hits[w.nf] = c;
  w.hrow[w.nf] = (uint8_t)r;
  w.nf++;
  if (Z) w.fwd = p;  // phase 1 parks it with the lane, phase 2 keeps it in shared memory
  else trk_put(sf, p);
  w.r_last = r;
  w.misses = 0;
  return true;
}

// One backward row step; false ends the pass.  Rows r >= r0 refit the
// forward clusters (an update where a forward cluster sits), rows below
// extend the tracklet inward with the gated pick-up.  M: BW_ANY takes both
// kinds of step; BW_REFIT is only ever called for a refit row (phase 4r) and
// BW_EXTEND only for an extension row (phase 4, after phase 4r), so each of
// those kernels carries one kind's code.
enum { BW_ANY = 0, BW_REFIT, BW_EXTEND };
template <bool Z, int M = BW_ANY>
__device__ __forceinline__ bool bwd_step(const GridView& g, const KConst& kc, const float* sX, const float* sYH,
                                         Lane& w, TrkState& p, double* D, float* C, Chi2Acc& chi2, LocalTally& tl,
                                         double* snap, float* so) {
  const int r = p.row - 1;
  if (r < 0) return false;
  if (r >= 1 && r - 1 < w.r0) prefetch_l1(g.par + w.ubase + r - 1);  // the next step's row-sector parameters
  const bool zone = Z && w.nupd < w.zend;
  if (!propagate_any(p, zone, D, C, r, sX[r], kc, w.flags, Z && w.dg)) {
    if (M == BW_REFIT || (M == BW_ANY && r >= w.r0)) w.flags |= TF_BACK_FAIL;
    return false;
  }
  if (Z) w.dg = false;
  tl.prop++;
  tl.prop64 += zone;
  float2 P;
  if (M == BW_REFIT || (M == BW_ANY && r >= w.r0)) {
    if (w.nx_row != r) return true;
    P = w.nx_yz;
    w.kf--;
    next_fwd_hit(w, g);
  } else {
    if (outside_sector(p, kc, w.flags)) return false;
    const int c = pick<!Z>(g, w.ubase + r, r, p, zone ? narrow(D[0]) : C[0], zone ? narrow(D[2]) : C[2], kc, sYH,
                       w.flags, tl.cand);
    if (c < 0) return ++w.misses < kc.max_miss;
    w.hits[w.nf + w.nb] = c;
    w.hrow[w.nf + w.nb] = (uint8_t)r;
    w.nb++;
    w.misses = 0;
    P = __ldg(g.yz + c);
  }
  lane_update<Z>(w, kc, p, zone, D, C, P, chi2, 1);
  if (zone) tl.upd64++;
  else tl.upd32++;
  keep_output<Z>(w, p, w.nupd < w.zend, D, C, chi2, snap, so);
  return true;
}

// Fresh covariance for a (re)seed: diag(c0) in D (zone) or C.
__device__ __forceinline__ void reseed_cov(const KConst& kc, double* D, float* C) {
  cov_seed<double>(D, kc);
  cov_seed<float>(C, kc);
}

// Tracklet state parked in global memory (L2-resident) between the phase
// kernels of the follow stage.
struct FollowWork {
  Lane w;
  TrkState p;
  float C[15];
  Chi2Acc chi2;
  int32_t go;
  int32_t pad[3];
  float out[OUT_WORDS];    // the backward pass's output snapshot, as out_put lays it out
};

__device__ __forceinline__ void work_store(FollowWork* W, int64_t t, const Lane& w, const TrkState& p,
                                           const float* C, const Chi2Acc& chi2, bool go) {
  FollowWork& s = W[t];
  s.w = w;
  s.p = p;
#pragma unroll
  for (int i = 0; i < 15; i++) s.C[i] = C[i];
  s.chi2 = chi2;
  s.go = go;
}
// Phase 3 reads what its re-seed and backward zone use and writes back only
// what it changes and the later phases read (a whole-lane load and store
// would keep the lane's forward fields in registers through the zone).
__device__ __forceinline__ void zone_bwd_load(const FollowWork* W, int64_t t, Lane& w, TrkState& p) {
  const FollowWork& s = W[t];
  w.ubase = s.w.ubase;
  w.r0 = s.w.r0;
  w.nf = s.w.nf;
  w.nb = s.w.nb;
  w.flags = s.w.flags;
  w.seed_fail = s.w.seed_fail;
  w.tr = s.w.tr;
  p = s.w.fwd;
}
__device__ __forceinline__ void zone_bwd_store(FollowWork* W, int64_t t, const Lane& w, const TrkState& p,
                                               const float* C, const Chi2Acc& chi2, const float* so, bool go) {
  FollowWork& s = W[t];
  s.w.nb = w.nb;
  s.w.kf = w.kf;
  s.w.misses = w.misses;
  s.w.nupd = w.nupd;
  s.w.nx_row = w.nx_row;
  s.w.nx_c = w.nx_c;
  s.w.nx_yz = w.nx_yz;
  s.w.flags = w.flags;
  s.p = p;
#pragma unroll
  for (int i = 0; i < 15; i++) s.C[i] = C[i];
  s.chi2 = chi2;
  s.go = go;
#pragma unroll
  for (int i = 0; i < OUT_WORDS; i++) s.out[i] = so[i * SNAP_STRIDE];
}

// A backward zone parked by phase 3 (zone_bwd_store, plus zend), for its
// zone tail kernel: the fields the zone's row steps use, and the output
// snapshot into the lane's shared-memory slot.
__device__ __forceinline__ void zone_tail_bwd_load(const FollowWork* W, int64_t t, Lane& w, TrkState& p,
                                                   Chi2Acc& chi2, float* so) {
  const FollowWork& s = W[t];
  w.ubase = s.w.ubase;
  w.r0 = s.w.r0;
  w.nf = s.w.nf;
  w.nb = s.w.nb;
  w.kf = s.w.kf;
  w.misses = s.w.misses;
  w.nupd = s.w.nupd;
  w.zend = s.w.zend;
  w.nx_row = s.w.nx_row;
  w.nx_c = s.w.nx_c;
  w.nx_yz = s.w.nx_yz;
  w.flags = s.w.flags;
  w.seed_fail = false;
  w.tr = s.w.tr;
  w.snap = false;
  w.dg = false;
  p = s.p;
  chi2 = s.chi2;
#pragma unroll
  for (int i = 0; i < OUT_WORDS; i++) so[i * SNAP_STRIDE] = s.out[i];
}

// The binary32 phases touch only their half of the parked lane, so that
// neither carries the other's state in registers (the large-input builds
// spilled it) nor moves it to and from memory.  Phase 2 reads the forward
// fields and writes back what phase 3 uses (the forward state after its last
// update, the forward hit count and the flags; phase 3 re-seeds, so the
// running state, covariance and chi2 of phase 2 are not kept).  Phase 4 reads
// the backward fields.
__device__ __forceinline__ bool fwd_load(const FollowWork* W, int64_t t, Lane& w, TrkState& p, float* C,
                                         Chi2Acc& chi2, float* sf) {
  const FollowWork& s = W[t];
  w.ubase = s.w.ubase;
  w.L = s.w.L;
  w.nf = s.w.nf;
  w.k = s.w.k;
  w.nk = s.w.nk;
  w.i = s.w.i;
  w.r_last = s.w.r_last;
  w.misses = s.w.misses;
  w.nupd = s.w.nupd;
  w.flags = s.w.flags;
  w.seed_fail = s.w.seed_fail;
  w.tr = s.w.tr;
  trk_put(sf, s.w.fwd);
  p = s.p;
#pragma unroll
  for (int i = 0; i < 15; i++) C[i] = s.C[i];
  chi2 = s.chi2;
  return s.go != 0;
}
__device__ __forceinline__ void fwd_store(FollowWork* W, int64_t t, const Lane& w, const float* sf) {
  FollowWork& s = W[t];
  s.w.nf = w.nf;
  s.w.flags = w.flags;
  s.w.seed_fail = w.seed_fail;
  s.w.fwd = trk_get(sf);
}
__device__ __forceinline__ bool bwd_load(const FollowWork* W, int64_t t, Lane& w, TrkState& p, float* C,
                                         Chi2Acc& chi2, float* so) {
  const FollowWork& s = W[t];
  w.ubase = s.w.ubase;
  w.r0 = s.w.r0;
  w.nf = s.w.nf;
  w.nb = s.w.nb;
  w.kf = s.w.kf;
  w.misses = s.w.misses;
  w.nupd = s.w.nupd;
  w.nx_row = s.w.nx_row;
  w.nx_c = s.w.nx_c;
  w.nx_yz = s.w.nx_yz;
  w.flags = s.w.flags;
  w.seed_fail = s.w.seed_fail;
  w.tr = s.w.tr;
#pragma unroll
  for (int i = 0; i < OUT_WORDS; i++) so[i * SNAP_STRIDE] = s.out[i];  // (unused after a seed failure)
  p = s.p;
#pragma unroll
  for (int i = 0; i < 15; i++) C[i] = s.C[i];
  chi2 = s.chi2;
  return s.go != 0;
}

// Phase 4r parks what its refit steps changed for phase 4: the running
// state, covariance and chi2, the forward-hit cursor, the flags, whether the
// pass goes on, and the output snapshot.
__device__ __forceinline__ void bwd_store(FollowWork* W, int64_t t, const Lane& w, const TrkState& p,
                                          const float* C, const Chi2Acc& chi2, const float* so, bool go) {
  FollowWork& s = W[t];
  s.w.kf = w.kf;
  s.w.nupd = w.nupd;
  s.w.nx_row = w.nx_row;
  s.w.nx_c = w.nx_c;
  s.w.nx_yz = w.nx_yz;
  s.w.flags = w.flags;
  s.p = p;
#pragma unroll
  for (int i = 0; i < 15; i++) s.C[i] = C[i];
  s.chi2 = chi2;
  s.go = go;
#pragma unroll
  for (int i = 0; i < OUT_WORDS; i++) s.out[i] = so[i * SNAP_STRIDE];
}

// Work distribution of the persistent Kalman kernels: the lanes in `need`,
// all of which make this call, take consecutive indices of *counter with one
// atomic for the warp.
__device__ __forceinline__ int64_t warp_fetch(int32_t* counter, unsigned need) {
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(need) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(need));
  base = __shfl_sync(need, base, leader);
  return (int64_t)base + __popc(need & ((1u << lane) - 1u));
}

// Refill decision of a refilling kernel: the mask of lanes to refill now --
// the idle lanes that can still get work, once at least kc.refill of them
// are idle or no lane has work left.
__device__ __forceinline__ unsigned refill_mask(bool idle, bool busy, int refill) {
  const unsigned m = __ballot_sync(FULL_MASK, idle);
  const unsigned b = __ballot_sync(FULL_MASK, busy);
  return (m && (__popc(m) >= refill || b == 0)) ? m : 0u;
}

__device__ __forceinline__ void load_tables(float* sX, float* sYH) {
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) {
    sX[i] = g_row_x[i];
    sYH[i] = g_row_yhi[i];
  }
  __syncthreads();
}

// Zone tails.  A zone kernel's warp runs its 32 tracklets' zones in step,
// so each warp ran to its longest zone while most lanes had ended theirs at
// about ten steps (the pick-up's misses and rows without a forward cluster
// lengthen a few): 22-26% of the lane slots of the FP64 instructions were
// idle, and the FP64 pipe spends the same time on an instruction whatever
// its active lanes.  So a zone kernel takes kc.zone_steps steps in step and
// parks a tracklet whose zone is still open (its FP64 covariance in a list
// slot of its own); a tail kernel then finishes those zones with lanes that
// refill from the list.  Chunk c of nc owns slots [c cap / nc, (c+1) cap / nc)
// of a pass's list; a tracklet that finds its chunk's slots taken finishes
// its zone in place.
struct ZoneTail {
  int32_t* list;  // [3 * cap] item of each slot (pass 0: follow forward, 1: follow backward, 2: refit)
  double* cov;    // [3 * cap * 15] its FP64 covariance
};
__device__ __forceinline__ int64_t tail_base(const KConst& kc, int pass, int chunk, int nchunk) {
  return pass * kc.zone_tail_cap + kc.zone_tail_cap * chunk / nchunk;
}
__device__ __forceinline__ int64_t tail_size(const KConst& kc, int chunk, int nchunk) {
  return kc.zone_tail_cap * (chunk + 1) / nchunk - kc.zone_tail_cap * chunk / nchunk;
}
// A list slot for each lane with pend (all 32 lanes make the call; one
// atomic per warp); -1 for the others and when the chunk's slots are taken.
__device__ __forceinline__ int64_t tail_claim(const KConst& kc, Counts* cn, int pass, int chunk, int nchunk,
                                              bool pend) {
  const unsigned m = __ballot_sync(FULL_MASK, pend);
  if (!m) return -1;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&cn->zone_pend[pass * MAX_CHUNKS + chunk], __popc(m));
  base = __shfl_sync(FULL_MASK, base, leader);
  const int64_t k = (int64_t)base + __popc(m & ((1u << lane) - 1u));
  return pend && k < tail_size(kc, chunk, nchunk) ? tail_base(kc, pass, chunk, nchunk) + k : -1;
}
__device__ __forceinline__ void tail_park(const ZoneTail& zt, int64_t slot, int64_t t, const double* D) {
  zt.list[slot] = (int32_t)t;
#pragma unroll
  for (int i = 0; i < 15; i++) zt.cov[slot * 15 + i] = D[i];
}
// Zone steps of one lane: up to cap steps (0: until the zone or the pass
// ends).  True while the pass goes on.
__device__ __forceinline__ bool fwd_zone(const GridView& g, const int32_t* __restrict__ up_m, const KConst& kc,
                                         const float* sX, const float* sYH, Lane& w, TrkState& p, double* D,
                                         float* C, Chi2Acc& chi2, LocalTally& tl, int cap) {
  bool go = true;
  for (int k = 0; go && w.nupd < w.zend && (cap == 0 || k < cap); k++)
    go = fwd_step<true>(g, up_m, kc, sX, sYH, w, p, D, C, chi2, tl, nullptr);
  return go;
}

// Phase 1: seed and the forward pass while its covariance is in FP64 (the
// first kc.zone_steps[0] row steps of the zone; the rest in the tail kernel
// k_follow_p1t).  A warp takes 32 consecutive tracklets at a time and starts
// their zones together; the grid is the resident capacity (one wave).
__global__ void __launch_bounds__(128, 4) k_follow_p1(GridView g, const int32_t* __restrict__ tl_start,
                                                   const int32_t* __restrict__ tl_len,
                                                   const int32_t* __restrict__ tl_end,
                                                   const int32_t* __restrict__ up_m, KConst kc, FollowOut o,
                                                   FollowWork* W, ZoneTail zt, WorkOrder next, int chunk,
                                                   int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  const Chunk ch = chunk_range(cn->n_tracklets, chunk, nchunk);
  LocalTally tl;
  double D[15];
  float C[15];
  for (;;) {
    const int64_t t = ch.begin + warp_fetch(work_counter(cn, PH_FOLLOW_P1, chunk), FULL_MASK);
    if (__shfl_sync(FULL_MASK, t, 0) >= ch.end) break;
    const bool valid = t < ch.end;
    Lane w;
    TrkState p;
    Chi2Acc chi2;
    bool go = false;
    if (valid) {
      w.hits = o.hits + t * NROW;
      w.hrow = o.hrow + t * NROW;
      w.flags = 0;
      w.seed_fail = false;
      w.tr = (t == kc.trace_t);
      w.cn = cn;
      const int c0 = tl_start[t], cl = tl_end[t];
      w.L = tl_len[t];
      const int rs0 = __ldg(g.rs_of + c0);
      w.ubase = rs0 - rs0 % NROW;
      w.r0 = rs0 % NROW;
      const float2 P0 = __ldg(g.yz + c0), P1 = __ldg(g.yz + cl);
      {
        // the chain's last row: r0 + L - 1 unless its links skip rows
        const int r_end = kc.link_skip ? __ldg(g.rs_of + cl) % NROW : w.r0 + w.L - 1;
        const float x0 = sX[w.r0], x1 = sX[r_end];
        const float dX = x1 - x0, dY = P1.x - P0.x, dZ = P1.y - P0.y;
        const float Lc = sqrtf(dX * dX + dY * dY);
        seed_state(p, w.r0, x0, P0.x, P0.y, dY / Lc, dZ / Lc, 0.0f);
      }
      w.k = c0;
      w.nk = w.L > 1 ? __ldg(up_m + c0) : -1;
      w.i = 1;
      w.misses = 0;
      w.r_last = w.r0;
      w.hits[0] = c0;
      w.hrow[0] = (uint8_t)w.r0;
      w.nf = 1;
      w.nb = 0;
      w.kf = 0;
      chi2.reset();
      reseed_cov(kc, D, C);
      w.nupd = 0;
      w.zend = kc.fp64_updates;
    }
    __syncwarp();  // the zones of the warp's lanes start together
    if (valid) {
      const bool zone0 = kc.fp64_updates > 0;
      lane_update<true>(w, kc, p, zone0, D, C, __ldg(g.yz + tl_start[t]), chi2, 0, true);  // diagonal seed covariance
      w.dg = zone0;
      if (zone0) tl.upd64++;
      else tl.upd32++;
      w.fwd = p;
      go = true;
    }
    // round 0: the in-step rows; round 1: the rest of a zone that found no
    // tail slot (one copy of the row step in the code)
    int64_t slot = -1;
#pragma unroll 1
    for (int round = 0; round < 2; round++) {
      if (go && slot < 0) go = fwd_zone(g, up_m, kc, sX, sYH, w, p, D, C, chi2, tl, round ? 0 : kc.zone_steps[0]);
      if (round) break;
      slot = tail_claim(kc, cn, 0, chunk, nchunk, go && w.nupd < w.zend);
    }
    if (valid) {
      if (slot >= 0) {
        tail_park(zt, slot, t, D);
      } else if (w.nupd < w.zend) {
#pragma unroll
        for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
      }
      work_store(W, t, w, p, C, chi2, go);
    }
    order_count(next, t, valid && slot < 0, go ? NROW - 1 - p.row : 0);  // rows left outward
  }
  tl.flush(cn, PH_FOLLOW_P1);
}

// Zone tail of phase 1: the forward zones phase 1 parked, each to the end
// of its zone (or of its pass).  Their remaining rows differ widely (1 to
// 10 and more), so the lanes refill as phase 2's do; a refill loads a parked
// state and makes no FP64 operation.
__global__ void __launch_bounds__(128, 4) k_follow_p1t(GridView g, const int32_t* __restrict__ up_m, KConst kc,
                                                    FollowWork* W, ZoneTail zt, WorkOrder next, int chunk,
                                                    int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  const int64_t n = min((int64_t)cn->zone_pend[0 * MAX_CHUNKS + chunk], tail_size(kc, chunk, nchunk));
  const int64_t base = tail_base(kc, 0, chunk, nchunk);
  LocalTally tl;
  double D[15];
  float C[15];
  Lane w;
  TrkState p;
  Chi2Acc chi2;
  int64_t t = -1;     // tracklet held by the lane (-1: none)
  bool zgo = false;   // its zone has rows left
  bool pass = false;  // its pass goes on
  bool live = true;   // the lane may still get work
  for (;;) {
    const unsigned need = refill_mask(live && !zgo, zgo, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (t >= 0) {
        if (w.nupd < w.zend) {  // the pass ended inside the zone
#pragma unroll
          for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
        }
        work_store(W, t, w, p, C, chi2, pass);
      }
      order_count(next, t, t >= 0, pass ? NROW - 1 - p.row : 0, need);  // rows left outward
      const int64_t k = warp_fetch(work_counter(cn, PH_FOLLOW_P1T, chunk), need);
      t = -1;
      live = k < n;
      if (live) {
        t = zt.list[base + k];
        const FollowWork& s = W[t];
        w = s.w;
        p = s.p;
        chi2 = s.chi2;
#pragma unroll
        for (int i = 0; i < 15; i++) D[i] = zt.cov[(base + k) * 15 + i];
        pass = true;
        zgo = w.nupd < w.zend;
      }
    }
    if (!__any_sync(FULL_MASK, zgo)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    if (zgo) {
      pass = fwd_step<true>(g, up_m, kc, sX, sYH, w, p, D, C, chi2, tl, nullptr);
      zgo = pass && w.nupd < w.zend;
    }
  }
  tl.flush(cn, PH_FOLLOW_P1T);
}

// Phase 2: the rest of the forward pass (covariance in FP32).  MINB: CTAs
// per SM the registers are budgeted for -- 4 (no spills) where the longest
// tracklet bounds the kernel, 7 here and in phase 4 (72 registers, more
// resident warps) on inputs that fill the GPU.  A lane
// that finishes a tracklet idles until kc.refill lanes of its warp have,
// then they store their results and take new tracklets together, so that
// the refill runs with many lanes at once and no lane waits for the longest
// tracklet of its warp.
template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_follow_p2(GridView g, const int32_t* __restrict__ up_m, KConst kc,
                                                   FollowOut o, FollowWork* W, const int32_t* __restrict__ order,
                                                   int chunk, int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  __shared__ float sFwd[TRK_WORDS * SNAP_STRIDE];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  float* sf = sFwd + threadIdx.x;
  const int32_t T = cn->n_tracklets;
  const Chunk ch = chunk_range(T, chunk, nchunk);
  LocalTally tl;
  double D[15];  // unused in this phase (the zone is over)
  float C[15];
  Lane w;
  TrkState p;
  Chi2Acc chi2;
  chi2.reset();
  int64_t t = -1;      // tracklet held by the lane (-1: none yet)
  bool go = false;     // the lane's tracklet has steps left
  bool live = true;    // the lane may still get work
  bool dirty = false;  // the held tracklet advanced since it was loaded
  for (;;) {
    const unsigned need = refill_mask(live && !go, go, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (dirty) fwd_store(W, t, w, sf);
      const int64_t idx = ch.begin + warp_fetch(work_counter(cn, PH_FOLLOW_P2, chunk), need);
      t = idx < ch.end ? (order ? order[idx] : idx) : T;
      dirty = false;
      if (t < T) {
        go = fwd_load(W, t, w, p, C, chi2, sf) && !w.seed_fail;
      } else {
        live = false;
      }
    }
    if (!__any_sync(FULL_MASK, go)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    if (go) {
      for (int k = 0; k < max(kc.inner_steps, 1) && go; k++) {
        // the lane's output pointers are formed at each step from t, not
        // kept across the refill logic (4 + 2 registers: no spills at 72)
        w.hits = o.hits + t * NROW;
        w.hrow = o.hrow + t * NROW;
        w.cn = cn;
        go = fwd_step<false, MINB == 4>(g, up_m, kc, sX, sYH, w, p, D, C, chi2, tl, sf);
      }
      dirty = true;
    }
  }
  tl.flush(cn, PH_FOLLOW_P2);
}

__device__ __forceinline__ bool bwd_zone(const GridView& g, const KConst& kc, const float* sX, const float* sYH,
                                         Lane& w, TrkState& p, double* D, float* C, Chi2Acc& chi2, LocalTally& tl,
                                         double* snap, float* so, int cap) {
  bool go = true;
  for (int k = 0; go && w.nupd < w.zend && (cap == 0 || k < cap); k++)
    go = bwd_step<true>(g, kc, sX, sYH, w, p, D, C, chi2, tl, snap, so);
  return go;
}
// The end of a backward zone kernel's tracklet: its FP64 covariance moved
// to C if the pass ended inside the zone, the output snapshot taken, and
// what the later phases read parked.
__device__ __forceinline__ void zone_bwd_end(FollowWork* W, int64_t t, Lane& w, const TrkState& p, const double* D,
                                             float* C, const Chi2Acc& chi2, const double* snap, float* so, bool go) {
  if (w.nupd < w.zend) {
#pragma unroll
    for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
  }
  zone_snap_take(w, snap, so);
  zone_bwd_store(W, t, w, p, C, chi2, so, go);
}

// Phase 3: re-seed at the outermost forward cluster and run the backward
// pass while its covariance is in FP64 (warps take 32 tracklets at a time,
// as phase 1; the zone's first kc.zone_steps[1] steps, the rest in the tail
// kernel k_follow_p3t).
__global__ void __launch_bounds__(128, 4) k_follow_p3(GridView g, KConst kc, FollowOut o, FollowWork* W,
                                                   ZoneTail zt, WorkOrder next, int chunk, int nchunk,
                                                   Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  __shared__ double sSnap[15 * SNAP_STRIDE];
  __shared__ float sOut[OUT_WORDS * SNAP_STRIDE];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  double* snap = sSnap + threadIdx.x;
  float* so = sOut + threadIdx.x;
  const Chunk ch = chunk_range(cn->n_tracklets, chunk, nchunk);
  LocalTally tl;
  double D[15];
  float C[15];
  for (;;) {
    const int64_t t = ch.begin + warp_fetch(work_counter(cn, PH_FOLLOW_P3, chunk), FULL_MASK);
    if (__shfl_sync(FULL_MASK, t, 0) >= ch.end) break;
    const bool valid = t < ch.end;
    Lane w;
    TrkState p;
    Chi2Acc chi2;
    bool go = false;
    if (valid) {
      zone_bwd_load(W, t, w, p);
      w.hits = o.hits + t * NROW;
      w.hrow = o.hrow + t * NROW;
      w.cn = cn;
      w.snap = false;
      if (!w.seed_fail) {
        chi2.reset();
        w.kf = w.nf - 2;
        next_fwd_hit(w, g);
        w.misses = 0;
        reseed_cov(kc, D, C);
        w.nupd = 0;
        w.zend = kc.fp64_updates;
        go = true;
      }
    }
    __syncwarp();  // the zones of the warp's lanes start together
    const bool run = go;
    if (run) {
      const bool zone0 = kc.fp64_updates > 0;
      lane_update<true>(w, kc, p, zone0, D, C, __ldg(g.yz + w.hits[w.nf - 1]), chi2, 1, true);  // diagonal seed
      w.dg = zone0;
      if (zone0) tl.upd64++;
      else tl.upd32++;
      keep_output<true>(w, p, w.nupd < w.zend, D, C, chi2, snap, so);
    }
    // round 0: the in-step rows; round 1: the rest of a zone that found no
    // tail slot (one copy of the row step in the code)
    int64_t slot = -1;
#pragma unroll 1
    for (int round = 0; round < 2; round++) {
      if (go && slot < 0) go = bwd_zone(g, kc, sX, sYH, w, p, D, C, chi2, tl, snap, so, round ? 0 : kc.zone_steps[1]);
      if (round) break;
      slot = tail_claim(kc, cn, 1, chunk, nchunk, go && w.nupd < w.zend);
    }
    if (run) {
      if (slot >= 0) {
        tail_park(zt, slot, t, D);
        W[t].w.zend = w.zend;
      }
      zone_bwd_end(W, t, w, p, D, C, chi2, snap, so, go);
    } else if (valid) {
      W[t].go = 0;  // a seed failure: the later phases read only the lane's forward fields
    }
    order_count(next, t, valid && slot < 0, go ? p.row : 0);  // rows left inward
  }
  tl.flush(cn, PH_FOLLOW_P3);
}

// Zone tail of phase 3: the backward zones phase 3 parked, lanes refilling
// as in k_follow_p1t.
__global__ void __launch_bounds__(128, 4) k_follow_p3t(GridView g, KConst kc, FollowOut o, FollowWork* W,
                                                    ZoneTail zt, WorkOrder next, int chunk, int nchunk,
                                                    Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  __shared__ double sSnap[15 * SNAP_STRIDE];
  __shared__ float sOut[OUT_WORDS * SNAP_STRIDE];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  double* snap = sSnap + threadIdx.x;
  float* so = sOut + threadIdx.x;
  const int64_t n = min((int64_t)cn->zone_pend[1 * MAX_CHUNKS + chunk], tail_size(kc, chunk, nchunk));
  const int64_t base = tail_base(kc, 1, chunk, nchunk);
  LocalTally tl;
  double D[15];
  float C[15];
  Lane w;
  TrkState p;
  Chi2Acc chi2;
  int64_t t = -1;
  bool zgo = false, pass = false, live = true;
  for (;;) {
    const unsigned need = refill_mask(live && !zgo, zgo, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (t >= 0) zone_bwd_end(W, t, w, p, D, C, chi2, snap, so, pass);
      order_count(next, t, t >= 0, pass ? p.row : 0, need);  // rows left inward
      const int64_t k = warp_fetch(work_counter(cn, PH_FOLLOW_P3T, chunk), need);
      t = -1;
      live = k < n;
      if (live) {
        t = zt.list[base + k];
        zone_tail_bwd_load(W, t, w, p, chi2, so);
        w.hits = o.hits + t * NROW;
        w.hrow = o.hrow + t * NROW;
        w.cn = cn;
#pragma unroll
        for (int i = 0; i < 15; i++) D[i] = zt.cov[(base + k) * 15 + i];
        pass = true;
        zgo = w.nupd < w.zend;
      }
    }
    if (!__any_sync(FULL_MASK, zgo)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    if (zgo) {
      pass = bwd_step<true>(g, kc, sX, sYH, w, p, D, C, chi2, tl, snap, so);
      zgo = pass && w.nupd < w.zend;
    }
  }
  tl.flush(cn, PH_FOLLOW_P3T);
}

// Phase 4r: the binary32 refit of the forward clusters below the FP64 zone
// (rows from the zone's end down to the chain's first row r0; an update
// wherever a forward cluster sits).  Apart from phase 4 its warps take no
// candidate searches, so their lanes step together; phase 4 takes the
// inward extension below r0.  Lanes refill as in phase 2; a tracklet whose
// refit rows are done (or whose pass ended) is parked again only if it
// advanced.
template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_follow_p4r(GridView g, KConst kc, FollowOut o, FollowWork* W,
                                                    const int32_t* __restrict__ order, int chunk, int nchunk,
                                                    Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  __shared__ float sOut[OUT_WORDS * SNAP_STRIDE];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  float* so = sOut + threadIdx.x;
  const int32_t T = cn->n_tracklets;
  const Chunk ch = chunk_range(T, chunk, nchunk);
  LocalTally tl;
  double D[15];  // unused in this phase (the zone is over)
  float C[15];
  Lane w;
  TrkState p;
  Chi2Acc chi2;
  chi2.reset();
  int64_t t = -1;
  bool go = false;     // the lane's tracklet has refit rows left
  bool pass = false;   // its backward pass goes on
  bool live = true;
  bool dirty = false;
  for (;;) {
    const unsigned need = refill_mask(live && !go, go, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (dirty) bwd_store(W, t, w, p, C, chi2, so, pass);
      const int64_t idx = ch.begin + warp_fetch(work_counter(cn, PH_FOLLOW_P4R, chunk), need);
      t = idx < ch.end ? (order ? order[idx] : idx) : T;
      dirty = false;
      if (t < T) {
        pass = bwd_load(W, t, w, p, C, chi2, so);
        go = pass && p.row > w.r0;
      } else {
        live = false;
      }
    }
    if (!__any_sync(FULL_MASK, go)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    if (go) {
      for (int k = 0; k < max(kc.inner_steps, 1) && go; k++) {
        w.hits = o.hits + t * NROW;  // formed at each step, as in phase 2
        w.hrow = o.hrow + t * NROW;
        w.cn = cn;
        pass = bwd_step<false, BW_REFIT>(g, kc, sX, sYH, w, p, D, C, chi2, tl, nullptr, so);
        go = pass && p.row > w.r0;
      }
      dirty = true;
    }
  }
  tl.flush(cn, PH_FOLLOW_P4R);
}

// Output of one tracklet from its phase-4 slot (out_put).
__device__ __forceinline__ void write_follow_output(const FollowOut& o, int64_t t, const Lane& w, float zref0,
                                                    const float* so) {
  if (w.seed_fail) {
    o.n[t] = 0;
    o.nf[t] = 0;
    o.nb[t] = 0;
    o.flags[t] = (int32_t)(w.flags | TF_SEED_FAIL);
    o.row[t] = w.r0;
#pragma unroll
    for (int i = 0; i < 5; i++) o.par[t * 5 + i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 15; i++) o.cov[t * 15 + i] = 0.0f;
    o.zref[t] = zref0;
    o.chi2[t] = 0.0;
    return;
  }
  o.n[t] = w.nf + w.nb;
  o.nf[t] = w.nf;
  o.nb[t] = w.nb;
  o.flags[t] = (int32_t)w.flags;
  o.row[t] = __float_as_int(so[0]);
#pragma unroll
  for (int i = 0; i < 5; i++) o.par[t * 5 + i] = so[(1 + i) * SNAP_STRIDE];
  o.zref[t] = so[6 * SNAP_STRIDE];
#pragma unroll
  for (int i = 0; i < 15; i++) o.cov[t * 15 + i] = so[(7 + i) * SNAP_STRIDE];
  Chi2Acc c;
  c.total = __hiloint2double(__float_as_int(so[22 * SNAP_STRIDE]), __float_as_int(so[23 * SNAP_STRIDE]));
  c.part = so[24 * SNAP_STRIDE];
  o.chi2[t] = c.value();
}

// Phase 4: the rest of the backward pass (FP32, lanes refill as in phase 2)
// and the outputs.  M = BW_EXTEND after phase 4r, which has made every refit
// row: the inward extension below the chain's first row.  M = BW_ANY without
// phase 4r, on batches bound by their longest tracklet, where a second
// kernel between refit and extension would lengthen that tracklet's path.
template <int MINB, int M>
__global__ void __launch_bounds__(128, MINB) k_follow_p4(GridView g, const int32_t* __restrict__ tl_start, KConst kc,
                                                   FollowOut o, FollowWork* W, const int32_t* __restrict__ order,
                                                   int chunk, int nchunk, Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  __shared__ float sOut[OUT_WORDS * SNAP_STRIDE];
  load_tables(sX, sYH);
  if (fatal(cn)) return;
  float* so = sOut + threadIdx.x;
  const int32_t T = cn->n_tracklets;
  const Chunk ch = chunk_range(T, chunk, nchunk);
  LocalTally tl;
  double D[15];  // unused in this phase (the zone is over)
  float C[15];
  Lane w;
  TrkState p;
  Chi2Acc chi2;
  chi2.reset();
  int64_t t = -1;
  bool go = false, live = true;
  for (;;) {
    const unsigned need = refill_mask(live && !go, go, kc.refill);
    if (need & (1u << (threadIdx.x & 31))) {
      if (t >= 0) write_follow_output(o, t, w, __ldg(g.yz + tl_start[t]).y, so);
      const int64_t idx = ch.begin + warp_fetch(work_counter(cn, PH_FOLLOW_P4, chunk), need);
      t = idx < ch.end ? (order ? order[idx] : idx) : T;
      if (t < T) {
        go = bwd_load(W, t, w, p, C, chi2, so);
        w.hits = o.hits + t * NROW;
        w.hrow = o.hrow + t * NROW;
        w.cn = cn;
      } else {
        live = false;
      }
    }
    if (!__any_sync(FULL_MASK, go)) {
      if (!__any_sync(FULL_MASK, live)) break;
      continue;
    }
    for (int k = 0; k < max(kc.inner_steps, 1) && go; k++)
      go = bwd_step<false, M>(g, kc, sX, sYH, w, p, D, C, chi2, tl, nullptr, so);
  }
  tl.flush(cn, PH_FOLLOW_P4);
}

}  // namespace tpc
