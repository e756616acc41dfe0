// a3 cellular-automaton neighbour finder (Fig. 1a), a4 link cleaning and
// a5 chain starts (Fig. 1b).
#pragma once
#include "common.cuh"

namespace tpc {

// Bin index range of a row-sector covering [v0, v1], both edges moved out by
// a margin far above their binary32 rounding so that no cluster inside the
// window is dropped (the caller applies the exact test to every candidate).
__device__ __forceinline__ void bin_range(float v0, float v1, float lo, float inv, int nb, int& i0, int& i1) {
  const float m = 1e-3f + 2e-6f * fmaxf(fabsf(v0), fabsf(v1));
  float f0 = floorf((v0 - m - lo) * inv), f1 = floorf((v1 + m - lo) * inv);
  float top = (float)(nb - 1);
  i0 = !(f0 >= 0.0f) ? 0 : (f0 > top ? nb - 1 : (int)f0);
  i1 = !(f1 >= 0.0f) ? 0 : (f1 > top ? nb - 1 : (int)f1);
}

// For every cluster on rows 1..157: the pair (d on r-1, u on r+1) inside the
// link windows minimising the squared deviation of the cluster from the d-u
// chord, ties to the lower sorted index of d, then of u; accepted if
// D <= d_max.  D is evaluated in binary32 with one rounding per operation in
// the order of the reading, so the choice is reproducible bit for bit; the
// pick is a lexicographic minimum, so it does not depend on the order in
// which candidates are visited.
//
// One lane per cluster, consecutive clusters of the sorted order in a warp
// (neighbouring windows, so candidate loads hit in L1).  The lane scans the
// bins of its row r+1 window once and keeps the in-window candidates in its
// column of a shared list, then scans its row r-1 window and pairs every
// in-window d with that list: the work is (scanned candidates of both rows)
// + (pairs), not (in-window d) x (scanned u) as a nested scan would be.  A
// lane with more than NB_ULIST in-window candidates on row r+1 (dense
// pile-ups) falls back to the nested scan.
constexpr int NB_THREADS = 256;
constexpr int NB_ULIST = 8;

struct PairPick {
  float best, second;
  int32_t d, u;  // -1: no pair yet
};

// True if (D, d, u) precedes the pick's best pair.
__device__ __forceinline__ bool pair_before(float D, int32_t d, int32_t u, const PairPick& b) {
  return b.d < 0 || D < b.best || (D == b.best && (d < b.d || (d == b.d && u < b.u)));
}

__device__ __forceinline__ void pair_add(PairPick& b, float D, int32_t d, int32_t u) {
  if (pair_before(D, d, u, b)) {
    if (b.d >= 0) b.second = fminf(b.second, b.best);
    b.best = D;
    b.d = d;
    b.u = u;
  } else {
    b.second = fminf(b.second, D);
  }
}

// D of cluster (yc, zc) against the pair (d, u), in the reading's order.
__device__ __forceinline__ float pair_dev(float2 me, float2 pd, float2 pu, float f) {
  const float ddy = __fsub_rn(pd.x, me.x), ddz = __fsub_rn(pd.y, me.y);
  const float ey = __fadd_rn(ddy, __fmul_rn(__fsub_rn(pu.x, pd.x), f));
  const float ez = __fadd_rn(ddz, __fmul_rn(__fsub_rn(pu.y, pd.y), f));
  return __fadd_rn(__fmul_rn(ey, ey), __fmul_rn(ez, ez));
}

__device__ __forceinline__ bool in_window(float2 q, float2 me, float WY, float WZ) {
  return fabsf(__fsub_rn(q.x, me.x)) <= WY && fabsf(__fsub_rn(q.y, me.y)) <= WZ;
}

// A lane's search window on one candidate row (global bin numbering).
struct NbWin {
  int base, ny, y0, y1, z0, z1;
};

// All in-window (d, u) pairs of one centre cluster by a nested scan (the
// fallback for dense windows).
__device__ __noinline__ void nb_nested(const float2* __restrict__ yz, const int32_t* __restrict__ bin_start,
                                       float2 me, float f, float WY, float WZ, NbWin wd, NbWin wu, PairPick& b) {
  for (int izd = wd.z0; izd <= wd.z1; izd++) {
    const int jd = wd.base + izd * wd.ny;
    const int a = __ldg(bin_start + jd + wd.y0), e = __ldg(bin_start + jd + wd.y1 + 1);
    for (int d = a; d < e; d++) {
      const float2 pdv = __ldg(yz + d);
      if (!in_window(pdv, me, WY, WZ)) continue;
      for (int izu = wu.z0; izu <= wu.z1; izu++) {
        const int ju = wu.base + izu * wu.ny;
        const int a2 = __ldg(bin_start + ju + wu.y0), e2 = __ldg(bin_start + ju + wu.y1 + 1);
        for (int u = a2; u < e2; u++) {
          const float2 puv = __ldg(yz + u);
          if (!in_window(puv, me, WY, WZ)) continue;
          pair_add(b, pair_dev(me, pdv, puv, f), d, u);
        }
      }
    }
  }
}

// The next-row variant (link_skip), for a cluster without an accepted
// r-1/r+1 pair: the best pair skipping one row on one side, (r-2, r+1) or
// (r-1, r+2), and failing that on both sides, (r-2, r+2) -- the smallest
// skip first, as a further pair on a straight line is as good and would
// break the chain.  Windows scale with the row distance and the chord
// fraction is that of the rows involved (nested scans by one lane: the
// clusters that need it are a minority).
__device__ __noinline__ void nb_skip(const float2* __restrict__ yz, const int32_t* __restrict__ bin_start,
                                     const RsParams* __restrict__ par, int rs, int row, float2 me, const KConst& kc,
                                     PairPick& b) {
  const int dr[3] = {-2, -1, -2}, ur[3] = {1, 2, 2};
  for (int m = 0; m < 3; m++) {
    if (m == 2) {  // both sides skipped: only without an accepted one-sided skip
      if (b.d >= 0 && b.best <= kc.d_max) break;
      b = PairPick{__int_as_float(0x7F800000), __int_as_float(0x7F800000), -1, -1};
    }
    const int rd = row + dr[m], ru = row + ur[m];
    const RsParams pd = load_params(par + rs + dr[m]), pu = load_params(par + rs + ur[m]);
    if (pd.count == 0 || pu.count == 0) continue;
    const float xd = g_row_x[rd], x0 = g_row_x[row], xu = g_row_x[ru];
    const float f = __fdiv_rn(__fsub_rn(x0, xd), __fsub_rn(xu, xd));
    const float WYd = dr[m] == -2 ? kc.wy2 : kc.wy, WZd = dr[m] == -2 ? kc.wz2 : kc.wz;
    const float WYu = ur[m] == 2 ? kc.wy2 : kc.wy, WZu = ur[m] == 2 ? kc.wz2 : kc.wz;
    NbWin wd, wu;
    wd.base = pd.bin_base;
    wd.ny = pd.n_y;
    wu.base = pu.bin_base;
    wu.ny = pu.n_y;
    bin_range(me.x - WYd, me.x + WYd, -g_row_yhi[rd], pd.inv_y, pd.n_y, wd.y0, wd.y1);
    bin_range(me.y - WZd, me.y + WZd, pd.z_lo, pd.inv_z, pd.n_z, wd.z0, wd.z1);
    bin_range(me.x - WYu, me.x + WYu, -g_row_yhi[ru], pu.inv_y, pu.n_y, wu.y0, wu.y1);
    bin_range(me.y - WZu, me.y + WZu, pu.z_lo, pu.inv_z, pu.n_z, wu.z0, wu.z1);
    for (int izd = wd.z0; izd <= wd.z1; izd++) {
      const int jd = wd.base + izd * wd.ny;
      const int a = __ldg(bin_start + jd + wd.y0), e = __ldg(bin_start + jd + wd.y1 + 1);
      for (int d = a; d < e; d++) {
        const float2 pdv = __ldg(yz + d);
        if (!in_window(pdv, me, WYd, WZd)) continue;
        for (int izu = wu.z0; izu <= wu.z1; izu++) {
          const int ju = wu.base + izu * wu.ny;
          const int a2 = __ldg(bin_start + ju + wu.y0), e2 = __ldg(bin_start + ju + wu.y1 + 1);
          for (int u = a2; u < e2; u++) {
            const float2 puv = __ldg(yz + u);
            if (!in_window(puv, me, WYu, WZu)) continue;
            pair_add(b, pair_dev(me, pdv, puv, f), d, u);
          }
        }
      }
    }
  }
}

// Six blocks per SM (40 registers, a few spilled): more resident lanes hide
// more of each lane's dependent loads (10 ms timeframe 8.66 -> 8.11 ms against
// five blocks at 48 registers; eight blocks at 32 registers spill more).
__global__ void __launch_bounds__(NB_THREADS, 6) k_neighbours(const float2* __restrict__ yz,
                                                           const int32_t* __restrict__ rs_of,
                                                           const RsParams* __restrict__ par,
                                                           const int32_t* __restrict__ bin_start, KConst kc,
                                                           int32_t* __restrict__ up, int32_t* __restrict__ dn,
                                                           uint8_t* __restrict__ tie, const Counts* cn) {
  if (fatal(cn)) return;
  // each thread's list of in-window row r+1 candidates, one column per thread
  __shared__ float2 s_upos[NB_ULIST][NB_THREADS];
  __shared__ int32_t s_uidx[NB_ULIST][NB_THREADS];
  const int tid = threadIdx.x;
  const int64_t n = cn->n;
  const float WY = kc.wy, WZ = kc.wz;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    const int rs = __ldg(rs_of + c);
    const int row = rs % NROW;
    PairPick b{__int_as_float(0x7F800000), __int_as_float(0x7F800000), -1, -1};
    if (row >= 1 && row <= NROW - 2) {
      const RsParams pd = load_params(par + rs - 1), pu = load_params(par + rs + 1);
      if (pd.count > 0 && pu.count > 0) {
        const float2 me = __ldg(yz + c);
        const float xm = g_row_x[row - 1], x0 = g_row_x[row], xp = g_row_x[row + 1];
        const float f = __fdiv_rn(__fsub_rn(x0, xm), __fsub_rn(xp, xm));
        NbWin wd, wu;
        wd.base = pd.bin_base;
        wd.ny = pd.n_y;
        wu.base = pu.bin_base;
        wu.ny = pu.n_y;
        bin_range(me.x - WY, me.x + WY, -g_row_yhi[row - 1], pd.inv_y, pd.n_y, wd.y0, wd.y1);
        bin_range(me.y - WZ, me.y + WZ, pd.z_lo, pd.inv_z, pd.n_z, wd.z0, wd.z1);
        bin_range(me.x - WY, me.x + WY, -g_row_yhi[row + 1], pu.inv_y, pu.n_y, wu.y0, wu.y1);
        bin_range(me.y - WZ, me.y + WZ, pu.z_lo, pu.inv_z, pu.n_z, wu.z0, wu.z1);
        // row r+1: the in-window candidates, in sorted order
        int nu = 0;
        for (int iz = wu.z0; iz <= wu.z1; iz++) {
          const int j = wu.base + iz * wu.ny;
          const int a = __ldg(bin_start + j + wu.y0), e = __ldg(bin_start + j + wu.y1 + 1);
          for (int u = a; u < e; u++) {
            const float2 q = __ldg(yz + u);
            if (in_window(q, me, WY, WZ)) {
              if (nu < NB_ULIST) {
                s_upos[nu][tid] = q;
                s_uidx[nu][tid] = u;
              }
              nu++;
            }
          }
        }
        if (nu > NB_ULIST) {
          nb_nested(yz, bin_start, me, f, WY, WZ, wd, wu, b);
        } else if (nu > 0) {
          // row r-1: every in-window d against the list
          for (int iz = wd.z0; iz <= wd.z1; iz++) {
            const int j = wd.base + iz * wd.ny;
            const int a = __ldg(bin_start + j + wd.y0), e = __ldg(bin_start + j + wd.y1 + 1);
            for (int d = a; d < e; d++) {
              const float2 q = __ldg(yz + d);
              if (!in_window(q, me, WY, WZ)) continue;
              for (int k = 0; k < nu; k++) pair_add(b, pair_dev(me, q, s_upos[k][tid], f), d, s_uidx[k][tid]);
            }
          }
        }
      }
    }
    int32_t bu = -1, bd = -1;
    uint8_t tflag = 0;
    if (b.d >= 0 && b.best <= kc.d_max) {
      bd = b.d;
      bu = b.u;
      tflag = (b.second != __int_as_float(0x7F800000) &&
               fabsf(__fsub_rn(b.second, b.best)) <= __fmul_rn(1e-6f, fmaxf(b.best, 1e-12f)))
                  ? 1
                  : 0;
    }
    up[c] = bu;
    dn[c] = bd;
    tie[c] = tflag;
  }
}

// The next-row variant's second pass (launched only with link_skip): every
// cluster on rows 2..156 that k_neighbours left without an accepted pair.
__global__ void k_neighbours_skip(const float2* __restrict__ yz, const int32_t* __restrict__ rs_of,
                                  const RsParams* __restrict__ par, const int32_t* __restrict__ bin_start, KConst kc,
                                  int32_t* __restrict__ up, int32_t* __restrict__ dn, uint8_t* __restrict__ tie,
                                  const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    if (up[c] >= 0) continue;
    const int rs = __ldg(rs_of + c);
    const int row = rs % NROW;
    if (row < 2 || row > NROW - 3) continue;
    PairPick b{__int_as_float(0x7F800000), __int_as_float(0x7F800000), -1, -1};
    nb_skip(yz, bin_start, par, rs, row, __ldg(yz + c), kc, b);
    if (b.d >= 0 && b.best <= kc.d_max) {
      up[c] = b.u;
      dn[c] = b.d;
      tie[c] = (b.second != __int_as_float(0x7F800000) &&
                fabsf(__fsub_rn(b.second, b.best)) <= __fmul_rn(1e-6f, fmaxf(b.best, 1e-12f)))
                   ? 1
                   : 0;
    }
  }
}

// a4: keep the links both ends agree on, and flag the chain starts (a kept
// upward link and no kept downward link).  Also clears the selection's
// owner keys (32- or 64-bit), whose space the grid stage used until now.
__global__ void k_clean(const int32_t* __restrict__ up, const int32_t* __restrict__ dn, int32_t* __restrict__ up_m,
                        int32_t* __restrict__ dn_m, int32_t* __restrict__ start, void* __restrict__ owner,
                        bool key32, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    const int u = up[c], d = dn[c];
    const int um = (u >= 0 && __ldg(dn + u) == (int)c) ? u : -1;
    const int dm = (d >= 0 && __ldg(up + d) == (int)c) ? d : -1;
    up_m[c] = um;
    dn_m[c] = dm;
    start[c] = um >= 0 && dm < 0;
    if (key32) reinterpret_cast<uint32_t*>(owner)[c] = 0u;
    else reinterpret_cast<uint64_t*>(owner)[c] = 0ull;
  }
}

// The chain starts in sorted order (start[] scanned into sidx[]).
__global__ void k_start_list(const int32_t* __restrict__ start, const int32_t* __restrict__ sidx,
                             int32_t* __restrict__ starts, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride())
    if (start[c]) starts[sidx[c]] = (int32_t)c;
}

// a5: walk every chain from its start over the kept links (one dependent
// load per cluster), one thread per start so that every lane walks, and
// flag the chains of at least min_chain clusters (indexed like starts[]).
__global__ void k_chains(const int32_t* __restrict__ up_m, const int32_t* __restrict__ starts, KConst kc,
                         int32_t* __restrict__ flag, int32_t* __restrict__ clen, int32_t* __restrict__ cend,
                         const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t S = cn->n_starts;
  for (int64_t j = gtid(); j < S; j += gstride()) {
    int len = 1, k = starts[j];
    for (int uk = __ldg(up_m + k); uk >= 0; uk = __ldg(up_m + k)) {
      k = uk;
      len++;
    }
    flag[j] = len >= kc.min_chain;
    clen[j] = len;
    cend[j] = k;
  }
}

// Tracklets in the sorted order of their start cluster (idx: flag scanned).
__global__ void k_tracklet_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ idx,
                                   const int32_t* __restrict__ starts, const int32_t* __restrict__ clen,
                                   const int32_t* __restrict__ cend, int32_t* __restrict__ tl_start,
                                   int32_t* __restrict__ tl_len, int32_t* __restrict__ tl_end, Counts* cn,
                                   int64_t tl_cap) {
  if (fatal(cn)) return;
  const int32_t S = cn->n_starts;
  int32_t total = idx[S];
  if (gtid() == 0) cn->n_tracklets = total;
  if (total > tl_cap) {
    if (gtid() == 0) atomicOr(&cn->status, ST_EOVERFLOW);
    return;
  }
  for (int64_t j = gtid(); j < S; j += gstride()) {
    if (!flag[j]) continue;
    int t = idx[j];
    tl_start[t] = starts[j];
    tl_len[t] = clen[j];
    tl_end[t] = cend[j];
  }
}

}  // namespace tpc
