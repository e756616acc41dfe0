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
// the order of the reading, so the choice is reproducible bit for bit.
//
// A group of NB_G lanes handles one cluster: the lanes scan the candidate
// bins of both rows together, stage the in-window candidates in shared
// memory, share the d x u pairs and merge their best pairs with shuffles,
// so the work of a cluster no longer depends on one lane's loop lengths.
// A cluster with more than NB_CAP in-window candidates on a row (dense
// pile-ups) is finished by the group's first lane alone.
#ifndef TPC_NB_G
#define TPC_NB_G 4
#endif
#ifndef TPC_NB_CAP
#define TPC_NB_CAP 16
#endif
constexpr int NB_G = TPC_NB_G;
constexpr int NB_CAP = TPC_NB_CAP;
constexpr int NB_THREADS = 256;

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

// One lane over all pairs (the fallback for dense windows).
__device__ __noinline__ void serial_pairs(const float2* __restrict__ yz, const int32_t* __restrict__ bin_start,
                                          float2 me, float f, float WY, float WZ, int bd_base, int bd_ny,
                                          int dy0, int dy1, int dz0, int dz1, int bu_base, int bu_ny, int uy0,
                                          int uy1, int uz0, int uz1, PairPick& b) {
  for (int izd = dz0; izd <= dz1; izd++) {
    const int rowd = bd_base + izd * bd_ny;
    const int a = __ldg(bin_start + rowd + dy0), e = __ldg(bin_start + rowd + dy1 + 1);
    for (int d = a; d < e; d++) {
      const float2 pdv = __ldg(yz + d);
      if (!in_window(pdv, me, WY, WZ)) continue;
      for (int izu = uz0; izu <= uz1; izu++) {
        const int rowu = bu_base + izu * bu_ny;
        const int a2 = __ldg(bin_start + rowu + uy0), e2 = __ldg(bin_start + rowu + uy1 + 1);
        for (int u = a2; u < e2; u++) {
          const float2 puv = __ldg(yz + u);
          if (!in_window(puv, me, WY, WZ)) continue;
          pair_add(b, pair_dev(me, pdv, puv, f), d, u);
        }
      }
    }
  }
}

// The group stages the in-window candidates of one row; returns their
// count (> NB_CAP: too many, nothing beyond NB_CAP stored).
__device__ __forceinline__ int stage_row(const float2* __restrict__ yz, const int32_t* __restrict__ bin_start,
                                         float2 me, float WY, float WZ, int base, int ny, int y0, int y1, int z0,
                                         int z1, float2* s_pos, int32_t* s_idx, int sub, unsigned gmask) {
  int cnt = 0;
  const unsigned below = gmask & ((1u << (threadIdx.x & 31)) - 1u);
  for (int iz = z0; iz <= z1; iz++) {
    const int row = base + iz * ny;
    const int a = __ldg(bin_start + row + y0), e = __ldg(bin_start + row + y1 + 1);
    for (int k0 = a; k0 < e; k0 += NB_G) {
      const int k = k0 + sub;
      float2 q = make_float2(0.0f, 0.0f);
      const bool hit = k < e && in_window(q = __ldg(yz + min(k, e - 1)), me, WY, WZ);
      const unsigned m = __ballot_sync(gmask, hit);
      const int pos = cnt + __popc(m & below);
      if (hit && pos < NB_CAP) {
        s_pos[pos] = q;
        s_idx[pos] = k;
      }
      cnt += __popc(m);
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(NB_THREADS) k_neighbours(const float2* __restrict__ yz,
                                                           const int32_t* __restrict__ rs_of,
                                                           const RsParams* __restrict__ par,
                                                           const int32_t* __restrict__ bin_start, KConst kc,
                                                           int32_t* __restrict__ up, int32_t* __restrict__ dn,
                                                           uint8_t* __restrict__ tie, const Counts* cn) {
  if (fatal(cn)) return;
  __shared__ float2 s_dp[NB_THREADS / NB_G][NB_CAP], s_up[NB_THREADS / NB_G][NB_CAP];
  __shared__ int32_t s_di[NB_THREADS / NB_G][NB_CAP], s_ui[NB_THREADS / NB_G][NB_CAP];
  const int64_t n = cn->n;
  const float WY = kc.wy, WZ = kc.wz;
  const int sub = threadIdx.x & (NB_G - 1), grp = threadIdx.x / NB_G;
  const unsigned gmask = ((1u << NB_G) - 1u) << ((threadIdx.x & 31) & ~(NB_G - 1));
  const int64_t groups = gstride() / NB_G;
  for (int64_t c = gtid() / NB_G; c < n; c += groups) {  // group-uniform
    const int rs = __ldg(rs_of + c);
    const int row = rs % NROW;
    PairPick b{__int_as_float(0x7F800000), __int_as_float(0x7F800000), -1, -1};
    if (row >= 1 && row <= NROW - 2) {
      const RsParams pd = load_params(par + rs - 1), pu = load_params(par + rs + 1);
      if (pd.count > 0 && pu.count > 0) {
        const float2 me = __ldg(yz + c);
        const float xm = g_row_x[row - 1], x0 = g_row_x[row], xp = g_row_x[row + 1];
        const float f = __fdiv_rn(__fsub_rn(x0, xm), __fsub_rn(xp, xm));
        const float yld = -g_row_yhi[row - 1], ylu = -g_row_yhi[row + 1];
        int dy0, dy1, dz0, dz1, uy0, uy1, uz0, uz1;
        bin_range(me.x - WY, me.x + WY, yld, pd.inv_y, pd.n_y, dy0, dy1);
        bin_range(me.y - WZ, me.y + WZ, pd.z_lo, pd.inv_z, pd.n_z, dz0, dz1);
        bin_range(me.x - WY, me.x + WY, ylu, pu.inv_y, pu.n_y, uy0, uy1);
        bin_range(me.y - WZ, me.y + WZ, pu.z_lo, pu.inv_z, pu.n_z, uz0, uz1);
        const int nd = stage_row(yz, bin_start, me, WY, WZ, pd.bin_base, pd.n_y, dy0, dy1, dz0, dz1, s_dp[grp],
                                 s_di[grp], sub, gmask);
        const int nu = stage_row(yz, bin_start, me, WY, WZ, pu.bin_base, pu.n_y, uy0, uy1, uz0, uz1, s_up[grp],
                                 s_ui[grp], sub, gmask);
        __syncwarp(gmask);
        if (nd > NB_CAP || nu > NB_CAP) {
          if (sub == 0)
            serial_pairs(yz, bin_start, me, f, WY, WZ, pd.bin_base, pd.n_y, dy0, dy1, dz0, dz1, pu.bin_base,
                         pu.n_y, uy0, uy1, uz0, uz1, b);
        } else {
          for (int p = sub; p < nd * nu; p += NB_G) {
            const int i = p / nu, j = p - i * nu;
            pair_add(b, pair_dev(me, s_dp[grp][i], s_up[grp][j], f), s_di[grp][i], s_ui[grp][j]);
          }
          // merge the lanes' picks: the lexicographic minimum, and the
          // smallest D of every other pair
#pragma unroll
          for (int o = NB_G / 2; o >= 1; o >>= 1) {
            PairPick q;
            q.best = __shfl_xor_sync(gmask, b.best, o);
            q.second = __shfl_xor_sync(gmask, b.second, o);
            q.d = __shfl_xor_sync(gmask, b.d, o);
            q.u = __shfl_xor_sync(gmask, b.u, o);
            if (q.d >= 0 && pair_before(q.best, q.d, q.u, b)) {
              b.second = fminf(q.second, b.d >= 0 ? b.best : b.second);
              b.best = q.best;
              b.d = q.d;
              b.u = q.u;
            } else {
              b.second = fminf(b.second, q.d >= 0 ? q.best : q.second);
              b.second = fminf(b.second, q.second);
            }
          }
        }
        __syncwarp(gmask);  // the staged candidates are reused by the next cluster
      }
    }
    if (sub == 0) {
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
}

// a4: keep the links both ends agree on.
__global__ void k_clean(const int32_t* __restrict__ up, const int32_t* __restrict__ dn, int32_t* __restrict__ up_m,
                        int32_t* __restrict__ dn_m, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    const int u = up[c], d = dn[c];
    up_m[c] = (u >= 0 && __ldg(dn + u) == (int)c) ? u : -1;
    dn_m[c] = (d >= 0 && __ldg(up + d) == (int)c) ? d : -1;
  }
}

// a5: a cluster with a kept upward link and no kept downward link starts a
// chain; walk it over the kept links (one dependent load per cluster) and
// flag chains of at least min_chain clusters.
__global__ void k_chains(const int32_t* __restrict__ up_m, const int32_t* __restrict__ dn_m, KConst kc,
                         int32_t* __restrict__ flag, int32_t* __restrict__ clen, int32_t* __restrict__ cend,
                         const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    int f = 0;
    if (up_m[c] >= 0 && dn_m[c] < 0) {
      int len = 1, k = (int)c;
      for (int uk = __ldg(up_m + k); uk >= 0; uk = __ldg(up_m + k)) {
        k = uk;
        len++;
      }
      if (len >= kc.min_chain) {
        f = 1;
        clen[c] = len;
        cend[c] = k;
      }
    }
    flag[c] = f;
  }
}

__global__ void k_tracklet_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ idx,
                                   const int32_t* __restrict__ clen, const int32_t* __restrict__ cend,
                                   int32_t* __restrict__ tl_start, int32_t* __restrict__ tl_len,
                                   int32_t* __restrict__ tl_end, Counts* cn, int64_t tl_cap) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  int32_t total = idx[n];
  if (gtid() == 0) cn->n_tracklets = total;
  if (total > tl_cap) {
    if (gtid() == 0) atomicOr(&cn->status, ST_EOVERFLOW);
    return;
  }
  for (int64_t c = gtid(); c < n; c += gstride()) {
    if (!flag[c]) continue;
    int t = idx[c];
    tl_start[t] = (int32_t)c;
    tl_len[t] = clen[c];
    tl_end[t] = cend[c];
  }
}

}  // namespace tpc
