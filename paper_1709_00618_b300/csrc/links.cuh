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
__global__ void __launch_bounds__(256) k_neighbours(const float2* __restrict__ yz, const int32_t* __restrict__ rs_of,
                                                    const RsParams* __restrict__ par,
                                                    const int32_t* __restrict__ bin_start, KConst kc,
                                                    int32_t* __restrict__ up, int32_t* __restrict__ dn,
                                                    uint8_t* __restrict__ tie, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  const float WY = kc.wy, WZ = kc.wz;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    int rs = __ldg(rs_of + c);
    int row = rs % NROW;
    int bu = -1, bd = -1;
    uint8_t tflag = 0;
    if (row >= 1 && row <= NROW - 2) {
      RsParams pd = load_params(par + rs - 1), pu = load_params(par + rs + 1);
      if (pd.count > 0 && pu.count > 0) {
        float2 me = __ldg(yz + c);
        float xm = g_row_x[row - 1], x0 = g_row_x[row], xp = g_row_x[row + 1];
        float f = __fdiv_rn(__fsub_rn(x0, xm), __fsub_rn(xp, xm));
        float yld = -g_row_yhi[row - 1], ylu = -g_row_yhi[row + 1];
        int dy0, dy1, dz0, dz1, uy0, uy1, uz0, uz1;
        bin_range(me.x - WY, me.x + WY, yld, pd.inv_y, pd.n_y, dy0, dy1);
        bin_range(me.y - WZ, me.y + WZ, pd.z_lo, pd.inv_z, pd.n_z, dz0, dz1);
        bin_range(me.x - WY, me.x + WY, ylu, pu.inv_y, pu.n_y, uy0, uy1);
        bin_range(me.y - WZ, me.y + WZ, pu.z_lo, pu.inv_z, pu.n_z, uz0, uz1);
        float best = __int_as_float(0x7F800000), second = best;
        for (int izd = dz0; izd <= dz1; izd++) {
          int rowd = pd.bin_base + izd * pd.n_y;
          int a = __ldg(bin_start + rowd + dy0), b = __ldg(bin_start + rowd + dy1 + 1);
          for (int d = a; d < b; d++) {
            float2 pdv = __ldg(yz + d);
            float ddy = __fsub_rn(pdv.x, me.x), ddz = __fsub_rn(pdv.y, me.y);
            if (!(fabsf(ddy) <= WY && fabsf(ddz) <= WZ)) continue;
            for (int izu = uz0; izu <= uz1; izu++) {
              int rowu = pu.bin_base + izu * pu.n_y;
              int a2 = __ldg(bin_start + rowu + uy0), b2 = __ldg(bin_start + rowu + uy1 + 1);
              for (int u = a2; u < b2; u++) {
                float2 puv = __ldg(yz + u);
                if (!(fabsf(__fsub_rn(puv.x, me.x)) <= WY && fabsf(__fsub_rn(puv.y, me.y)) <= WZ)) continue;
                float ey = __fadd_rn(ddy, __fmul_rn(__fsub_rn(puv.x, pdv.x), f));
                float ez = __fadd_rn(ddz, __fmul_rn(__fsub_rn(puv.y, pdv.y), f));
                float D = __fadd_rn(__fmul_rn(ey, ey), __fmul_rn(ez, ez));
                bool better = D < best || (D == best && (d < bd || (d == bd && u < bu)));
                if (bd < 0 || better) {
                  if (bd >= 0) second = fminf(second, best);
                  best = D;
                  bd = d;
                  bu = u;
                } else {
                  second = fminf(second, D);
                }
              }
            }
          }
        }
        if (bd >= 0 && best <= kc.d_max) {
          tflag = (second != __int_as_float(0x7F800000) &&
                   fabsf(__fsub_rn(second, best)) <= __fmul_rn(1e-6f, fmaxf(best, 1e-12f)))
                      ? 1
                      : 0;
        } else {
          bd = bu = -1;
        }
      }
    }
    up[c] = bu;
    dn[c] = bd;
    tie[c] = tflag;
  }
}

// a4 + a5: keep links both ends agree on; a cluster with a kept upward link
// and no kept downward link starts a chain; walk it and flag chains of at
// least min_chain clusters.
__global__ void k_chains(const int32_t* __restrict__ up, const int32_t* __restrict__ dn, KConst kc,
                         int32_t* __restrict__ up_m, int32_t* __restrict__ dn_m, int32_t* __restrict__ flag,
                         int32_t* __restrict__ clen, int32_t* __restrict__ cend, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t c = gtid(); c < n; c += gstride()) {
    int u = up[c], d = dn[c];
    int um = (u >= 0 && __ldg(dn + u) == (int)c) ? u : -1;
    int dm = (d >= 0 && __ldg(up + d) == (int)c) ? d : -1;
    up_m[c] = um;
    dn_m[c] = dm;
    int f = 0;
    if (um >= 0 && dm < 0) {
      int len = 1, k = (int)c;
      for (;;) {
        int uk = __ldg(up + k);
        if (uk < 0 || __ldg(dn + uk) != k) break;
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
