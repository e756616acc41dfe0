// a6 track following (Fig. 1c): one thread per tracklet, whole state in
// registers.  Seed from the chain chord, forward pass over the chain and
// outward with gated pick-up, fresh backward pass refitting the forward
// clusters and extending inward.
#pragma once
#include "kalman.cuh"

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

__device__ __forceinline__ bool outside_sector(const TrkState& p, float yhi_edge, const KConst& kc,
                                               uint32_t& flags) {
  const float lim = yhi_edge;
  const float y = p.y + p.yl;
  if (fabsf(fabsf(y) - lim) <= 1e-3f) flags |= TF_EDGE;
  return fabsf(y) > lim;
}

// Best cluster of row-sector rs for the predicted state: minimum chi2 =
// dy^2/Syy + dz^2/Szz within the gate, ties to the lower sorted index.
__device__ __forceinline__ int pick(const GridView& g, int rs, int row, const Filter& f, const KConst& kc,
                                    const float* sYH, uint32_t& flags) {
  const RsParams P = load_params(g.par + rs);
  if (P.count == 0) return -1;
  const float Syy = f.cyy() + kc.V, Szz = f.czz() + kc.V;
  const float wy = sqrtf(kc.gate * Syy), wz = sqrtf(kc.gate * Szz);
  const float iSyy = 1.0f / Syy, iSzz = 1.0f / Szz;
  const float y = f.p.y, yl = f.p.yl, zr = f.p.z, zl = f.p.zl, zref = f.p.zref;
  const float zabs = zref + zr;
  int iy0, iy1, iz0, iz1;
  {
    const float yl = -sYH[row];
    float a0 = floorf((y - wy - yl) * P.inv_y) - 1.0f, a1 = floorf((y + wy - yl) * P.inv_y) + 1.0f;
    float b0 = floorf((zabs - wz - P.z_lo) * P.inv_z) - 1.0f, b1 = floorf((zabs + wz - P.z_lo) * P.inv_z) + 1.0f;
    const float ty = (float)(P.n_y - 1), tz = (float)(P.n_z - 1);
    iy0 = !(a0 >= 0.0f) ? 0 : (a0 > ty ? P.n_y - 1 : (int)a0);
    iy1 = !(a1 >= 0.0f) ? 0 : (a1 > ty ? P.n_y - 1 : (int)a1);
    iz0 = !(b0 >= 0.0f) ? 0 : (b0 > tz ? P.n_z - 1 : (int)b0);
    iz1 = !(b1 >= 0.0f) ? 0 : (b1 > tz ? P.n_z - 1 : (int)b1);
  }
  const float gate = kc.gate, eps = kc.taint;
  float b1v = __int_as_float(0x7F800000), b2v = b1v;
  int best = -1;
  for (int iz = iz0; iz <= iz1; iz++) {
    const int base = P.bin_base + iz * P.n_y;
    const int a = __ldg(g.bin_start + base + iy0), b = __ldg(g.bin_start + base + iy1 + 1);
    f.tally->cand += (unsigned)(b - a);
    for (int c = a; c < b; c++) {
      const float2 q = __ldg(g.yz + c);
      const float dy = (q.x - y) - yl;
      const float dz = ((q.y - zref) - zr) - zl;
      const float chi = dy * dy * iSyy + dz * dz * iSzz;
      if (fabsf(chi - gate) <= eps * (1.0f + gate)) flags |= TF_GATE;
      if (!(chi <= gate)) continue;
      if (chi < b1v || (chi == b1v && c < best)) {
        b2v = b1v;
        b1v = chi;
        best = c;
      } else if (chi < b2v) {
        b2v = chi;
      }
    }
  }
  if (best >= 0 && b2v != __int_as_float(0x7F800000) && b2v - b1v <= eps * (1.0f + b1v)) flags |= TF_TIE;
  return best;
}

struct Saved {
  TrkState p;
  float C[15];
  double chi2;
};

__device__ __forceinline__ void save(Saved& s, const Filter& f) {
  s.p = f.p;
  f.cov_out(s.C);
  s.chi2 = f.chi2;
}

__global__ void __launch_bounds__(128) k_follow(GridView g, const int32_t* __restrict__ tl_start,
                                                const int32_t* __restrict__ tl_len,
                                                const int32_t* __restrict__ tl_end,
                                                const int32_t* __restrict__ up_m, KConst kc, FollowOut o,
                                                Counts* cn) {
  __shared__ float sX[NROW + 1], sYH[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) {
    sX[i] = g_row_x[i];
    sYH[i] = g_row_yhi[i];
  }
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t T = cn->n_tracklets;
  Tally tally;
  for (int64_t t = gtid(); t < T; t += gstride()) {
    int32_t* hits = o.hits + t * NROW;
    uint8_t* hrow = o.hrow + t * NROW;
    uint32_t flags = 0;
    const int c0 = tl_start[t], L = tl_len[t], cl = tl_end[t];
    const int rs0 = __ldg(g.rs_of + c0);
    const int ubase = rs0 - rs0 % NROW, r0 = rs0 % NROW;
    const float2 P0 = __ldg(g.yz + c0), P1 = __ldg(g.yz + cl);
    Filter f;
    f.tally = &tally;
    {
      const float x0 = sX[r0], x1 = sX[r0 + L - 1];
      const float dX = x1 - x0, dY = P1.x - P0.x, dZ = P1.y - P0.y;
      const float Lc = sqrtf(dX * dX + dY * dY);
      f.seed(r0, x0, P0.x, P0.y, dY / Lc, dZ / Lc, 0.0f);
    }
    f.reset_cov(kc);
    f.update(P0.x, P0.y, kc);
    int nf = 0, nb = 0;
    hits[nf] = c0;
    hrow[nf++] = (uint8_t)r0;
    bool seed_ok = true;
    int k = c0;
    for (int i = 1; i < L; i++) {
      k = __ldg(up_m + k);
      if (!f.propagate(r0 + i, sX[r0 + i], kc, flags)) {
        seed_ok = false;
        break;
      }
      const float2 P = __ldg(g.yz + k);
      f.update(P.x, P.y, kc);
      hits[nf] = k;
      hrow[nf++] = (uint8_t)(r0 + i);
    }
    if (!seed_ok) {
      o.n[t] = 0;
      o.nf[t] = 0;
      o.nb[t] = 0;
      o.flags[t] = (int32_t)(flags | TF_SEED_FAIL);
      o.row[t] = r0;
#pragma unroll
      for (int i = 0; i < 5; i++) o.par[t * 5 + i] = 0.0f;
#pragma unroll
      for (int i = 0; i < 15; i++) o.cov[t * 15 + i] = 0.0f;
      o.zref[t] = P0.y;
      o.chi2[t] = 0.0;
      continue;
    }
    // forward extension
    TrkState fwd = f.p;
    int r_last = r0 + L - 1, misses = 0;
    for (int r = r_last + 1; r < NROW; r++) {
      if (!f.propagate(r, sX[r], kc, flags)) break;
      if (outside_sector(f.p, f.p.x * 0.17632698070846498f + kc.edge, kc, flags)) break;
      const int c = pick(g, ubase + r, r, f, kc, sYH, flags);
      if (c >= 0) {
        const float2 P = __ldg(g.yz + c);
        f.update(P.x, P.y, kc);
        hits[nf] = c;
        hrow[nf++] = (uint8_t)r;
        fwd = f.p;
        r_last = r;
        misses = 0;
      } else if (++misses >= kc.max_miss) {
        break;
      }
    }
    // backward pass: forward state at the outermost cluster, fresh covariance
    f.p = fwd;
    f.reset_cov(kc);
    {
      const float2 P = __ldg(g.yz + hits[nf - 1]);
      f.update(P.x, P.y, kc);
    }
    Saved sv;
    save(sv, f);
    int kf = nf - 2;
    bool ok = true;
    for (int r = r_last - 1; r >= r0; r--) {
      if (!f.propagate(r, sX[r], kc, flags)) {
        ok = false;
        flags |= TF_BACK_FAIL;
        break;
      }
      if (kf >= 0 && hrow[kf] == r) {
        const float2 P = __ldg(g.yz + hits[kf]);
        f.update(P.x, P.y, kc);
        kf--;
        save(sv, f);
      }
    }
    if (ok) {
      misses = 0;
      for (int r = r0 - 1; r >= 0; r--) {
        if (!f.propagate(r, sX[r], kc, flags)) break;
        if (outside_sector(f.p, f.p.x * 0.17632698070846498f + kc.edge, kc, flags)) break;
        const int c = pick(g, ubase + r, r, f, kc, sYH, flags);
        if (c >= 0) {
          const float2 P = __ldg(g.yz + c);
          f.update(P.x, P.y, kc);
          hits[nf + nb] = c;
          hrow[nf + nb] = (uint8_t)r;
          nb++;
          save(sv, f);
          misses = 0;
        } else if (++misses >= kc.max_miss) {
          break;
        }
      }
    }
    o.n[t] = nf + nb;
    o.nf[t] = nf;
    o.nb[t] = nb;
    o.flags[t] = (int32_t)flags;
    o.row[t] = sv.p.row;
    o.par[t * 5 + 0] = sv.p.y + sv.p.yl;
    o.par[t * 5 + 1] = sv.p.z + sv.p.zl;
    o.par[t * 5 + 2] = sv.p.s + sv.p.sl;
    o.par[t * 5 + 3] = sv.p.t;
    o.par[t * 5 + 4] = sv.p.q;
    o.zref[t] = sv.p.zref;
#pragma unroll
    for (int i = 0; i < 15; i++) o.cov[t * 15 + i] = sv.C[i];
    o.chi2[t] = sv.chi2;
  }
  tally.flush(cn);
}

}  // namespace tpc
