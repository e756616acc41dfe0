// Second tracking phase (Sec. 2): the segments found in different sectors
// are merged and the merged tracks refitted.  An inner segment A and an
// outer segment B in neighbouring sectors of one side are compared at B's
// first row: A's fitted state and covariance are turned into B's frame and
// carried there; if their z there lie within the window, chi2 = d^T (C_A +
// C_B)^-1 d over the five parameters.  A pair within chi2_max that is the
// best choice of both A and B is merged; chains of merges are refitted from
// the outermost segment's seed inward, the frame turned between segments.
// Candidates: the segments of every (request, sector) are binned by the z
// of their first row (bins one window wide, hashed into a power-of-two
// count); a warp per segment A carries A over the rows a partner can start
// on, and scans only the bins of the z range it sweeps (plus the window).
// The refit is one thread per chain.
#pragma once
#include "kalman.cuh"

namespace tpc {

constexpr int MERGE_MAX_SEG = 8;  // segments per chain (a longer chain is cut)

struct MergeConst {
  float chi2_max;
  int32_t overlap, min_clusters;
  float window, inv_window;  // z window at B's first row (cm) and its inverse
  int32_t nz_mask;           // z bins per unit - 1 (a power of two minus one)
};

// A segment in its (unit, z bin) cell: the fields the candidate tests read.
struct MergeKey {
  int32_t m;      // track index
  int32_t rows;   // first_row | last_row << 16
  float z, t, q;  // at the first row
  float vt, vq;   // their variances
  int32_t pad;
};
static_assert(sizeof(MergeKey) == 32, "one 32-byte sector per key");

struct MergeBuf {
  int32_t* cell;                  // [M] cell of each segment, -1: takes no part
  int32_t* cell_cnt;              // [units * bins] segments per cell (then the fill cursor)
  int32_t* cell_start;            // [units * bins + 1] exclusive scan
  MergeKey* keys;                 // [M] segments grouped by cell
  int32_t* best_out;              // [M] A's best outer partner
  float* chi2_out;                // [M] its chi2
  float* second_out;              // [M] A's second-best chi2 (for near ties)
  unsigned long long* best_in;    // [M] B's best inner partner: (chi2 bits << 32) | A
  int32_t* link;                  // [M] merged outer partner or -1
  int32_t* has_inner;             // [M]
  int32_t* head;                  // [M + 1] 1 for the innermost segment of a chain
  int32_t* chain_of_head;         // [M + 1] exclusive scan of head
  int32_t* chain;                 // [M] merged track of a segment, -1: none
  tpc_track* merged;              // [M] merged tracks
  int32_t* n;                     // [2] chains, status
};

__device__ __forceinline__ float sector_angle(int s) {
  return (float)(((s % NSEC) % 18) * 20 + 10) * 0.017453292519943295f;
}

__device__ __forceinline__ bool sectors_adjacent(int s1, int s2) {
  if ((s1 % NSEC) / 18 != (s2 % NSEC) / 18) return false;
  const int d = ((s2 % 18) - (s1 % 18) + 18) % 18;
  return d == 1 || d == 17;
}

// The state on its own point expressed in the frame rotated by +beta:
// x' = x cos b + y sin b, y' = -x sin b + y cos b, phi' = phi - b; the
// covariance with the derivatives at fixed x' (J[y][y] = cos phi/cos phi',
// J[s][s] = cos phi'/cos phi, J[z][y] = -t sin b/cos phi').  False if the
// direction would leave the new frame's outward half-plane.
template <typename T>
__device__ __forceinline__ bool rotate_state(TrkState& p, T* C, float beta) {
  float sb, cb;
  sincosf(beta, &sb, &cb);
  const float s = p.s + p.sl, c = sqrtf(fmaxf(1.0f - s * s, 0.0f));
  const float s2 = s * cb - c * sb, c2 = c * cb + s * sb;
  if (!(c2 > 0.05f)) return false;
  const T j00 = (T)(c / c2), j22 = (T)(c2 / c), j10 = (T)(-p.t * sb / c2);
  // C' = J C J^T with J = I except (0,0), (2,2), (1,0)
  T M[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) M[i][j] = C[TPC_CI(i > j ? i : j, i > j ? j : i)];
  T A[5][5];  // J M
#pragma unroll
  for (int j = 0; j < 5; j++) {
    A[0][j] = j00 * M[0][j];
    A[1][j] = M[1][j] + j10 * M[0][j];
    A[2][j] = j22 * M[2][j];
    A[3][j] = M[3][j];
    A[4][j] = M[4][j];
  }
#pragma unroll
  for (int i = 0; i < 5; i++) {  // (J M) J^T, lower triangle
    const T r0 = A[i][0] * j00;
    const T r1 = A[i][1] + A[i][0] * j10;
    const T r2 = A[i][2] * j22;
    const T row[5] = {r0, r1, r2, A[i][3], A[i][4]};
#pragma unroll
    for (int j = 0; j <= i; j++) C[TPC_CI(i, j)] = row[j];
  }
  const float x = p.x, y = p.y + p.yl;
  p.x = x * cb + y * sb;
  p.y = -x * sb + y * cb;
  p.yl = 0.0f;
  p.s = s2;
  p.sl = 0.0f;
  return true;
}

// z bin of a first-row z (clamped so the integer conversion is defined).
__device__ __forceinline__ int64_t merge_zbin(float z, const MergeConst& mc) {
  return (int64_t)floorf(fminf(fmaxf(z * mc.inv_window, -1e15f), 1e15f));
}

__device__ __forceinline__ bool merge_eligible(const tpc_track& T, const MergeConst& mc) {
  return !(T.flags & TF_REFIT_FAIL) && T.n_clusters >= mc.min_clusters && isfinite(T.par[1]);
}

// Cells: every taking-part segment counted in its (request, sector, z bin).
__global__ void k_merge_cells(const tpc_track* __restrict__ tr, MergeConst mc, MergeBuf mb, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const tpc_track T = tr[m];
    int32_t c = -1;
    if (merge_eligible(T, mc)) {
      const int64_t u = (int64_t)T.request * NSEC + T.sector;
      c = (int32_t)(u * (mc.nz_mask + 1) + (merge_zbin(T.par[1], mc) & mc.nz_mask));
      atomicAdd(&mb.cell_cnt[c], 1);
    }
    mb.cell[m] = c;
  }
}

// Keys grouped by cell (the order inside a cell is arbitrary: the pairing
// below does not depend on it).
__global__ void k_merge_scatter(const tpc_track* __restrict__ tr, MergeBuf mb, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const int32_t c = mb.cell[m];
    if (c < 0) continue;
    const tpc_track T = tr[m];
    MergeKey k;
    k.m = (int32_t)m;
    k.rows = T.first_row | (T.last_row << 16);
    k.z = T.par[1];
    k.t = T.par[3];
    k.q = T.par[4];
    k.vt = T.cov[TPC_CI(3, 3)];
    k.vq = T.cov[TPC_CI(4, 4)];
    k.pad = 0;
    mb.keys[mb.cell_start[c] + atomicSub(&mb.cell_cnt[c], 1) - 1] = k;
  }
}

// 5x5 chi2 d^T S^-1 d by Cholesky; negative if S is not positive definite.
__device__ __forceinline__ float chi2_5(const float d[5], float S[15]) {
  float L[15];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) {
      float a = S[TPC_CI(i, j)];
#pragma unroll
      for (int m = 0; m < j; m++) a -= L[TPC_CI(i, m)] * L[TPC_CI(j, m)];
      if (i == j) {
        if (!(a > 0.0f)) return -1.0f;
        L[TPC_CI(i, i)] = sqrtf(a);
      } else {
        L[TPC_CI(i, j)] = a / L[TPC_CI(j, j)];
      }
    }
  float w[5], c = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    float a = d[i];
#pragma unroll
    for (int m = 0; m < i; m++) a -= L[TPC_CI(i, m)] * w[m];
    w[i] = a / L[TPC_CI(i, i)];
    c += w[i] * w[i];
  }
  return c;
}

// Candidate (best, second) of one lane, merged across the warp: the best is
// the least (chi2, index); the second the least of the rest.
__device__ __forceinline__ void pick_merge(float& bc, int32_t& best, float& sc, float c, int32_t b) {
  if (c < bc || (c == bc && b < best)) {
    sc = fminf(sc, bc);
    bc = c;
    best = b;
  } else {
    sc = fminf(sc, c);
  }
}

// Pairing: per segment A (one warp) its best outer partner and the
// second-best chi2; per segment B its best inner partner (packed atomic
// minimum).  Before the full chi2, a candidate must start on a row A may
// meet, lie in the z range A sweeps over those rows (widened by the window),
// and pass two exact bounds of the chi2: dz/ds_T and q/pT do not change when
// A is turned and carried, and neither do their variances, so chi2 >=
// d_t^2/(V_t,A + V_t,B) and the same for q/pT (taken with a 10% margin).
__global__ void __launch_bounds__(256) k_merge_pairs(const tpc_track* __restrict__ tr, KConst kc, MergeConst mc,
                                                     MergeBuf mb, const Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const float inf = __int_as_float(0x7F800000);
  const int lane = threadIdx.x & 31;
  const float cut = 1.1f * mc.chi2_max;
  for (int64_t a = gtid() >> 5; a < M; a += gstride() >> 5) {
    const tpc_track A = tr[a];
    int32_t best = -1;
    float bc = inf, sc = inf;
    if (merge_eligible(A, mc)) {
      const int side = A.sector / 18, sa = A.sector % 18;
      const int lo = max(A.first_row + 1, A.last_row - mc.overlap);
      const float vtA = A.cov[TPC_CI(3, 3)], vqA = A.cov[TPC_CI(4, 4)];
      for (int k = 0; k < 2 && lo < NROW; k++) {
        const int sb = side * 18 + (sa + (k ? 17 : 1)) % 18;
        const int64_t u = (int64_t)A.request * NSEC + sb;
        TrkState p0;
        seed_state(p0, A.first_row, sX[A.first_row], A.par[0], A.par[1], A.par[2], A.par[3], A.par[4]);
        float C0[15];
#pragma unroll
        for (int i = 0; i < 15; i++) C0[i] = A.cov[i];
        if (!rotate_state<float>(p0, C0, sector_angle(sb) - sector_angle(A.sector))) continue;  // warp-uniform
        // the z A reaches on the rows lo..NROW-1 of B's sector
        float zmin = inf, zmax = -inf;
        for (int r = lo + lane; r < NROW; r += 32) {
          TrkState p = p0;
          uint32_t flags = 0;
          if (prop_state(p, r, sX[r], kc, flags, nullptr)) {
            const float z = p.zref + (p.z + p.zl);
            zmin = fminf(zmin, z);
            zmax = fmaxf(zmax, z);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          zmin = fminf(zmin, __shfl_xor_sync(FULL_MASK, zmin, o));
          zmax = fmaxf(zmax, __shfl_xor_sync(FULL_MASK, zmax, o));
        }
        if (!(zmin <= zmax)) continue;  // no row reachable
        const float margin = 0.01f + 1e-5f * fmaxf(fabsf(zmin), fabsf(zmax));
        const float zlo = zmin - mc.window - margin, zhi = zmax + mc.window + margin;
        int64_t b0 = merge_zbin(zlo, mc), nb = merge_zbin(zhi, mc) - b0 + 1;
        if (nb > mc.nz_mask) {
          b0 = 0;
          nb = mc.nz_mask + 1;
        }
        for (int64_t i = 0; i < nb; i++) {
          const int64_t c = u * (mc.nz_mask + 1) + ((b0 + i) & mc.nz_mask);
          const int32_t e1 = mb.cell_start[c + 1];
          for (int32_t e = mb.cell_start[c] + lane; e < e1; e += 32) {
            const MergeKey K = mb.keys[e];
            const int rin = K.rows & 0xFFFF;
            if (rin < lo || !(K.z >= zlo && K.z <= zhi)) continue;
            const float dt = A.par[3] - K.t, dq = A.par[4] - K.q;
            if (dt * dt > cut * (vtA + K.vt) || dq * dq > cut * (vqA + K.vq)) continue;
            const int32_t b = K.m;
            const tpc_track B = tr[b];
            TrkState p = p0;
            float C[15];
#pragma unroll
            for (int q = 0; q < 15; q++) C[q] = C0[q];
            uint32_t flags = 0;
            Jac J;
            if (!prop_state(p, B.first_row, sX[B.first_row], kc, flags, &J)) continue;
            const float d[5] = {(p.y + p.yl) - B.par[0], (p.zref + (p.z + p.zl)) - B.par[1],
                                (p.s + p.sl) - B.par[2], p.t - B.par[3], p.q - B.par[4]};
            if (!(fabsf(d[1]) <= mc.window)) continue;
            cov_transport<float>(C, J.j02, J.j12, J.j13, J.kap);
#pragma unroll
            for (int q = 0; q < 15; q++) C[q] += B.cov[q];
            const float c2 = chi2_5(d, C);
            if (!(c2 >= 0.0f) || !(c2 <= mc.chi2_max)) continue;
            pick_merge(bc, best, sc, c2, b);
            atomicMin(&mb.best_in[b], ((unsigned long long)__float_as_uint(c2) << 32) | (unsigned long long)a);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oc = __shfl_xor_sync(FULL_MASK, bc, o), os = __shfl_xor_sync(FULL_MASK, sc, o);
        const int32_t ob = __shfl_xor_sync(FULL_MASK, best, o);
        sc = fminf(sc, os);
        pick_merge(bc, best, sc, oc, ob);
      }
    }
    if (lane == 0) {
      mb.best_out[a] = best;
      mb.chi2_out[a] = bc;
      mb.second_out[a] = sc;
    }
  }
}

// Mutual best choices become links; the innermost segment of a chain is
// its head.
__global__ void k_merge_links(MergeBuf mb, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t a = gtid(); a < M; a += gstride()) {
    const int32_t b = mb.best_out[a];
    const bool ok = b >= 0 && (int64_t)(mb.best_in[b] & 0xFFFFFFFFull) == a;
    mb.link[a] = ok ? b : -1;
    if (ok) mb.has_inner[b] = 1;
  }
}

__global__ void k_merge_heads(MergeBuf mb, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t a = gtid(); a < M; a += gstride()) {
    mb.head[a] = mb.link[a] >= 0 && !mb.has_inner[a];
    mb.chain[a] = -1;
  }
}

// Refit of a chain: the outermost segment's refit seed (its follow state
// carried to its outermost row), then every segment's clusters outermost
// first, the frame turned between segments; the FP64 zone as in the refit.
__global__ void __launch_bounds__(128) k_merge_refit(const tpc_track* __restrict__ tr,
                                                     const tpc_cluster* __restrict__ in, RefitIn rin,
                                                     const int32_t* __restrict__ track_clusters, KConst kc,
                                                     MergeBuf mb, const Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  for (int64_t h = gtid(); h < M; h += gstride()) {
    if (!mb.head[h]) continue;
    const int32_t k = mb.chain_of_head[h];
    int32_t seg[MERGE_MAX_SEG];
    int ns = 0;
    for (int32_t g = (int32_t)h; g >= 0 && ns < MERGE_MAX_SEG; g = mb.link[g]) seg[ns++] = g;
    int32_t ncl = 0;
    for (int i = 0; i < ns; i++) {
      mb.chain[seg[i]] = k;
      ncl += tr[seg[i]].n_clusters;
    }
    // seed: the outermost segment's follow state carried to its last row
    const tpc_track O = tr[seg[ns - 1]];
    const int t = rin.track_tl[seg[ns - 1]];
    TrkState p;
    const int fr = rin.f_row[t];
    seed_state(p, fr, sX[fr], rin.f_par[t * 5 + 0], rin.f_zref[t], rin.f_par[t * 5 + 2], rin.f_par[t * 5 + 3],
               rin.f_par[t * 5 + 4]);
    p.z = rin.f_par[t * 5 + 1];
    uint32_t flags = 0;
    bool ok = true;
    const int step = O.last_row >= p.row ? 1 : -1;
    for (int r = p.row + step; ok && (step > 0 ? r <= O.last_row : r >= O.last_row); r += step)
      ok = prop_state(p, r, sX[r], kc, flags, nullptr);
    double D[15];
    float C[15];
    cov_seed<double>(D, kc);
    cov_seed<float>(C, kc);
    Chi2Acc chi2;
    chi2.reset();
    int nupd = 0, zend = kc.fp64_updates;
    int row = O.last_row;
    for (int gi = ns - 1; ok && gi >= 0; gi--) {
      const tpc_track S = tr[seg[gi]];
      if (gi < ns - 1) {
        const float beta = sector_angle(S.sector) - sector_angle(tr[seg[gi + 1]].sector);
        ok = nupd < zend ? rotate_state<double>(p, D, beta) : rotate_state<float>(p, C, beta);
        row = NROW;  // the next step goes to this segment's first cluster row
      }
      const int64_t off = S.cluster_offset, n = S.n_clusters;
      for (int64_t i = n - 1; ok && i >= 0; i--) {
        const tpc_cluster c = in[track_clusters[off + i]];
        if (row == NROW) {
          ok = propagate_any(p, nupd < zend, D, C, c.row, sX[c.row], kc, flags);
          row = c.row;
        }
        while (ok && row > c.row) {
          row--;
          ok = propagate_any(p, nupd < zend, D, C, row, sX[row], kc, flags);
        }
        if (!ok) break;
        chi2.add(zone_update(p, nupd < zend, D, C, c.y, c.z, kc, nupd, zend, 2 * kc.fp64_updates));
      }
    }
    if (ok && nupd < zend) {
#pragma unroll
      for (int q = 0; q < 15; q++) C[q] = narrow(D[q]);
    }
    const tpc_track I = tr[seg[0]];
    tpc_track out;
    out.x = p.x;
    out.par[0] = p.y + p.yl;
    out.par[1] = p.zref + (p.z + p.zl);
    out.par[2] = p.s + p.sl;
    out.par[3] = p.t;
    out.par[4] = p.q;
#pragma unroll
    for (int q = 0; q < 15; q++) out.cov[q] = C[q];
    out.reserved = ns;
    out.chi2 = chi2.value();
    out.ndf = 2 * ncl - 5;
    out.n_clusters = ncl;
    out.sector = I.sector;
    out.request = I.request;
    out.first_row = row;
    out.last_row = O.last_row;
    out.cluster_offset = (int32_t)h;  // the chain's innermost segment
    out.flags = ok ? 0 : TF_REFIT_FAIL;
    mb.merged[k] = out;
  }
}

}  // namespace tpc
