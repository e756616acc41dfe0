// Track-model compression (the paper's compression section): each selected
// track is refitted over its own clusters, outermost first; at every cluster
// the residual between the fixed-point cluster and the rounded extrapolated
// track position is stored, and the fit is updated with the fixed-point
// value.  Decompression runs the same fit from the same header and adds
// the residuals back, so it restores every fixed-point cluster exactly.
// Encoding and decoding are one instruction stream (a runtime flag selects
// where the cluster comes from), so the two fits cannot round differently.
// The paper's distortion transform is the identity here.
#pragma once
#include "kalman.cuh"

namespace tpc {

// == tpc_codec_header (include/tpcca.h)
struct CodecHeader {
  float par[5];       // y, z (absolute), sin phi, dz/ds_T, q/pT at row_out
  int32_t row_out;    // row of the outermost cluster
  int32_t n_clusters;
  int32_t ok;         // 0: the fit stopped at the |sin phi| limit; clusters kept in fixed point
};
static_assert(sizeof(CodecHeader) == 32, "tpc_codec_header layout");

struct CodecIo {
  CodecHeader* head;    // [tracks]
  const int64_t* off;   // [tracks + 1] first cluster of each track (decode)
  uint8_t* rows;        // [clusters] outermost first
  int32_t* qy;          // fixed-point clusters
  int32_t* qz;
  int32_t* ry;          // residuals
  int32_t* rz;
};

// Fixed-point coordinate of a binary32 value: rint(v * (1/unit)).
__device__ __forceinline__ int32_t codec_q(float v, float inv) { return (int32_t)rintf(__fmul_rn(v, inv)); }

// The fit of one track over its n clusters (outermost first); decode: the
// clusters from the residuals, else the residuals from the clusters.
// Returns false when a propagation reaches the |sin phi| limit.
__device__ __noinline__ bool codec_track(const KConst& kc, const float* sX, const CodecHeader& h, int64_t n,
                                         const uint8_t* rows, int32_t* qy, int32_t* qz, int32_t* ry, int32_t* rz,
                                         bool decode, float unit, float inv) {
  TrkState p;
  seed_state(p, h.row_out, sX[h.row_out], h.par[0], h.par[1], h.par[2], h.par[3], h.par[4]);
  double D[15];
  float C[15];
  cov_seed<double>(D, kc);
  cov_seed<float>(C, kc);
  uint32_t flags = 0;
  int nupd = 0, zend = kc.fp64_updates;
  int row = h.row_out;
  for (int64_t i = 0; i < n; i++) {
    while (row > rows[i]) {
      row--;
      if (!propagate_any(p, nupd < zend, D, C, row, sX[row], kc, flags)) return false;
    }
    const int32_t py = (int32_t)rintf(__fmul_rn(p.y + p.yl, inv));
    const int32_t pz = (int32_t)rintf(__fmul_rn(p.zref + (p.z + p.zl), inv));
    int32_t a, b;
    if (decode) {
      a = py + ry[i];
      b = pz + rz[i];
      qy[i] = a;
      qz[i] = b;
    } else {
      a = qy[i];
      b = qz[i];
      ry[i] = a - py;
      rz[i] = b - pz;
    }
    zone_update(p, nupd < zend, D, C, __fmul_rn((float)a, unit), __fmul_rn((float)b, unit), kc, nupd, zend,
                2 * kc.fp64_updates);
  }
  return true;
}

// Encoding: per selected track, the header (the follow state carried to the
// outermost owned row, as the refit starts), the owned clusters outermost
// first in fixed point, and the residuals.
__global__ void __launch_bounds__(128) k_codec_encode(const tpc_track* __restrict__ tracks,
                                                      const tpc_cluster* __restrict__ in, RefitIn rin,
                                                      const int32_t* __restrict__ track_clusters, KConst kc,
                                                      CodecIo io, float unit, const Counts* cn) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const float inv = __frcp_rn(unit);
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const tpc_track tr = tracks[m];
    const int t = rin.track_tl[m];
    const int64_t off = tr.cluster_offset, n = tr.n_clusters;
    CodecHeader h;
    h.row_out = tr.last_row;
    h.n_clusters = (int32_t)n;
    // carry the follow state to row_out (state only)
    TrkState p;
    const int fr = rin.f_row[t];
    seed_state(p, fr, sX[fr], rin.f_par[t * 5 + 0], rin.f_zref[t], rin.f_par[t * 5 + 2], rin.f_par[t * 5 + 3],
               rin.f_par[t * 5 + 4]);
    p.z = rin.f_par[t * 5 + 1];
    uint32_t flags = 0;
    bool ok = !(tr.flags & TF_REFIT_FAIL);
    const int step = h.row_out >= p.row ? 1 : -1;
    for (int r = p.row + step; ok && (step > 0 ? r <= h.row_out : r >= h.row_out); r += step)
      ok = prop_state(p, r, sX[r], kc, flags, nullptr);
    h.par[0] = p.y + p.yl;
    h.par[1] = p.zref + (p.z + p.zl);
    h.par[2] = p.s + p.sl;
    h.par[3] = p.t;
    h.par[4] = p.q;
    for (int64_t i = 0; i < n; i++) {
      const tpc_cluster c = in[track_clusters[off + n - 1 - i]];
      io.rows[off + i] = (uint8_t)c.row;
      io.qy[off + i] = codec_q(c.y, inv);
      io.qz[off + i] = codec_q(c.z, inv);
      io.ry[off + i] = 0;
      io.rz[off + i] = 0;
    }
    if (ok)
      ok = codec_track(kc, sX, h, n, io.rows + off, io.qy + off, io.qz + off, io.ry + off, io.rz + off, false, unit,
                       inv);
    if (!ok) {  // the fit does not run: the residual streams carry the fixed-point clusters
      for (int64_t i = 0; i < n; i++) {
        io.ry[off + i] = io.qy[off + i];
        io.rz[off + i] = io.qz[off + i];
      }
    }
    h.ok = ok;
    io.head[m] = h;
  }
}

// Decoding of n_tracks tracks given their headers, offsets, rows and
// residuals.
__global__ void __launch_bounds__(128) k_codec_decode(KConst kc, CodecIo io, int64_t n_tracks, float unit,
                                                      int32_t* __restrict__ bad) {
  __shared__ float sX[NROW + 1];
  for (int i = threadIdx.x; i < NROW; i += blockDim.x) sX[i] = g_row_x[i];
  __syncthreads();
  const float inv = __frcp_rn(unit);
  for (int64_t m = gtid(); m < n_tracks; m += gstride()) {
    const CodecHeader h = io.head[m];
    const int64_t off = io.off[m], n = io.off[m + 1] - off;
    if (!h.ok) {  // stored in fixed point
      for (int64_t i = 0; i < n; i++) {
        io.qy[off + i] = io.ry[off + i];
        io.qz[off + i] = io.rz[off + i];
      }
      continue;
    }
    if (h.row_out < 0 || h.row_out >= NROW) {
      atomicAdd(bad, 1);
      continue;
    }
    bool valid = true;
    for (int64_t i = 0; i < n; i++) valid = valid && io.rows[off + i] <= h.row_out;
    if (!valid || !codec_track(kc, sX, h, n, io.rows + off, io.qy + off, io.qz + off, io.ry + off, io.rz + off, true,
                               unit, inv))
      atomicAdd(bad, 1);
  }
}

}  // namespace tpc
