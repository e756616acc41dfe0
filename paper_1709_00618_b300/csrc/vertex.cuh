// Vertex finding in the drift-time coordinate (Sec. 5, continuous read-out):
// the refitted tracks of a timeframe, whose z is the drift coordinate z_t,
// are extrapolated to their closest approach to the beam axis; z_t there
// gives the collision time of a track from z = 0; tracks sorted in time are
// cut into vertices at gaps; the vertex time then converts z_t to space.
//
// The sort is replaced by binning: with bins of half the gap, two tracks
// in one bin are never cut apart, so a cut can only fall between
// consecutive non-empty bins, where it is decided on the bins' extreme
// times exactly as between neighbours of the sorted list.
#pragma once
#include "common.cuh"

namespace tpc {

struct VtxConst {
  float K;         // 0.299792458e-3 * Bz
  float vdrift;    // cm/us
  float zmax;      // cm
  float dca_max;   // cm
  float ext_max;   // cm
  float gap;       // us
  float inv_w;     // 1 / bin width (bin width = gap / 2)
  int32_t min_tracks, min_clusters;
  int32_t bins_cap;
  float min_pt;    // GeV/c; 0: no cut
};

struct VtxBuf {
  float* t;            // [M] time estimate
  uint8_t* use;        // [M]
  int32_t* vertex;     // [M] final vertex index or -1
  float* z;            // [M] spatial z at the innermost row (NaN without a vertex)
  float* tgl;          // [M] spatial dz/ds_T
  int32_t* b_cnt;      // [bins] tracks per bin
  uint32_t* b_min;     // [bins] ordered-int min / max time of the bin
  uint32_t* b_max;
  int32_t* b_vid;      // [bins] provisional vertex of a non-empty bin
  int32_t* v_cnt;      // [bins] tracks per provisional vertex
  unsigned long long* v_sum;  // [bins] sum of times in 1e-6 us
  int32_t* v_keep;     // [bins + 1] 1 if the vertex has min_tracks tracks
  int32_t* v_idx;      // [bins + 1] its final index (exclusive scan)
  uint32_t* range;     // [2] ordered-int min / max time of the used tracks
  int32_t* n;          // [4] bins, provisional vertices, final vertices, status
};

constexpr unsigned long long VTX_FIX = 1000000ull;  // time unit of the sums: 1e-6 us
constexpr double VTX_OFFSET_US = 1.0e4;             // added before the fixed-point conversion (t > -1e4 us)

// Point of closest approach of the helix to the beam axis (the transverse
// plane of the sector's local frame): path length from the state's x and
// the distance there.  On the circle around c = (x - s/k, y + cos/k) the
// direction at the closest point is perpendicular to c; the path is the
// turn to it over the curvature.  The distance |c| - 1/|k| is formed as
// (|c|^2 - 1/k^2) / (|c| + 1/|k|) with the 1/k^2 terms cancelled exactly.
__device__ __forceinline__ void vtx_dca(float x, float y, float s, float q, float K, float& path, float& dist) {
  const float c = sqrtf(fmaxf(1.0f - s * s, 0.0f));
  const float k = -K * q;
  if (k == 0.0f) {
    path = -(x * c + y * s);
    dist = fabsf(x * s - y * c);
    return;
  }
  const float ik = 1.0f / k;
  const float cx = x - s * ik, cy = y + c * ik;
  const float sg = k > 0.0f ? 1.0f : -1.0f;
  const float psi = atan2f(-sg * cx, sg * cy);
  const float phi = atan2f(s, c);
  float d = psi - phi;
  const float pi = 3.14159265358979f;
  if (d > pi) d -= 2.0f * pi;
  if (d <= -pi) d += 2.0f * pi;
  path = d * ik;
  const float num = x * x + y * y + 2.0f * (y * c - x * s) * ik;
  dist = fabsf(num / (sqrtf(cx * cx + cy * cy) + fabsf(ik)));
}

// Step 1: time estimate and participation of every track; the time range
// of the participating ones.
__global__ void k_vtx_time(const tpc_track* __restrict__ tr, VtxConst vc, VtxBuf vb, const Counts* cn) {
  const int32_t M = cn->n_tracks;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const tpc_track t = tr[m];
    float path, dist;
    vtx_dca(t.x, t.par[0], t.par[2], t.par[4], vc.K, path, dist);
    const float dzt = t.par[3] * path;
    const float te = ((t.par[1] - vc.zmax) + dzt) / vc.vdrift;
    const bool use = dist <= vc.dca_max && fabsf(dzt) <= vc.ext_max && t.n_clusters >= vc.min_clusters &&
                     isfinite(te) && !(fabsf(t.par[4]) * vc.min_pt > 1.0f);
    vb.t[m] = te;
    vb.use[m] = use;
    if (use) {
      atomicMin(&vb.range[0], f2ord(te));
      atomicMax(&vb.range[1], f2ord(te));
    }
  }
}

__device__ __forceinline__ int32_t vtx_bins(const VtxBuf& vb, const VtxConst& vc, float& t0) {
  if (vb.range[0] > vb.range[1]) return 0;  // no participating track
  t0 = ord2f(vb.range[0]);
  const float t1 = ord2f(vb.range[1]);
  return (int32_t)floorf((t1 - t0) * vc.inv_w) + 1;
}

// Number of bins; clears them (and the vertex sums) up to that number.
__global__ void k_vtx_clear(VtxConst vc, VtxBuf vb) {
  float t0 = 0.0f;
  const int32_t nb = vtx_bins(vb, vc, t0);
  if (gtid() == 0) {
    vb.n[0] = nb;
    if (nb > vc.bins_cap) vb.n[3] = 1;  // the time range needs more bins than reserved
  }
  const int32_t lim = min(nb, vc.bins_cap);
  for (int64_t i = gtid(); i < lim; i += gstride()) {
    vb.b_cnt[i] = 0;
    vb.b_min[i] = 0xFFFFFFFFu;
    vb.b_max[i] = 0u;
    vb.v_cnt[i] = 0;
    vb.v_sum[i] = 0ull;
  }
}

__device__ __forceinline__ int32_t vtx_bin_of(float te, float t0, const VtxConst& vc, int32_t nb) {
  return min(max((int32_t)floorf((te - t0) * vc.inv_w), 0), nb - 1);
}

__global__ void k_vtx_bin(VtxConst vc, VtxBuf vb, const Counts* cn) {
  const int32_t nb = vb.n[0];
  if (nb <= 0 || nb > vc.bins_cap) return;
  const float t0 = ord2f(vb.range[0]);
  const int32_t M = cn->n_tracks;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    if (!vb.use[m]) continue;
    const float te = vb.t[m];
    const int32_t b = vtx_bin_of(te, t0, vc, nb);
    atomicAdd(&vb.b_cnt[b], 1);
    atomicMin(&vb.b_min[b], f2ord(te));
    atomicMax(&vb.b_max[b], f2ord(te));
  }
}

// Runs of non-empty bins -> provisional vertices (one block): each thread
// summarises a contiguous stretch of bins, thread 0 carries the last time
// and the vertex count across the stretches, then every thread numbers its
// bins.  A non-empty bin opens a vertex when its earliest time is more than
// the gap after the latest time of the previous non-empty bin.
constexpr int VTX_RUN_THREADS = 1024;

__global__ void __launch_bounds__(VTX_RUN_THREADS) k_vtx_runs(VtxConst vc, VtxBuf vb) {
  __shared__ float s_first[VTX_RUN_THREADS], s_last[VTX_RUN_THREADS];
  __shared__ int32_t s_has[VTX_RUN_THREADS], s_inner[VTX_RUN_THREADS], s_base[VTX_RUN_THREADS];
  const int32_t nb = vb.n[0];
  if (nb <= 0 || nb > vc.bins_cap) {
    if (threadIdx.x == 0) vb.n[1] = 0;
    return;
  }
  const int32_t per = (nb + VTX_RUN_THREADS - 1) / VTX_RUN_THREADS;
  const int32_t b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  bool has = false;
  float first = 0.0f, last = 0.0f;
  int32_t inner = 0;
  for (int32_t b = b0; b < b1; b++) {
    if (vb.b_cnt[b] == 0) continue;
    const float lo = ord2f(vb.b_min[b]), hi = ord2f(vb.b_max[b]);
    if (!has) {
      has = true;
      first = lo;
    } else if (lo - last > vc.gap) {
      inner++;
    }
    last = hi;
  }
  s_has[threadIdx.x] = has;
  s_first[threadIdx.x] = first;
  s_last[threadIdx.x] = last;
  s_inner[threadIdx.x] = inner;
  __syncthreads();
  if (threadIdx.x == 0) {
    bool any = false;
    float carry = 0.0f;
    int32_t count = 0;
    for (int k = 0; k < VTX_RUN_THREADS; k++) {
      if (!s_has[k]) continue;
      if (!any || s_first[k] - carry > vc.gap) count++;
      s_base[k] = count - 1;  // vertex of the stretch's first non-empty bin
      count += s_inner[k];
      carry = s_last[k];
      any = true;
    }
    vb.n[1] = count;
  }
  __syncthreads();
  if (!has) return;
  int32_t cur = s_base[threadIdx.x];
  bool seen = false;
  for (int32_t b = b0; b < b1; b++) {
    if (vb.b_cnt[b] == 0) continue;
    const float lo = ord2f(vb.b_min[b]);
    if (seen && lo - last > vc.gap) cur++;
    vb.b_vid[b] = cur;
    last = ord2f(vb.b_max[b]);
    seen = true;
  }
}

// Track counts and time sums per provisional vertex (fixed point, so the
// sums do not depend on the order of the additions).
__global__ void k_vtx_accum(VtxConst vc, VtxBuf vb, const Counts* cn) {
  const int32_t nb = vb.n[0];
  if (nb <= 0 || nb > vc.bins_cap) return;
  const float t0 = ord2f(vb.range[0]);
  const int32_t M = cn->n_tracks;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    if (!vb.use[m]) continue;
    const float te = vb.t[m];
    const int32_t v = vb.b_vid[vtx_bin_of(te, t0, vc, nb)];
    atomicAdd(&vb.v_cnt[v], 1);
    atomicAdd(&vb.v_sum[v], (unsigned long long)llrint(fmax((double)te + VTX_OFFSET_US, 0.0) * (double)VTX_FIX));
  }
}

__global__ void k_vtx_keep(VtxConst vc, VtxBuf vb) {
  const int32_t nv = vb.n[1];
  for (int64_t v = gtid(); v < nv; v += gstride()) vb.v_keep[v] = vb.v_cnt[v] >= vc.min_tracks;
}

__device__ __forceinline__ double vtx_time(const VtxBuf& vb, int32_t v) {
  return (double)vb.v_sum[v] / (double)VTX_FIX / (double)vb.v_cnt[v] - VTX_OFFSET_US;
}

// Final vertex of every track and its spatial z and dz/ds_T.
__global__ void k_vtx_tracks(const tpc_track* __restrict__ tr, VtxConst vc, VtxBuf vb, const Counts* cn) {
  const int32_t nb = vb.n[0], nv = vb.n[1];
  const bool ok = nb > 0 && nb <= vc.bins_cap;
  if (gtid() == 0) vb.n[2] = ok && nv > 0 ? vb.v_idx[nv] : 0;
  const float t0 = ok ? ord2f(vb.range[0]) : 0.0f;
  const int32_t M = cn->n_tracks;
  const float nan = __int_as_float(0x7FC00000);
  for (int64_t m = gtid(); m < M; m += gstride()) {
    int32_t fin = -1;
    if (ok && vb.use[m]) {
      const int32_t v = vb.b_vid[vtx_bin_of(vb.t[m], t0, vc, nb)];
      if (vb.v_keep[v]) fin = vb.v_idx[v];
      if (fin >= 0) {
        const tpc_track t = tr[m];
        const float side = (t.sector % NSEC) < NSEC / 2 ? 1.0f : -1.0f;
        const double tv = vtx_time(vb, v);
        vb.z[m] = side * (float)((double)vc.zmax - ((double)t.par[1] - (double)vc.vdrift * tv));
        vb.tgl[m] = -side * t.par[3];
      }
    }
    vb.vertex[m] = fin;
    if (fin < 0) {
      vb.z[m] = nan;
      vb.tgl[m] = nan;
    }
  }
}

// Compact vertex records {time, tracks} in time order.
__global__ void k_vtx_records(VtxConst vc, VtxBuf vb, double* __restrict__ t_out, int32_t* __restrict__ n_out) {
  const int32_t nb = vb.n[0], nv = vb.n[1];
  if (nb <= 0 || nb > vc.bins_cap) return;
  for (int64_t v = gtid(); v < nv; v += gstride()) {
    if (!vb.v_keep[v]) continue;
    const int32_t k = vb.v_idx[v];
    t_out[k] = vtx_time(vb, (int32_t)v);
    n_out[k] = vb.v_cnt[v];
  }
}

}  // namespace tpc
