// Cluster rejection (the paper's compression section): before compression
// the clusters of tracks that physics does not use are dropped -- momentum
// below p_min, |dz/ds_T| above tgl_max, and the further legs of loopers.  A
// looper is a track whose circle stays inside the outermost row radius;
// every leg of a helix from the collision passes the beam axis again after
// each full turn with z moved by 2 pi R t, so a looper whose z at its
// closest approach to the axis lies more than dz_leg from the collision
// (z_ref for an event, the nearest vertex in time for continuous read-out)
// is a further leg.  One thread per track; a rejected track clears the
// keep flags of its clusters.
#pragma once
#include "vertex.cuh"

namespace tpc {

struct RejConst {
  float p_min, tgl_max, dz_leg, z_ref;
  float K;              // 0.299792458e-3 * Bz
  float x_out;          // radius of the outermost row
  float vdrift;         // vertex mode: cm/us
  int32_t use_vertices; // 1: the nearest vertex of the request
};

enum : uint8_t { RJ_LOW_P = 1, RJ_INCLINED = 2, RJ_LOOPER_LEG = 4 };

struct RejBuf {
  uint8_t* cls;               // [M] class bits per track
  uint8_t* keep;              // [N] 1: the cluster stays
  unsigned long long* count;  // [4] rejected clusters: any, low p, inclined, further leg
};

// Farthest distance of the track's circle from the beam axis, |c| + 1/|k|
// (infinite for a straight track).
__device__ __forceinline__ float circle_reach(float x, float y, float s, float q, float K) {
  const float k = -K * q;
  if (k == 0.0f) return __int_as_float(0x7F800000);
  const float c = sqrtf(fmaxf(1.0f - s * s, 0.0f));
  const float ik = 1.0f / k;
  return hypotf(x - s * ik, y + c * ik) + fabsf(ik);
}

// Time distance to the nearest of n ascending vertex times.
__device__ __forceinline__ double nearest_vertex_dt(double te, const double* __restrict__ tv, int32_t n) {
  int32_t lo = 0, hi = n;  // first vertex with tv >= te
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (tv[mid] < te) lo = mid + 1;
    else hi = mid;
  }
  double d = INFINITY;
  if (lo < n) d = tv[lo] - te;
  if (lo > 0) d = fmin(d, te - tv[lo - 1]);
  return d;
}

// vt / vn / vtx_t: the vertex mode's vertex times, their count and each
// track's time estimate (unused otherwise).
__global__ void k_reject(const tpc_track* __restrict__ tr, const int32_t* __restrict__ track_clusters, RejConst rc,
                         const double* __restrict__ vt, const int32_t* __restrict__ vn,
                         const float* __restrict__ vtx_t, RejBuf rb, const Counts* cn) {
  if (fatal(cn)) return;
  const int32_t M = cn->n_tracks;
  const int32_t nv = rc.use_vertices ? *vn : 0;
  for (int64_t m = gtid(); m < M; m += gstride()) {
    const tpc_track T = tr[m];
    const float t = T.par[3], q = T.par[4];
    uint8_t bits = 0;
    if (sqrtf(1.0f + t * t) / fabsf(q) < rc.p_min) bits |= RJ_LOW_P;
    if (fabsf(t) > rc.tgl_max) bits |= RJ_INCLINED;
    if (circle_reach(T.x, T.par[0], T.par[2], q, rc.K) < rc.x_out) {
      float dz;
      if (rc.use_vertices) {
        const double te = vtx_t[m];
        dz = (float)(rc.vdrift * nearest_vertex_dt(te, vt, nv));
      } else {
        float path, dist;
        vtx_dca(T.x, T.par[0], T.par[2], q, rc.K, path, dist);
        dz = fabsf((T.par[1] + t * path) - rc.z_ref);
      }
      if (dz > rc.dz_leg) bits |= RJ_LOOPER_LEG;
    }
    rb.cls[m] = bits;
    if (bits) {
      const int64_t off = T.cluster_offset, n = T.n_clusters;
      for (int64_t i = 0; i < n; i++) rb.keep[track_clusters[off + i]] = 0;
      atomicAdd(&rb.count[0], (unsigned long long)n);
      if (bits & RJ_LOW_P) atomicAdd(&rb.count[1], (unsigned long long)n);
      if (bits & RJ_INCLINED) atomicAdd(&rb.count[2], (unsigned long long)n);
      if (bits & RJ_LOOPER_LEG) atomicAdd(&rb.count[3], (unsigned long long)n);
    }
  }
}

}  // namespace tpc
