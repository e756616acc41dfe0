// a2: per-row (y, z) grid of every (request, sector, row) and the stable sort
// of the clusters by (row-sector, bin, load index).
//
// The bin arithmetic decides integers (bin indices), so it is written with
// explicitly rounded binary32 intrinsics (__fadd_rn & co. are never fused
// into FMAs): the result is bit-identical to any IEEE binary32 evaluation of
// the same expression sequence.
#pragma once
#include "common.cuh"
#include "order.cuh"

namespace tpc {

// Largest request q with off[q] <= i (empty requests are skipped naturally).
__device__ __forceinline__ int find_request(const int64_t* __restrict__ off, int n_req, int64_t i) {
  int lo = 0, hi = n_req - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_rs_init(int32_t* __restrict__ cnt, uint32_t* __restrict__ zmin, uint32_t* __restrict__ zmax,
                          int32_t* __restrict__ obins, Counts* cn) {
  // Per-run scalars: a run on the same loaded batch (a second tpc_find_tracks,
  // a graph replay, the autotuner's trials) starts from the state a load
  // leaves.  Work counters of every Kalman kernel and chunk, status, tallies.
  if (gtid() < PH_FETCH * MAX_CHUNKS) cn->work_next[gtid()] = 0;
  if (gtid() < 3 * MAX_CHUNKS) cn->zone_pend[gtid()] = 0;
  if (gtid() < PH_COUNT * 5) (&cn->phase_work[0][0])[gtid()] = 0ull;
  if (gtid() == 0) {
    cn->status = 0u;
    cn->n_prop = cn->n_upd32 = cn->n_upd64 = cn->n_cand = cn->n_prop64 = 0ull;
    cn->trace_n = 0;
  }
  for (int64_t i = gtid(); i < ORD_WORDS; i += gstride()) obins[i] = 0;  // their work-order histograms
  int32_t nrs = cn->n_rs;
  for (int64_t i = gtid(); i < nrs; i += gstride()) {
    cnt[i] = 0;
    zmin[i] = 0xFFFFFFFFu;
    zmax[i] = 0u;
  }
}

// Count per row-sector and exact z range; validates every cluster.
__global__ void k_grid_count(const tpc_cluster* __restrict__ in, const int64_t* __restrict__ req_off,
                             Counts* cn, int32_t* __restrict__ rs_in, int32_t* __restrict__ cnt,
                             uint32_t* __restrict__ zmin, uint32_t* __restrict__ zmax) {
  const int64_t n = cn->n;
  const int n_req = cn->n_req;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    int4 raw = __ldg(reinterpret_cast<const int4*>(in) + i);
    float y = __int_as_float(raw.x), z = __int_as_float(raw.y);
    uint32_t row = (uint32_t)raw.z & 0xFFFFu, sec = (uint32_t)raw.z >> 16;
    if (row >= NROW || sec >= NSEC || !isfinite(y) || !isfinite(z)) {
      atomicOr(&cn->status, ST_EINVAL);
      rs_in[i] = -1;
      continue;
    }
    int q = find_request(req_off, n_req, i);
    int rs = (q * NSEC + (int)sec) * NROW + (int)row;
    rs_in[i] = rs;
    atomicAdd(&cnt[rs], 1);
    // the range only widens, so a read (through the non-coherent cache:
    // possibly an older, wider value, which costs only an atomic) already
    // inside it means the cluster cannot move that bound
    const uint32_t zo = f2ord(z);
    if (zo < __ldg(zmin + rs)) atomicMin(&zmin[rs], zo);
    if (zo > __ldg(zmax + rs)) atomicMax(&zmax[rs], zo);
  }
}

// Bin parameters of one row-sector (same operation sequence as the reading).
__global__ void k_grid_params(const int32_t* __restrict__ cnt, const uint32_t* __restrict__ zmin,
                              const uint32_t* __restrict__ zmax, RsParams* __restrict__ par,
                              int32_t* __restrict__ nbins, const Counts* cn) {
  if (fatal(cn)) return;
  int32_t nrs = cn->n_rs;
  for (int64_t rs = gtid(); rs < nrs; rs += gstride()) {
    int row = (int)(rs % NROW);
    int n = cnt[rs];
    float zl = n ? ord2f(zmin[rs]) : 0.0f, zh = n ? ord2f(zmax[rs]) : 0.0f;
    float yh = g_row_yhi[row], yl = -yh;
    float wy = __fsub_rn(yh, yl);
    float dz = __fsub_rn(zh, zl);
    float area = __fmul_rn(wy, fmaxf(dz, 1.0f));
    float s = __fsqrt_rn(__fdiv_rn(__fmul_rn(area, 2.0f), __int2float_rn(n > 1 ? n : 1)));
    s = fminf(fmaxf(s, 1.0f), 64.0f);
    int ny = __float2int_rz(__fdiv_rn(wy, s)) + 1;
    int nz = __float2int_rz(__fdiv_rn(dz, s)) + 1;
    if (ny > 256) ny = 256;
    if (nz > 4096) nz = 4096;
    RsParams p;
    p.z_lo = zl;
    p.z_hi = zh;
    p.inv_y = __fdiv_rn(__int2float_rn(ny), wy);
    p.inv_z = __fdiv_rn(__int2float_rn(nz), fmaxf(dz, 1e-3f));
    p.n_y = ny;
    p.n_z = nz;
    p.bin_base = 0;  // filled after the scan
    p.count = n;
    par[rs] = p;
    nbins[rs] = ny * nz;
  }
}

// The sort runs in two levels.  Level one moves every record from load
// order into its bucket: buckets are ranges of whole row-sectors in sorted
// order, a row-sector going to bucket (its first sorted position) >>
// bucket_shift, so a bucket holds about 2^bucket_shift clusters (at most
// GRID_BUCKETS buckets).  Level two counts bins and scatters inside one
// bucket at a time, so its random accesses stay in L2.
constexpr int GRID_BUCKETS = 512;
struct GridBuckets {
  int32_t base[GRID_BUCKETS];  // first sorted position of each bucket
  int32_t fill[GRID_BUCKETS];  // records placed so far
};

// Bucket exponent for n clusters: 2^18 clusters (4 MB of records), or more
// so that at most GRID_BUCKETS buckets are needed.
__host__ __device__ inline int grid_bucket_shift(int64_t n) {
  int sh = 18;
  while ((n >> sh) >= GRID_BUCKETS) sh++;
  return sh;
}

// After the scans: store bin_base into the params, check the capacity, set
// the bucket bases and clear the bin counts.
__global__ void k_grid_finish_params(RsParams* __restrict__ par, const int32_t* __restrict__ bin_base,
                                     const int32_t* __restrict__ rs_start, Counts* cn, int64_t bins_cap,
                                     int32_t* __restrict__ bin_cnt, GridBuckets* __restrict__ bk) {
  if (fatal(cn)) return;
  int32_t nrs = cn->n_rs;
  int32_t nb = bin_base[nrs];
  if (gtid() == 0) cn->n_bins = nb;
  if ((int64_t)nb > bins_cap) {
    if (gtid() == 0) atomicOr(&cn->status, ST_EOVERFLOW);
    return;
  }
  const int sh = grid_bucket_shift(cn->n);
  for (int64_t q = gtid(); q < GRID_BUCKETS; q += gstride()) bk->fill[q] = 0;
  for (int64_t rs = gtid(); rs < nrs; rs += gstride()) {
    par[rs].bin_base = bin_base[rs];
    const int b = rs_start[rs] >> sh;
    if (rs == 0 || (rs_start[rs - 1] >> sh) != b) bk->base[b] = rs_start[rs];
  }
  for (int64_t b = gtid(); b <= nb; b += gstride()) bin_cnt[b] = 0;
}

__device__ __forceinline__ int bin_coord(float v, float lo, float inv, int nb) {
  float f = floorf(__fmul_rn(__fsub_rn(v, lo), inv));
  if (!(f >= 0.0f)) return 0;
  if (f > __int2float_rn(nb - 1)) return nb - 1;
  return __float2int_rz(f);
}

// Level one: record {load index, y, z, row-sector} of every cluster into
// its bucket.  A block takes GRID_TILE clusters at a time, counts them per
// bucket in shared memory and claims each bucket's range with one atomic, so
// a bucket receives contiguous runs from each tile.
constexpr int GRID_TILE_PER_THREAD = 4;
__global__ void k_grid_bucket(const tpc_cluster* __restrict__ in, const int32_t* __restrict__ rs_in,
                              const int32_t* __restrict__ rs_start, GridBuckets* __restrict__ bk,
                              int4* __restrict__ rec_b, const Counts* cn) {
  if (fatal(cn)) return;
  __shared__ int32_t s_cnt[GRID_BUCKETS], s_base[GRID_BUCKETS];
  const int64_t n = cn->n;
  const int sh = grid_bucket_shift(n);
  const int64_t tile = (int64_t)blockDim.x * GRID_TILE_PER_THREAD;
  for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < n; t0 += (int64_t)gridDim.x * tile) {  // block-uniform
    for (int b = threadIdx.x; b < GRID_BUCKETS; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    int b[GRID_TILE_PER_THREAD], r[GRID_TILE_PER_THREAD];
    int rs[GRID_TILE_PER_THREAD];
#pragma unroll
    for (int k = 0; k < GRID_TILE_PER_THREAD; k++) {
      const int64_t i = t0 + (int64_t)k * blockDim.x + threadIdx.x;
      b[k] = -1;
      rs[k] = -1;
      if (i < n && (rs[k] = rs_in[i]) >= 0) {
        b[k] = rs_start[rs[k]] >> sh;
        r[k] = atomicAdd(&s_cnt[b[k]], 1);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < GRID_BUCKETS; q += blockDim.x) {
      const int c = s_cnt[q];
      s_base[q] = c ? bk->base[q] + atomicAdd(&bk->fill[q], c) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GRID_TILE_PER_THREAD; k++) {
      if (b[k] < 0) continue;
      const int64_t i = t0 + (int64_t)k * blockDim.x + threadIdx.x;
      const int4 raw = __ldg(reinterpret_cast<const int4*>(in) + i);
      rec_b[s_base[b[k]] + r[k]] = make_int4((int32_t)i, raw.x, raw.y, rs[k]);
    }
    __syncthreads();
  }
}

// Level two, in bucket order: the global bin of every record and its
// (arrival-order) slot in that bin.
// Level two, in bucket order: the global bin of every record and its
// (arrival-order) slot in that bin.
__global__ void k_grid_bin(const int4* __restrict__ rec_b, const RsParams* __restrict__ par,
                           int32_t* __restrict__ bin_cnt, int32_t* __restrict__ gbin, int32_t* __restrict__ slot,
                           const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t p = gtid(); p < n; p += gstride()) {
    const int4 r = rec_b[p];
    const int rs = r.w;
    const RsParams P = load_params(par + rs);
    const int row = rs % NROW;
    const int iy = bin_coord(__int_as_float(r.y), -g_row_yhi[row], P.inv_y, P.n_y);
    const int iz = bin_coord(__int_as_float(r.z), P.z_lo, P.inv_z, P.n_z);
    const int gb = P.bin_base + iz * P.n_y + iy;
    gbin[p] = gb;
    slot[p] = atomicAdd(&bin_cnt[gb], 1);
  }
}

// Each record moved to its place in its bin (arrival order inside the bin):
// the writes of a bucket fall inside its own range of the sorted array, so
// they gather in L2 into whole lines.
__global__ void k_grid_scatter(const int4* __restrict__ rec_b, const int32_t* __restrict__ gbin,
                               const int32_t* __restrict__ slot, const int32_t* __restrict__ bin_start,
                               int4* __restrict__ rec_s, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t p = gtid(); p < n; p += gstride()) rec_s[bin_start[gbin[p]] + slot[p]] = rec_b[p];
}

// Stable order inside each bin: the record at sorted position p goes to
// a + rank, a the bin's first position and rank the number of bin members
// with a smaller load index.  Bins hold about two clusters on average (the
// bin edge is sqrt(2 A / n)), and the members sit next to p, so the count
// reads the lines that neighbouring threads read anyway; it is quadratic
// only in the fullest bin.  The bin of a record is recomputed with the
// binning arithmetic of k_grid_bin.  Also clears the cluster-to-track map
// (-1), which is as long as the cluster list.
__global__ void k_grid_order(const int4* __restrict__ rec_s, const RsParams* __restrict__ par,
                             const int32_t* __restrict__ bin_start, int32_t* __restrict__ perm,
                             float2* __restrict__ yz, int32_t* __restrict__ rs_of,
                             int32_t* __restrict__ cluster_track, const Counts* cn) {
  if (fatal(cn)) return;
  const int64_t n = cn->n;
  for (int64_t p = gtid(); p < n; p += gstride()) {
    const int4 r = rec_s[p];
    const int i = r.x, rs = r.w;
    const float y = __int_as_float(r.y), z = __int_as_float(r.z);
    const RsParams P = load_params(par + rs);
    const int row = rs % NROW;
    const int gb = P.bin_base + bin_coord(z, P.z_lo, P.inv_z, P.n_z) * P.n_y +
                   bin_coord(y, -g_row_yhi[row], P.inv_y, P.n_y);
    const int a = bin_start[gb], b = bin_start[gb + 1];
    int rank = 0;
    for (int q = a; q < b; q++) rank += __ldg(&rec_s[q].x) < i;
    const int dst = a + rank;
    perm[dst] = i;
    yz[dst] = make_float2(y, z);
    rs_of[dst] = rs;
    cluster_track[p] = -1;
  }
}

}  // namespace tpc
