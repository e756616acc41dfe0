/*
 * FP64 CPU oracle for per-sector TPC track finding.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg may load this file's library.  It
 * shares no code with the CUDA path and is written as the plain definition
 * of each step, in the order the method takes them:
 *
 *   Sec. 2 (sector tracker): the TPC is split into 36 sectors tracked
 *   independently.  A cellular automaton forms links between adjacent hits
 *   lying close to a straight line (Fig. 1a) and concatenates them into short
 *   candidates (Fig. 1b).  Track following fits the candidate, extrapolates
 *   row by row to pick up more clusters with a simplified Kalman filter
 *   (Fig. 1c).  A last step selects good tracks and assigns each cluster to
 *   at most one track.  Sec. 2 also: uniform Bz only (no Bx/By).  The final
 *   fit of selected tracks (Sec. 2, "final track fit") is the refit step.
 *
 * The paper gives no thresholds, state vector, Jacobian, grid or seeding;
 * every such constant below is a documented reading, not a printed value,
 * and is therefore "parity unpinned by the paper" as a number (the
 * algorithm is pinned by the invariants and closed forms in the tests).
 *
 * Arithmetic: FP64 throughout, except the grid-bin arithmetic and the
 * neighbour distance, which decide integers (bin indices, link choices) and
 * are therefore evaluated in IEEE binary32 with one rounding per operation,
 * exactly as the CUDA path evaluates them.  Build with -ffp-contract=off.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NROW 159
#define NSEC 36

typedef struct {
  float y, z;
  uint16_t row, sector;
  uint32_t id;
} orc_cluster;

/* Tunable constants of the reading (defaults in orc_default_config). */
typedef struct {
  double bz_kg;      /* uniform field, kG */
  double sigma;      /* cluster resolution in y and z, cm */
  float d_max;       /* max squared straight-line deviation for a link, cm^2 */
  int min_chain;     /* min clusters of a CA chain */
  int max_miss;      /* consecutive rows without a cluster that end an extension */
  int n_min_track;   /* min clusters of a selected track */
  double gate;       /* chi2 gate for picking up a cluster */
  double c0[5];      /* seed covariance diagonal */
  double s_max;      /* |sin phi| limit of the propagation */
  double edge;       /* cm beyond the sector edge that ends an extension */
  double taint_rel;  /* margin of the near-tie / near-gate flags */
  int trace_t;       /* tracklet whose updates are recorded (-1: none) */
  int link_skip;     /* 1: a cluster without an accepted r-1/r+1 pair may link across one empty row */
} orc_config;

void orc_default_config(orc_config *c) {
  c->bz_kg = 5.0;
  c->sigma = 0.1;
  c->d_max = 1.0f;
  c->min_chain = 3;
  c->max_miss = 5;
  c->n_min_track = 10;
  c->gate = 16.0;
  c->c0[0] = 100.0; c->c0[1] = 100.0; c->c0[2] = 1.0; c->c0[3] = 1.0; c->c0[4] = 100.0;
  c->s_max = 0.95;
  c->edge = 2.0;
  c->taint_rel = 1e-4;
  c->trace_t = -1;
  c->link_skip = 0;
}

/* ------------------------------------------------------------- geometry */
/* Pad-row radii linearly spaced 85.2..245.8 cm; active half-width x*tan(10 deg). */
static double row_x64(int r) { return 85.2 + r * ((245.8 - 85.2) / 158.0); }
static const double TAN10 = 0.17632698070846498;
static float X32[NROW], YHI32[NROW];
static void init_tables(void) {
  for (int r = 0; r < NROW; r++) {
    X32[r] = (float)row_x64(r);
    YHI32[r] = (float)(row_x64(r) * TAN10);
  }
}

/* ----------------------------------------------------------- result set */
typedef struct {
  /* counts */
  int64_t n;        /* clusters */
  int32_t n_req;
  int32_t n_rs;     /* row-sectors = n_req * 36 * 159 */
  int64_t n_bins;   /* total grid bins */
  int32_t n_tracklets;
  int32_t n_tracks;
  /* grid (a2): per row-sector */
  int32_t *row_start;  /* [n_rs+1] */
  float *z_lo, *z_hi, *inv_y, *inv_z; /* [n_rs] */
  int32_t *n_y, *n_z;  /* [n_rs] */
  int64_t *bin_base;   /* [n_rs+1] */
  int32_t *bin_start;  /* [n_bins+1] */
  int32_t *perm;       /* [n] sorted position -> input index */
  int32_t *rs_of;      /* [n] sorted position -> row-sector */
  float *sy, *sz;      /* [n] sorted positions */
  /* neighbours (a3) and cleaned links (a4), sorted indexing */
  int32_t *up, *dn, *up_m, *dn_m; /* [n] */
  uint8_t *tie;                   /* [n] */
  /* tracklets (a5) */
  int32_t *tl_start, *tl_len;     /* [n_tracklets] */
  /* follow (a6) per tracklet */
  int32_t *f_n, *f_nf, *f_nb, *f_flags, *f_row; /* [n_tracklets] */
  int32_t *f_hits;                 /* [n_tracklets*NROW] */
  double *f_par;                   /* [n_tracklets*5] at x = X[f_row] */
  double *f_cov;                   /* [n_tracklets*15] packed lower */
  double *f_chi2;                  /* [n_tracklets] */
  /* selection (a7) */
  uint64_t *owner;                 /* [n] max key */
  int32_t *tl_track;               /* [n_tracklets] track index or -1 */
  int32_t *cluster_track;          /* [n] input order */
  /* refit (a8) per track */
  int32_t *t_tracklet, *t_n, *t_ndf, *t_flags, *t_row_in, *t_row_out; /* [n_tracks] */
  double *t_par, *t_cov, *t_chi2;  /* [n_tracks*5], [*15], [n_tracks] */
  /* trace of one tracklet's updates (16 values per record, see follow) */
  double *trace;
  int32_t n_trace;
} orc_result;

enum {
  ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2
};
/* follow / refit flags */
enum {
  F_TAINT_TIE = 1, F_TAINT_GATE = 2, F_TAINT_EDGE = 4, F_TAINT_SLIM = 8,
  F_SEED_FAIL = 16, F_BACK_FAIL = 32, F_REFIT_FAIL = 64
};
#define F_TAINT_ANY (F_TAINT_TIE | F_TAINT_GATE | F_TAINT_EDGE | F_TAINT_SLIM)

/* ================================================================ a2 grid */
/* Bin parameters of one row-sector, in binary32 with one rounding per op. */
static void bin_params(int row, int32_t cnt, float zl, float zh, int32_t *nY, int32_t *nZ, float *invY,
                       float *invZ) {
  float yl = -YHI32[row], yh = YHI32[row];
  float wy = yh - yl;
  float dz = zh - zl;
  float area = wy * fmaxf(dz, 1.0f);
  float s = sqrtf((area * 2.0f) / (float)(cnt > 1 ? cnt : 1));
  s = fminf(fmaxf(s, 1.0f), 64.0f);
  int ny = (int)(wy / s) + 1;
  int nz = (int)(dz / s) + 1;
  if (ny > 256) ny = 256;
  if (nz > 4096) nz = 4096;
  *nY = ny;
  *nZ = nz;
  *invY = (float)ny / wy;
  *invZ = (float)nz / fmaxf(dz, 1e-3f);
}
static int bin_coord(float v, float lo, float inv, int nb) {
  float f = floorf((v - lo) * inv);
  if (f < 0.0f) return 0;
  if (f > (float)(nb - 1)) return nb - 1;
  return (int)f;
}

typedef struct { int32_t bin; int32_t idx; } sort_item;
static int cmp_item(const void *a, const void *b) {
  const sort_item *x = (const sort_item *)a, *y = (const sort_item *)b;
  if (x->bin != y->bin) return x->bin < y->bin ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int build_grid(const orc_cluster *c, int64_t n, const int64_t *req_off, int32_t n_req, orc_result *R) {
  int32_t nrs = n_req * NSEC * NROW;
  R->n_rs = nrs;
  int32_t *cnt = (int32_t *)calloc((size_t)nrs, sizeof(int32_t));
  int32_t *rs_in = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  R->row_start = (int32_t *)calloc((size_t)nrs + 1, sizeof(int32_t));
  R->z_lo = (float *)calloc((size_t)nrs, sizeof(float));
  R->z_hi = (float *)calloc((size_t)nrs, sizeof(float));
  R->inv_y = (float *)calloc((size_t)nrs, sizeof(float));
  R->inv_z = (float *)calloc((size_t)nrs, sizeof(float));
  R->n_y = (int32_t *)calloc((size_t)nrs, sizeof(int32_t));
  R->n_z = (int32_t *)calloc((size_t)nrs, sizeof(int32_t));
  R->bin_base = (int64_t *)calloc((size_t)nrs + 1, sizeof(int64_t));
  if (!cnt || !rs_in || !R->row_start || !R->z_lo || !R->z_hi || !R->inv_y || !R->inv_z || !R->n_y || !R->n_z ||
      !R->bin_base) { free(cnt); free(rs_in); return ORC_ENOMEM; }
  /* row-sector of every cluster; z range per row-sector */
  for (int32_t q = 0; q < n_req; q++)
    for (int64_t i = req_off[q]; i < req_off[q + 1]; i++) {
      int32_t rs = (q * NSEC + c[i].sector) * NROW + c[i].row;
      rs_in[i] = rs;
      if (cnt[rs] == 0 || c[i].z < R->z_lo[rs]) R->z_lo[rs] = c[i].z;
      if (cnt[rs] == 0 || c[i].z > R->z_hi[rs]) R->z_hi[rs] = c[i].z;
      cnt[rs]++;
    }
  for (int32_t rs = 0; rs < nrs; rs++) {
    bin_params(rs % NROW, cnt[rs], R->z_lo[rs], R->z_hi[rs], &R->n_y[rs], &R->n_z[rs], &R->inv_y[rs],
               &R->inv_z[rs]);
    R->row_start[rs + 1] = R->row_start[rs] + cnt[rs];
    R->bin_base[rs + 1] = R->bin_base[rs] + (int64_t)R->n_y[rs] * R->n_z[rs];
  }
  R->n_bins = R->bin_base[nrs];
  /* sort by (row-sector, bin, input index) */
  sort_item *it = (sort_item *)malloc(sizeof(sort_item) * (size_t)(n ? n : 1));
  int32_t *fill = (int32_t *)calloc((size_t)nrs, sizeof(int32_t));
  R->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  R->rs_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  R->sy = (float *)malloc(sizeof(float) * (size_t)(n ? n : 1));
  R->sz = (float *)malloc(sizeof(float) * (size_t)(n ? n : 1));
  R->bin_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R->n_bins + 1));
  if (!it || !fill || !R->perm || !R->rs_of || !R->sy || !R->sz || !R->bin_start) {
    free(it); free(fill); free(cnt); free(rs_in); return ORC_ENOMEM;
  }
  for (int64_t i = 0; i < n; i++) {
    int32_t rs = rs_in[i], row = rs % NROW;
    int iy = bin_coord(c[i].y, -YHI32[row], R->inv_y[rs], R->n_y[rs]);
    int iz = bin_coord(c[i].z, R->z_lo[rs], R->inv_z[rs], R->n_z[rs]);
    int32_t pos = R->row_start[rs] + fill[rs]++;
    it[pos].bin = iz * R->n_y[rs] + iy;
    it[pos].idx = (int32_t)i;
  }
  for (int32_t rs = 0; rs < nrs; rs++) {
    int32_t a = R->row_start[rs], b = R->row_start[rs + 1];
    qsort(it + a, (size_t)(b - a), sizeof(sort_item), cmp_item);
    int64_t nb = R->bin_base[rs + 1] - R->bin_base[rs];
    int32_t p = a;
    for (int64_t k = 0; k < nb; k++) {
      while (p < b && it[p].bin < k) p++;
      R->bin_start[R->bin_base[rs] + k] = p;
    }
    for (int32_t q = a; q < b; q++) {
      R->perm[q] = it[q].idx;
      R->rs_of[q] = rs;
      R->sy[q] = c[it[q].idx].y;
      R->sz[q] = c[it[q].idx].z;
    }
  }
  R->bin_start[R->n_bins] = (int32_t)n;
  free(it); free(fill); free(cnt); free(rs_in);
  return ORC_OK;
}

/* Visit every cluster of row-sector rs whose position lies in the box
   [y0,y1] x [z0,z1], using the grid to skip far bins.  The bin range is
   widened by one bin on each side so that rounding of the box edges can
   never drop a cluster inside the box; the caller applies its exact test. */
typedef struct { int32_t a, b; } span;
static int box_bins(const orc_result *R, int32_t rs, double y0, double y1, double z0, double z1, int *iy0,
                    int *iy1, int *iz0, int *iz1) {
  int row = rs % NROW;
  if (R->row_start[rs + 1] == R->row_start[rs]) return 0;
  double yl = -(double)YHI32[row];
  double fy0 = floor((y0 - yl) * R->inv_y[rs]) - 1, fy1 = floor((y1 - yl) * R->inv_y[rs]) + 1;
  double fz0 = floor((z0 - R->z_lo[rs]) * R->inv_z[rs]) - 1, fz1 = floor((z1 - R->z_lo[rs]) * R->inv_z[rs]) + 1;
  int ny = R->n_y[rs], nz = R->n_z[rs];
  if (fy1 < 0 || fz1 < 0) { /* box entirely below: only the clamped first bins can hold candidates */ }
  *iy0 = fy0 < 0 ? 0 : (fy0 > ny - 1 ? ny - 1 : (int)fy0);
  *iy1 = fy1 < 0 ? 0 : (fy1 > ny - 1 ? ny - 1 : (int)fy1);
  *iz0 = fz0 < 0 ? 0 : (fz0 > nz - 1 ? nz - 1 : (int)fz0);
  *iz1 = fz1 < 0 ? 0 : (fz1 > nz - 1 ? nz - 1 : (int)fz1);
  return 1;
}

/* ========================================================== a3 neighbours */
/* Straight-line deviation of c from the chord d-u, binary32, fixed order. */
static float line_dev(float yd, float zd, float yc, float zc, float yu, float zu, float f) {
  float dy = (yd - yc) + (yu - yd) * f;
  float dz = (zd - zc) + (zu - zd) * f;
  return dy * dy + dz * dz;
}

/* Link windows for a candidate k rows away: k times the one-row slope
   allowance plus the resolution margin (the reading's windows for k = 1). */
static float window_y_k(int k) { return (float)(k * 2.0 * ((245.8 - 85.2) / 158.0) + 0.5); }
static float window_z_k(int k) { return (float)(k * 2.5 * ((245.8 - 85.2) / 158.0) + 0.5); }

/* The clusters of row-sector rs2 inside the window of (yc, zc), appended to
   *lst (brute: every cluster of the row-sector is tested, no grid). */
static void window_list(const orc_result *R, int32_t rs2, float yc, float zc, float WY, float WZ, int brute,
                        int32_t **lst, int *cnt, int *cap) {
  int32_t a0 = 0, a1 = 0;
  int iy0 = 0, iy1 = 0, iz0 = 0, iz1 = 0;
  if (brute) {
    a0 = R->row_start[rs2];
    a1 = R->row_start[rs2 + 1];
  } else if (!box_bins(R, rs2, (double)yc - WY, (double)yc + WY, (double)zc - WZ, (double)zc + WZ, &iy0, &iy1,
                       &iz0, &iz1)) {
    return;
  }
  for (int iz = iz0; iz <= (brute ? iz0 : iz1); iz++)
    for (int iy = iy0; iy <= (brute ? iy0 : iy1); iy++) {
      if (!brute) {
        int64_t gb = R->bin_base[rs2] + (int64_t)iz * R->n_y[rs2] + iy;
        a0 = R->bin_start[gb];
        a1 = R->bin_start[gb + 1];
      }
      for (int32_t k = a0; k < a1; k++)
        if (fabsf(R->sy[k] - yc) <= WY && fabsf(R->sz[k] - zc) <= WZ) {
          if (*cnt == *cap) {
            *cap *= 2;
            *lst = (int32_t *)realloc(*lst, sizeof(int32_t) * (size_t)*cap);
          }
          (*lst)[(*cnt)++] = k;
        }
    }
}

typedef struct {
  float best, second;
  int32_t d, u;
} pair_pick;

/* Every (d, u) pair of the two lists into the pick: the lexicographic
   minimum of (D, d, u) and the smallest D of the other pairs. */
static void pick_pairs(const orc_result *R, float yc, float zc, float f, const int32_t *cd, int nd,
                       const int32_t *cu, int nu, pair_pick *b) {
  for (int i = 0; i < nd; i++)
    for (int j = 0; j < nu; j++) {
      int32_t d = cd[i], u = cu[j];
      float D = line_dev(R->sy[d], R->sz[d], yc, zc, R->sy[u], R->sz[u], f);
      int better = D < b->best || (D == b->best && (d < b->d || (d == b->d && u < b->u)));
      if (b->d < 0 || better) {
        if (b->d >= 0) b->second = fminf(b->second, b->best);
        b->best = D;
        b->d = d;
        b->u = u;
      } else {
        b->second = fminf(b->second, D);
      }
    }
}

/* a3: for each cluster on rows 1..157 the best straight-line pair (d on
   row r-1, u on row r+1).  With link_skip (the next-row variant against
   duplicate tracklets), a cluster on rows 2..156 without an accepted pair
   takes the best pair skipping one row on one side -- (r-2, r+1) or
   (r-1, r+2) -- and, failing that, on both sides (r-2, r+2); windows scale
   with the row distance and the chord fraction is that of the rows
   involved.  The smallest skip is tried first: on a straight line a pair
   further out is as good, and would break the chain. */
static void neighbours(const orc_config *cfg, orc_result *R, int brute) {
  int64_t n = R->n;
  const float WY1 = window_y_k(1), WZ1 = window_z_k(1), WY2 = window_y_k(2), WZ2 = window_z_k(2);
  int cap[4] = {256, 256, 256, 256};
  int32_t *lst[4];
  for (int i = 0; i < 4; i++) lst[i] = (int32_t *)malloc(sizeof(int32_t) * cap[i]);
  for (int64_t c = 0; c < n; c++) {
    R->up[c] = R->dn[c] = -1;
    R->tie[c] = 0;
  }
  for (int64_t c = 0; c < n; c++) {
    int32_t rs = R->rs_of[c], row = rs % NROW;
    if (row < 1 || row > NROW - 2) continue;
    float yc = R->sy[c], zc = R->sz[c];
    /* lists: 0 row r-1, 1 row r+1, 2 row r-2, 3 row r+2 */
    int cnt[4] = {0, 0, 0, 0};
    window_list(R, rs - 1, yc, zc, WY1, WZ1, brute, &lst[0], &cnt[0], &cap[0]);
    window_list(R, rs + 1, yc, zc, WY1, WZ1, brute, &lst[1], &cnt[1], &cap[1]);
    pair_pick b = {INFINITY, INFINITY, -1, -1};
    float f = (X32[row] - X32[row - 1]) / (X32[row + 1] - X32[row - 1]);
    pick_pairs(R, yc, zc, f, lst[0], cnt[0], lst[1], cnt[1], &b);
    if (cfg->link_skip && !(b.d >= 0 && b.best <= cfg->d_max) && row >= 2 && row <= NROW - 3) {
      b.best = b.second = INFINITY;
      b.d = b.u = -1;
      window_list(R, rs - 2, yc, zc, WY2, WZ2, brute, &lst[2], &cnt[2], &cap[2]);
      window_list(R, rs + 2, yc, zc, WY2, WZ2, brute, &lst[3], &cnt[3], &cap[3]);
      const int dr[3] = {-2, -1, -2}, ur[3] = {1, 2, 2}, dl[3] = {2, 0, 2}, ul[3] = {1, 3, 3};
      for (int m = 0; m < 3; m++) {
        if (m == 2) {  /* both sides skipped: only without an accepted one-sided skip */
          if (b.d >= 0 && b.best <= cfg->d_max) break;
          b.best = b.second = INFINITY;
          b.d = b.u = -1;
        }
        float fm = (X32[row] - X32[row + dr[m]]) / (X32[row + ur[m]] - X32[row + dr[m]]);
        pick_pairs(R, yc, zc, fm, lst[dl[m]], cnt[dl[m]], lst[ul[m]], cnt[ul[m]], &b);
      }
    }
    if (b.d >= 0 && b.best <= cfg->d_max) {
      R->up[c] = b.u;
      R->dn[c] = b.d;
      R->tie[c] = (b.second < INFINITY && fabsf(b.second - b.best) <= 1e-6f * fmaxf(b.best, 1e-12f)) ? 1 : 0;
    }
  }
  for (int i = 0; i < 4; i++) free(lst[i]);
}

/* ===================================================== a4 link cleaning */
static void clean_links(orc_result *R) {
  for (int64_t c = 0; c < R->n; c++) {
    int32_t u = R->up[c], d = R->dn[c];
    R->up_m[c] = (u >= 0 && R->dn[u] == c) ? u : -1;
    R->dn_m[c] = (d >= 0 && R->up[d] == c) ? d : -1;
  }
}

/* ========================================================= a5 tracklets */
static int build_tracklets(const orc_config *cfg, orc_result *R) {
  int32_t cap = 1024, nt = 0;
  int32_t *st = (int32_t *)malloc(sizeof(int32_t) * cap), *ln = (int32_t *)malloc(sizeof(int32_t) * cap);
  if (!st || !ln) { free(st); free(ln); return ORC_ENOMEM; }
  for (int64_t c = 0; c < R->n; c++) {
    if (R->up_m[c] < 0 || R->dn_m[c] >= 0) continue;
    int32_t len = 1;
    for (int32_t k = (int32_t)c; R->up_m[k] >= 0; k = R->up_m[k]) len++;
    if (len < cfg->min_chain) continue;
    if (nt == cap) {
      cap *= 2;
      int32_t *a = (int32_t *)realloc(st, sizeof(int32_t) * cap), *b = (int32_t *)realloc(ln, sizeof(int32_t) * cap);
      if (!a || !b) { free(a ? a : st); free(b ? b : ln); return ORC_ENOMEM; }
      st = a; ln = b;
    }
    st[nt] = (int32_t)c;
    ln[nt] = len;
    nt++;
  }
  R->n_tracklets = nt;
  R->tl_start = st;
  R->tl_len = ln;
  return ORC_OK;
}

/* ============================================= a6 Kalman track following */
/* State p = (y, z, sin phi, dz/ds_T, q/pT) at x, full symmetric 5x5 C. */
typedef struct {
  double x, p[5], C[5][5], chi2;
  int nupd;
} kstate;

typedef struct {
  const orc_config *cfg;
  double K;   /* 0.299792458e-3 * Bz[kG], curvature per unit q/pT */
  double V;   /* sigma^2 */
} kctx;

/* C <- J C J^T (full 5x5). */
static void jcjt(const double J[5][5], double C[5][5]) {
  double T[5][5], N[5][5];
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) {
      double a = 0;
      for (int m = 0; m < 5; m++) a += J[i][m] * C[m][j];
      T[i][j] = a;
    }
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) {
      double a = 0;
      for (int m = 0; m < 5; m++) a += T[i][m] * J[j][m];
      N[i][j] = a;
    }
  memcpy(C, N, sizeof(N));
}

/* Propagate to x2 along the helix (exact for the state), first-order
   Jacobian for C.  Returns 0 when |sin phi| would reach s_max. */
static int propagate(const kctx *k, kstate *s, double x2, int *flags) {
  double dx = x2 - s->x;
  double kap = -k->K * s->p[4];
  double s1 = s->p[2], s2 = s1 + kap * dx;
  double smax = k->cfg->s_max;
  if (fabs(fabs(s1) - smax) <= 1e-5 || fabs(fabs(s2) - smax) <= 1e-5) *flags |= F_TAINT_SLIM;
  if (fabs(s1) >= smax || fabs(s2) >= smax) return 0;
  double c1 = sqrt(1.0 - s1 * s1), c2 = sqrt(1.0 - s2 * s2);
  double dy = dx * (s1 + s2) / (c1 + c2);
  double dS;
  /* signed arc length; below |kappa dx| = 1e-6 the chord, signed like dx */
  if (fabs(kap * dx) < 1e-6) dS = copysign(sqrt(dx * dx + dy * dy), dx);
  else dS = (asin(s2) - asin(s1)) / kap;
  double t = s->p[3];
  double sm = 0.5 * (s1 + s2), cm = sqrt(1.0 - sm * sm), cm3 = cm * cm * cm;
  double J[5][5] = {{0}};
  for (int i = 0; i < 5; i++) J[i][i] = 1.0;
  J[0][2] = dx / cm3;
  J[0][4] = -k->K * dx * dx / (2.0 * cm3);
  J[2][4] = -k->K * dx;
  J[1][3] = dS;
  J[1][2] = t * dx * sm / cm3;
  J[1][4] = -t * k->K * dx * dx * sm / (2.0 * cm3);
  jcjt(J, s->C);
  s->p[0] += dy;
  s->p[1] += t * dS;
  s->p[2] = s2;
  s->x = x2;
  return 1;
}

/* Kalman update with the measurement (my, mz), V = diag(sigma^2, sigma^2). */
static void update(const kctx *k, kstate *s, double my, double mz) {
  double r0 = my - s->p[0], r1 = mz - s->p[1];
  double S00 = s->C[0][0] + k->V, S01 = s->C[0][1], S11 = s->C[1][1] + k->V;
  double det = S00 * S11 - S01 * S01;
  double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  double G[5][2];
  for (int i = 0; i < 5; i++) {
    G[i][0] = s->C[i][0] * I00 + s->C[i][1] * I01;
    G[i][1] = s->C[i][0] * I01 + s->C[i][1] * I11;
  }
  for (int i = 0; i < 5; i++) s->p[i] += G[i][0] * r0 + G[i][1] * r1;
  double N[5][5];
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) N[i][j] = s->C[i][j] - (G[i][0] * s->C[0][j] + G[i][1] * s->C[1][j]);
  memcpy(s->C, N, sizeof(N));
  s->chi2 += r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
  s->nupd++;
}

static void reset_cov(const kctx *k, kstate *s) {
  memset(s->C, 0, sizeof(s->C));
  for (int i = 0; i < 5; i++) s->C[i][i] = k->cfg->c0[i];
  s->chi2 = 0.0;
  s->nupd = 0;
}

/* Best cluster on row-sector rs for the predicted state: minimum of
   dy^2/Syy + dz^2/Szz within the gate, ties to the lower sorted index.
   Near-ties and near-gate candidates raise taint flags. */
static int32_t pick(const kctx *k, const orc_result *R, int32_t rs, const kstate *s, int *flags) {
  double Syy = s->C[0][0] + k->V, Szz = s->C[1][1] + k->V;
  double gate = k->cfg->gate, eps = k->cfg->taint_rel;
  double wy = sqrt(gate * Syy), wz = sqrt(gate * Szz);
  double y = s->p[0], z = s->p[1];
  int iy0, iy1, iz0, iz1;
  if (!box_bins(R, rs, y - wy, y + wy, z - wz, z + wz, &iy0, &iy1, &iz0, &iz1)) return -1;
  double b1 = INFINITY, b2 = INFINITY;
  int32_t best = -1;
  for (int iz = iz0; iz <= iz1; iz++)
    for (int iy = iy0; iy <= iy1; iy++) {
      int64_t gb = R->bin_base[rs] + (int64_t)iz * R->n_y[rs] + iy;
      for (int32_t c = R->bin_start[gb]; c < R->bin_start[gb + 1]; c++) {
        double dy = (double)R->sy[c] - y, dz = (double)R->sz[c] - z;
        double chi = dy * dy / Syy + dz * dz / Szz;
        if (fabs(chi - gate) <= eps * (1.0 + gate)) *flags |= F_TAINT_GATE;
        if (!(chi <= gate)) continue;
        if (chi < b1 || (chi == b1 && c < best)) {
          b2 = b1;
          b1 = chi;
          best = c;
        } else if (chi < b2) {
          b2 = chi;
        }
      }
    }
  if (best >= 0 && b2 < INFINITY && b2 - b1 <= eps * (1.0 + b1)) *flags |= F_TAINT_TIE;
  return best;
}

static int outside_sector(const kctx *k, const kstate *s, int *flags) {
  double lim = s->x * TAN10 + k->cfg->edge;
  if (fabs(fabs(s->p[0]) - lim) <= 1e-3) *flags |= F_TAINT_EDGE;
  return fabs(s->p[0]) > lim;
}

static void pack_cov(const double C[5][5], double *out15) {
  int q = 0;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) out15[q++] = C[i][j];
}

/* Update, recording (pass, row, updates since seed, y, z, sin phi, dz/ds,
   q/pT, C_yy, C_zz, C_ss, C_tt, C_qq, chi2, residual y, residual z) when
   tracklet t is the traced one. */
#define ORC_TRACE_MAX 2048
static void traced_update(const kctx *k, orc_result *R, int32_t t, int pass, int row, kstate *s, double my,
                          double mz) {
  double r0 = my - s->p[0], r1 = mz - s->p[1];
  update(k, s, my, mz);
  if (t != k->cfg->trace_t || !R->trace || R->n_trace >= ORC_TRACE_MAX) return;
  double *o = R->trace + 16 * (int64_t)R->n_trace++;
  double v[16] = {pass, row, s->nupd, s->p[0], s->p[1], s->p[2], s->p[3], s->p[4], s->C[0][0], s->C[1][1],
                  s->C[2][2], s->C[3][3], s->C[4][4], s->chi2, r0, r1};
  memcpy(o, v, sizeof(v));
}

/* Follow one tracklet (forward over the chain and outward, then a fresh
   backward pass that refits the forward clusters and extends inward). */
static void follow_one(const kctx *k, orc_result *R, int32_t t) {
  const orc_config *cfg = k->cfg;
  int32_t *hits = R->f_hits + (int64_t)t * NROW;
  int flags = 0, nf = 0, nb = 0;
  int32_t c0 = R->tl_start[t], L = R->tl_len[t];
  int32_t rs0 = R->rs_of[c0];
  int32_t unit_base = rs0 - rs0 % NROW, r0 = rs0 % NROW;
  int32_t chain[NROW];
  chain[0] = c0;
  for (int i = 1; i < L; i++) chain[i] = R->up_m[chain[i - 1]];
  int32_t cl = chain[L - 1];
  const int r_end = R->rs_of[cl] % NROW; /* r0 + L - 1 unless links skip rows */
  /* seed from the chord first -> last chain cluster */
  double x0 = X32[r0], x1 = X32[r_end];
  double dX = x1 - x0, dY = (double)R->sy[cl] - R->sy[c0], dZ = (double)R->sz[cl] - R->sz[c0];
  double Lc = sqrt(dX * dX + dY * dY);
  kstate s;
  s.x = x0;
  s.p[0] = R->sy[c0];
  s.p[1] = R->sz[c0];
  s.p[2] = dY / Lc;
  s.p[3] = dZ / Lc;
  s.p[4] = 0.0;
  reset_cov(k, &s);
  traced_update(k, R, t, 0, r0, &s, R->sy[c0], R->sz[c0]);
  hits[nf++] = c0;
  /* over the chain row by row: an update on every row holding the chain's
     next cluster (a row the links skipped is only crossed) */
  int r = r0;
  for (int i = 1; i < L; i++) {
    const int ri = R->rs_of[chain[i]] % NROW;
    while (r < ri) {
      if (!propagate(k, &s, X32[++r], &flags)) {
        R->f_n[t] = 0; R->f_nf[t] = 0; R->f_nb[t] = 0; R->f_flags[t] = flags | F_SEED_FAIL; R->f_row[t] = r0;
        memset(R->f_par + 5 * (int64_t)t, 0, 5 * sizeof(double));
        memset(R->f_cov + 15 * (int64_t)t, 0, 15 * sizeof(double));
        R->f_chi2[t] = 0;
        return;
      }
    }
    traced_update(k, R, t, 0, ri, &s, R->sy[chain[i]], R->sz[chain[i]]);
    hits[nf++] = chain[i];
  }
  kstate saved = s;
  int r_last = r_end, misses = 0;
  for (int r = r_last + 1; r < NROW; r++) {
    if (!propagate(k, &s, X32[r], &flags)) break;
    if (outside_sector(k, &s, &flags)) break;
    int32_t c = pick(k, R, unit_base + r, &s, &flags);
    if (c >= 0) {
      traced_update(k, R, t, 0, r, &s, R->sy[c], R->sz[c]);
      hits[nf++] = c;
      saved = s;
      r_last = r;
      misses = 0;
    } else if (++misses >= cfg->max_miss) {
      break;
    }
  }
  /* backward pass: re-seed with the forward state at the outermost cluster */
  s = saved;
  reset_cov(k, &s);
  traced_update(k, R, t, 1, r_last, &s, R->sy[hits[nf - 1]], R->sz[hits[nf - 1]]);
  saved = s;
  int kf = nf - 2, ok = 1;
  for (int r = r_last - 1; r >= r0; r--) {
    if (!propagate(k, &s, X32[r], &flags)) { ok = 0; flags |= F_BACK_FAIL; break; }
    if (kf >= 0 && R->rs_of[hits[kf]] % NROW == r) {
      traced_update(k, R, t, 1, r, &s, R->sy[hits[kf]], R->sz[hits[kf]]);
      kf--;
      saved = s;
    }
  }
  if (ok) {
    misses = 0;
    for (int r = r0 - 1; r >= 0; r--) {
      if (!propagate(k, &s, X32[r], &flags)) break;
      if (outside_sector(k, &s, &flags)) break;
      int32_t c = pick(k, R, unit_base + r, &s, &flags);
      if (c >= 0) {
        traced_update(k, R, t, 1, r, &s, R->sy[c], R->sz[c]);
        hits[nf + nb++] = c;
        saved = s;
        misses = 0;
      } else if (++misses >= cfg->max_miss) {
        break;
      }
    }
  }
  R->f_n[t] = nf + nb;
  R->f_nf[t] = nf;
  R->f_nb[t] = nb;
  R->f_flags[t] = flags;
  /* x of the saved state is a row radius */
  int row = 0;
  for (int r = 0; r < NROW; r++)
    if ((double)X32[r] == saved.x) row = r;
  R->f_row[t] = row;
  memcpy(R->f_par + 5 * (int64_t)t, saved.p, 5 * sizeof(double));
  pack_cov(saved.C, R->f_cov + 15 * (int64_t)t);
  R->f_chi2[t] = saved.chi2;
}

typedef struct {
  const kctx *k;
  orc_result *R;
  int32_t lo, hi;
} job;
static void *follow_range(void *arg) {
  job *j = (job *)arg;
  for (int32_t t = j->lo; t < j->hi; t++) follow_one(j->k, j->R, t);
  return NULL;
}

/* ============================================================ a7 select */
static int select_tracks(const orc_config *cfg, orc_result *R) {
  int32_t nt = R->n_tracklets;
  R->owner = (uint64_t *)calloc((size_t)(R->n ? R->n : 1), sizeof(uint64_t));
  R->tl_track = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
  R->cluster_track = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R->n ? R->n : 1));
  if (!R->owner || !R->tl_track || !R->cluster_track) return ORC_ENOMEM;
  /* ownership: the highest key (cluster count, then lower tracklet id) */
  for (int32_t t = 0; t < nt; t++) {
    if (R->f_n[t] < cfg->n_min_track) continue;
    uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
    const int32_t *h = R->f_hits + (int64_t)t * NROW;
    for (int i = 0; i < R->f_n[t]; i++)
      if (key > R->owner[h[i]]) R->owner[h[i]] = key;
  }
  int32_t ntr = 0;
  for (int32_t t = 0; t < nt; t++) {
    R->tl_track[t] = -1;
    if (R->f_n[t] < cfg->n_min_track) continue;
    uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
    const int32_t *h = R->f_hits + (int64_t)t * NROW;
    int kept = 0;
    for (int i = 0; i < R->f_n[t]; i++) kept += R->owner[h[i]] == key;
    if (kept >= cfg->n_min_track) R->tl_track[t] = ntr++;
  }
  R->n_tracks = ntr;
  for (int64_t i = 0; i < R->n; i++) R->cluster_track[i] = -1;
  for (int32_t t = 0; t < nt; t++) {
    if (R->tl_track[t] < 0) continue;
    uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
    const int32_t *h = R->f_hits + (int64_t)t * NROW;
    for (int i = 0; i < R->f_n[t]; i++)
      if (R->owner[h[i]] == key) R->cluster_track[R->perm[h[i]]] = R->tl_track[t];
  }
  return ORC_OK;
}

/* ============================================================= a8 refit */
static int cmp_int(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/* Kalman refit of a kept track over the clusters it owns, from the
   outermost to the innermost, seeded with the follow result carried out to
   the outermost owned row and the seed covariance. */
static void refit_one(const kctx *k, orc_result *R, int32_t tr, int32_t t) {
  const int32_t *h = R->f_hits + (int64_t)t * NROW;
  uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);
  int32_t own[NROW];
  int no = 0;
  for (int i = 0; i < R->f_n[t]; i++)
    if (R->owner[h[i]] == key) own[no++] = h[i];
  qsort(own, (size_t)no, sizeof(int32_t), cmp_int); /* sorted index order = row order within a sector */
  int r_in = R->rs_of[own[0]] % NROW, r_out = R->rs_of[own[no - 1]] % NROW;
  int flags = 0;
  kstate s;
  s.x = X32[R->f_row[t]];
  memcpy(s.p, R->f_par + 5 * (int64_t)t, 5 * sizeof(double));
  reset_cov(k, &s);
  int ok = 1;
  int step = r_out >= R->f_row[t] ? 1 : -1;
  for (int r = R->f_row[t] + step; ok && (step > 0 ? r <= r_out : r >= r_out); r += step) {
    ok = propagate(k, &s, X32[r], &flags);
  }
  if (ok) {
    reset_cov(k, &s);
    int q = no - 1;
    update(k, &s, R->sy[own[q]], R->sz[own[q]]);
    q--;
    for (int r = r_out - 1; ok && r >= r_in; r--) {
      ok = propagate(k, &s, X32[r], &flags);
      if (ok && q >= 0 && R->rs_of[own[q]] % NROW == r) {
        update(k, &s, R->sy[own[q]], R->sz[own[q]]);
        q--;
      }
    }
  }
  R->t_tracklet[tr] = t;
  R->t_n[tr] = no;
  R->t_row_in[tr] = r_in;
  R->t_row_out[tr] = r_out;
  if (ok) {
    memcpy(R->t_par + 5 * (int64_t)tr, s.p, 5 * sizeof(double));
    pack_cov(s.C, R->t_cov + 15 * (int64_t)tr);
    R->t_chi2[tr] = s.chi2;
    R->t_ndf[tr] = 2 * no - 5;
    R->t_flags[tr] = flags;
  } else {
    memcpy(R->t_par + 5 * (int64_t)tr, R->f_par + 5 * (int64_t)t, 5 * sizeof(double));
    memcpy(R->t_cov + 15 * (int64_t)tr, R->f_cov + 15 * (int64_t)t, 15 * sizeof(double));
    R->t_chi2[tr] = R->f_chi2[t];
    R->t_ndf[tr] = 2 * no - 5;
    R->t_flags[tr] = F_REFIT_FAIL;
    R->t_row_in[tr] = R->f_row[t];
  }
}

static void *refit_range(void *arg) {
  job *j = (job *)arg;
  for (int32_t t = j->lo; t < j->hi; t++)
    if (j->R->tl_track[t] >= 0) refit_one(j->k, j->R, j->R->tl_track[t], t);
  return NULL;
}

static void run_parallel(void *(*fn)(void *), const kctx *k, orc_result *R, int32_t n, int threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pthread_t th[256];
  int started[256];
  job jobs[256];
  int32_t chunk = (n + threads - 1) / threads;
  for (int i = 0; i < threads; i++) {
    jobs[i].k = k;
    jobs[i].R = R;
    jobs[i].lo = (int64_t)i * chunk < n ? i * chunk : n;
    jobs[i].hi = (int64_t)(i + 1) * chunk < n ? (i + 1) * chunk : n;
    started[i] = threads > 1 && pthread_create(&th[i], NULL, fn, &jobs[i]) == 0;
    if (!started[i]) fn(&jobs[i]);
  }
  for (int i = 0; i < threads; i++)
    if (started[i]) pthread_join(th[i], NULL);
}

/* ================================================================ driver */
void orc_free(orc_result *R) {
  void *ptrs[] = {R->row_start, R->z_lo, R->z_hi, R->inv_y, R->inv_z, R->n_y, R->n_z, R->bin_base, R->bin_start,
                  R->perm, R->rs_of, R->sy, R->sz, R->up, R->dn, R->up_m, R->dn_m, R->tie, R->tl_start,
                  R->tl_len, R->f_n, R->f_nf, R->f_nb, R->f_flags, R->f_row, R->f_hits, R->f_par, R->f_cov,
                  R->f_chi2, R->owner, R->tl_track, R->cluster_track, R->t_tracklet, R->t_n, R->t_ndf,
                  R->t_flags, R->t_row_in, R->t_row_out, R->t_par, R->t_cov, R->t_chi2, R->trace};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
  memset(R, 0, sizeof(*R));
}

/*
 * Run the whole sector tracker on n clusters forming n_req independent
 * requests (request q = clusters [req_off[q], req_off[q+1])).  stop_after:
 * 2 grid, 3 neighbours, 4 links, 5 tracklets, 6 follow, 7 select, 8 refit.
 * brute != 0 uses an all-pairs neighbour scan instead of the grid.
 */
int orc_run(const orc_config *cfg_in, const orc_cluster *c, int64_t n, const int64_t *req_off, int32_t n_req,
            int stop_after, int brute, int threads, orc_result *R) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  memset(R, 0, sizeof(*R));
  init_tables();
  if (n < 0 || n_req < 1 || req_off[0] != 0 || req_off[n_req] != n || n > 0x7FFFFFFF) return ORC_EINVAL;
  for (int32_t q = 0; q < n_req; q++)
    if (req_off[q + 1] < req_off[q]) return ORC_EINVAL;
  for (int64_t i = 0; i < n; i++)
    if (c[i].row >= NROW || c[i].sector >= NSEC || !isfinite(c[i].y) || !isfinite(c[i].z)) return ORC_EINVAL;
  R->n = n;
  R->n_req = n_req;
  int rc = build_grid(c, n, req_off, n_req, R);
  if (rc || stop_after <= 2) return rc;
  size_t nn = (size_t)(n ? n : 1);
  R->up = (int32_t *)malloc(4 * nn); R->dn = (int32_t *)malloc(4 * nn);
  R->up_m = (int32_t *)malloc(4 * nn); R->dn_m = (int32_t *)malloc(4 * nn);
  R->tie = (uint8_t *)malloc(nn);
  if (!R->up || !R->dn || !R->up_m || !R->dn_m || !R->tie) return ORC_ENOMEM;
  neighbours(&cfg, R, brute);
  if (stop_after <= 3) return ORC_OK;
  clean_links(R);
  if (stop_after <= 4) return ORC_OK;
  rc = build_tracklets(&cfg, R);
  if (rc || stop_after <= 5) return rc;
  size_t nt = (size_t)(R->n_tracklets ? R->n_tracklets : 1);
  R->f_n = (int32_t *)calloc(nt, 4); R->f_nf = (int32_t *)calloc(nt, 4); R->f_nb = (int32_t *)calloc(nt, 4);
  R->f_flags = (int32_t *)calloc(nt, 4); R->f_row = (int32_t *)calloc(nt, 4);
  R->f_hits = (int32_t *)malloc(4 * nt * NROW);
  R->f_par = (double *)calloc(nt * 5, 8); R->f_cov = (double *)calloc(nt * 15, 8); R->f_chi2 = (double *)calloc(nt, 8);
  if (!R->f_n || !R->f_nf || !R->f_nb || !R->f_flags || !R->f_row || !R->f_hits || !R->f_par || !R->f_cov ||
      !R->f_chi2) return ORC_ENOMEM;
  for (size_t i = 0; i < nt * NROW; i++) R->f_hits[i] = -1;
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  if (cfg.trace_t >= 0) {
    R->trace = (double *)calloc(16 * ORC_TRACE_MAX, sizeof(double));
    if (!R->trace) return ORC_ENOMEM;
  }
  run_parallel(follow_range, &k, R, R->n_tracklets, threads);
  if (stop_after <= 6) return ORC_OK;
  rc = select_tracks(&cfg, R);
  if (rc || stop_after <= 7) return rc;
  size_t ntr = (size_t)(R->n_tracks ? R->n_tracks : 1);
  R->t_tracklet = (int32_t *)calloc(ntr, 4); R->t_n = (int32_t *)calloc(ntr, 4); R->t_ndf = (int32_t *)calloc(ntr, 4);
  R->t_flags = (int32_t *)calloc(ntr, 4); R->t_row_in = (int32_t *)calloc(ntr, 4);
  R->t_row_out = (int32_t *)calloc(ntr, 4);
  R->t_par = (double *)calloc(ntr * 5, 8); R->t_cov = (double *)calloc(ntr * 15, 8); R->t_chi2 = (double *)calloc(ntr, 8);
  if (!R->t_tracklet || !R->t_n || !R->t_ndf || !R->t_flags || !R->t_row_in || !R->t_row_out || !R->t_par ||
      !R->t_cov || !R->t_chi2) return ORC_ENOMEM;
  run_parallel(refit_range, &k, R, R->n_tracklets, threads);
  return ORC_OK;
}

/*
 * Direct Kalman fit (for the closed-form tests): starting from the state p0
 * at row rows[0] with covariance diag(c0) (cfg), update with (my[i], mz[i])
 * at rows[i] for i = 0..m-1, propagating row by row in between (rows must be
 * monotone).  Returns 1 on success and the final state, packed covariance
 * and chi2.
 */
int orc_kalman_fit(const orc_config *cfg_in, int m, const int32_t *rows, const double *my, const double *mz,
                   const double *p0, double *p_out, double *cov_out, double *chi2_out) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  init_tables();
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  kstate s;
  int flags = 0;
  s.x = X32[rows[0]];
  memcpy(s.p, p0, 5 * sizeof(double));
  reset_cov(&k, &s);
  for (int i = 0; i < m; i++) {
    if (i > 0) {
      int step = rows[i] > rows[i - 1] ? 1 : -1;
      for (int r = rows[i - 1] + step; step > 0 ? r <= rows[i] : r >= rows[i]; r += step)
        if (!propagate(&k, &s, X32[r], &flags)) return 0;
    }
    update(&k, &s, my[i], mz[i]);
  }
  memcpy(p_out, s.p, 5 * sizeof(double));
  pack_cov(s.C, cov_out);
  *chi2_out = s.chi2;
  return 1;
}

/* State-only helix propagation over a list of rows (for the exact-helix
   test): p is carried from rows[0] to rows[i] and written to out[5*i]. */
int orc_propagate_rows(const orc_config *cfg_in, int m, const int32_t *rows, const double *p0, double *out) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  init_tables();
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  kstate s;
  int flags = 0;
  s.x = X32[rows[0]];
  memcpy(s.p, p0, 5 * sizeof(double));
  reset_cov(&k, &s);
  memcpy(out, s.p, 5 * sizeof(double));
  for (int i = 1; i < m; i++) {
    int step = rows[i] > rows[i - 1] ? 1 : -1;
    for (int r = rows[i - 1] + step; step > 0 ? r <= rows[i] : r >= rows[i]; r += step)
      if (!propagate(&k, &s, X32[r], &flags)) return 0;
    memcpy(out + 5 * i, s.p, 5 * sizeof(double));
  }
  return 1;
}

/* ================================== track-model compression (next row) */
/* The track-model compression of the paper's compression section: the
   track is refitted over its own clusters, and at each cluster the residual
   between the cluster and the extrapolated track position is stored; the
   decompression repeats the same fit and adds the residuals back, which is
   exact because both sides see the same (quantised) clusters.  The
   distortion transform of the paper is the identity here (the synthetic
   clusters carry no distortion).  Cluster coordinates are fixed point:
   q = rint(v * (1/unit)) in binary32 (the lossy format conversion); the
   stored residual is q - rint(prediction / unit), and the fit is updated
   with the decoded value q * unit (binary32).
   Per track: a header (row_out, the state at the outermost cluster) and
   its clusters outermost first (rows, fixed-point y and z).  decode = 0:
   qy/qz in, ry/rz out; decode = 1: ry/rz in, qy/qz out.  margin (out,
   optional): distance of prediction / unit from the rounding boundary,
   per cluster.  Returns 1, or 0 if a propagation fails (that track's
   clusters are left as they are). */
static int codec_one(const kctx *k, int decode, int32_t row_out, const double *head, int64_t n,
                     const int32_t *rows, int32_t *qy, int32_t *qz, int32_t *ry, int32_t *rz, double *margin,
                     double unit) {
  kstate s;
  int flags = 0;
  s.x = X32[row_out];
  memcpy(s.p, head, 5 * sizeof(double));
  reset_cov(k, &s);
  int row = row_out;
  const float u32 = (float)unit;
  for (int64_t i = 0; i < n; i++) {
    while (row > rows[i]) {
      row--;
      if (!propagate(k, &s, X32[row], &flags)) return 0;
    }
    const double fy = s.p[0] / unit, fz = s.p[1] / unit;
    const double py = rint(fy), pz = rint(fz);
    if (margin) margin[i] = fmin(fabs(fabs(fy - floor(fy)) - 0.5), fabs(fabs(fz - floor(fz)) - 0.5));
    if (decode) {
      qy[i] = (int32_t)py + ry[i];
      qz[i] = (int32_t)pz + rz[i];
    } else {
      ry[i] = qy[i] - (int32_t)py;
      rz[i] = qz[i] - (int32_t)pz;
    }
    update(k, &s, (double)((float)qy[i] * u32), (double)((float)qz[i] * u32));
  }
  return 1;
}

int orc_codec(const orc_config *cfg_in, int decode, int32_t n_tracks, const int32_t *row_out, const double *head,
              const int64_t *off, const int32_t *rows, int32_t *qy, int32_t *qz, int32_t *ry, int32_t *rz,
              double *margin, double unit, int32_t *ok) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  init_tables();
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  for (int32_t t = 0; t < n_tracks; t++) {
    const int64_t a = off[t], n = off[t + 1] - off[t];
    ok[t] = codec_one(&k, decode, row_out[t], head + 5 * (int64_t)t, n, rows + a, qy + a, qz + a, ry + a, rz + a,
                      margin ? margin + a : NULL, unit);
  }
  return 0;
}

/* Fixed-point cluster coordinate: rint(v * (1/unit)) in binary32. */
void orc_quantise(int64_t n, const float *v, double unit, int32_t *q) {
  const float inv = (float)(1.0 / unit);
  for (int64_t i = 0; i < n; i++) q[i] = (int32_t)rintf(v[i] * inv);
}

/* ======================================== sector-track merging (next row) */
/* The second tracking phase of Sec. 2 merges the segments the sector
   tracker found in different sectors and refits the merged tracks.  The
   reading implemented here:
   - a segment is a refitted sector track: state at its innermost row in its
     sector's frame (centre angle (s mod 18)*20+10 degrees), covariance, its
     clusters;
   - an inner segment A (sector s) and an outer segment B (sector s' = s +-1
     on the same side, A.row_out <= B.row_in + overlap) are compared at B's
     innermost row: A's state is turned into B's frame and carried there;
     the pair is a candidate if the z of the two there differ by at most
     window_cm (a bound far wider than any true pair's residual: it lets a
     tracker look only at segments near the predicted z), and then
     chi2 = d^T (C_A + C_B)^-1 d over the five parameters; a pair with
     chi2 <= chi2_max that is the best of both A's and B's candidates is
     merged (chains follow the merges);
   - a merged track is refitted from its outermost segment's start (the
     refit's seed) inward over all its clusters, the state and covariance
     turned into the next segment's frame between segments; the result is
     given at the innermost cluster in the innermost segment's frame. */

static double sector_angle(int s) { return ((s % 18) * 20.0 + 10.0) * M_PI / 180.0; }

/* The state at x in a frame turned into the frame rotated by beta (new
   frame = old frame rotated by +beta about the beam axis), kept on its own
   point: x' = x cos b + y sin b, y' = -x sin b + y cos b, phi' = phi - b.
   Covariance: derivatives at fixed x', J[y][y] = cos phi / cos phi',
   J[s][s] = cos phi' / cos phi, J[z][y] = -t sin b / cos phi'.  Returns 0
   if the direction would leave the frame's outward half-plane. */
static int rotate(kstate *s, double beta) {
  const double ca = cos(beta), sa = sin(beta);
  const double sp = s->p[2], cp = sqrt(1.0 - sp * sp);
  const double sp2 = sp * ca - cp * sa, cp2 = cp * ca + sp * sa;
  if (!(cp2 > 0.05)) return 0;
  double J[5][5] = {{0}};
  for (int i = 0; i < 5; i++) J[i][i] = 1.0;
  J[0][0] = cp / cp2;
  J[2][2] = cp2 / cp;
  J[1][0] = -s->p[3] * sa / cp2;
  jcjt(J, s->C);
  const double x = s->x, y = s->p[0];
  s->x = x * ca + y * sa;
  s->p[0] = -x * sa + y * ca;
  s->p[2] = sp2;
  return 1;
}

/* Propagation to a radius that need not be a row's (row-by-row steps on
   the way, as the filter does, then the last piece). */
static int carry_to(const kctx *k, kstate *s, double x2, int *flags) {
  return propagate(k, s, x2, flags);
}

/* chi2 of d with covariance S (5x5, Cholesky); -1 if S is not positive. */
static double chi2_5(const double d[5], double S[5][5]) {
  double L[5][5] = {{0}};
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) {
      double a = S[i][j];
      for (int m = 0; m < j; m++) a -= L[i][m] * L[j][m];
      if (i == j) {
        if (!(a > 0)) return -1.0;
        L[i][i] = sqrt(a);
      } else {
        L[i][j] = a / L[j][j];
      }
    }
  double w[5], c = 0;
  for (int i = 0; i < 5; i++) {
    double a = d[i];
    for (int m = 0; m < i; m++) a -= L[i][m] * w[m];
    w[i] = a / L[i][i];
    c += w[i] * w[i];
  }
  return c;
}

static void unpack_cov(const double *c15, double C[5][5]) {
  int q = 0;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++, q++) C[i][j] = C[j][i] = c15[q];
}

/* Pair chi2 of inner segment a with outer segment b (-1: not comparable,
   or their z at b's first row further apart than window_cm). */
static double pair_chi2(const kctx *k, const int32_t *sector, const int32_t *row_in, const double *par,
                        const double *cov, int a, int b, double window_cm) {
  kstate s;
  int flags = 0;
  s.x = X32[row_in[a]];
  memcpy(s.p, par + 5 * (int64_t)a, 5 * sizeof(double));
  unpack_cov(cov + 15 * (int64_t)a, s.C);
  if (!rotate(&s, sector_angle(sector[b]) - sector_angle(sector[a]))) return -1.0;
  if (!carry_to(k, &s, X32[row_in[b]], &flags)) return -1.0;
  if (!(fabs(s.p[1] - par[5 * (int64_t)b + 1]) <= window_cm)) return -1.0;
  double d[5], Cb[5][5], S[5][5];
  unpack_cov(cov + 15 * (int64_t)b, Cb);
  for (int i = 0; i < 5; i++) {
    d[i] = s.p[i] - par[5 * (int64_t)b + i];
    for (int j = 0; j < 5; j++) S[i][j] = s.C[i][j] + Cb[i][j];
  }
  return chi2_5(d, S);
}

static int adjacent(int s1, int s2) {
  if (s1 / 18 != s2 / 18) return 0;
  const int d = ((s2 % 18) - (s1 % 18) + 18) % 18;
  return d == 1 || d == 17;
}

/* Pairing: for every segment its best partner inward (best_in) and outward
   (best_out) with the pair's chi2 and the second-best chi2 (for the taint
   of near ties); a merge where both choose each other.  out_link[a] = b
   (-1: none).  Segments: n_tracks, with request, sector, rows, state. */
int orc_merge_pairs(const orc_config *cfg_in, int32_t n, const int32_t *request, const int32_t *sector,
                    const int32_t *row_in, const int32_t *row_out, const int32_t *n_clusters, const double *par,
                    const double *cov, double chi2_max, int32_t overlap, int32_t min_clusters, double window_cm,
                    int32_t *out_link,
                    double *out_chi2, double *out_second, double *out_second_in) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  init_tables();
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  int32_t *bo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double *co = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *so = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *ci = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *si = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!bo || !bi || !co || !so || !ci || !si) {
    free(bo); free(bi); free(co); free(so); free(ci); free(si);
    return ORC_ENOMEM;
  }
  for (int32_t a = 0; a < n; a++) {
    bo[a] = bi[a] = -1;
    co[a] = ci[a] = so[a] = si[a] = INFINITY;
  }
  for (int32_t a = 0; a < n; a++) {
    if (n_clusters[a] < min_clusters) continue;
    for (int32_t b = 0; b < n; b++) {
      if (b == a || request[b] != request[a] || n_clusters[b] < min_clusters) continue;
      if (!adjacent(sector[a], sector[b])) continue;
      if (!(row_in[a] < row_in[b] && row_out[a] <= row_in[b] + overlap)) continue; /* a inner, b outer */
      const double c = pair_chi2(&k, sector, row_in, par, cov, a, b, window_cm);
      if (c < 0 || c > chi2_max) continue;
      if (c < co[a] || (c == co[a] && b < bo[a])) {
        so[a] = fmin(so[a], co[a]);
        co[a] = c;
        bo[a] = b;
      } else {
        so[a] = fmin(so[a], c);
      }
      if (c < ci[b] || (c == ci[b] && a < bi[b])) {
        si[b] = fmin(si[b], ci[b]);
        ci[b] = c;
        bi[b] = a;
      } else {
        si[b] = fmin(si[b], c);
      }
    }
  }
  for (int32_t a = 0; a < n; a++) {
    const int32_t b = bo[a];
    out_link[a] = (b >= 0 && bi[b] == a) ? b : -1;
    out_chi2[a] = co[a];
    out_second[a] = so[a];
    out_second_in[a] = si[a];
  }
  free(bo); free(bi); free(co); free(so); free(ci); free(si);
  return ORC_OK;
}

/* Refit of a chain of segments, outermost first: chain[0..m) segment ids,
   their clusters (rows, y, z in each segment's frame) outermost first in
   one list with offsets; seed = the outermost segment's state at its
   outermost row (the refit's seed).  Output at the innermost cluster in the
   innermost segment's frame. */
int orc_merge_refit(const orc_config *cfg_in, int32_t m, const int32_t *seg_sector, const int64_t *seg_off,
                    const int32_t *rows, const double *y, const double *z, int32_t seed_row, const double *seed,
                    double *par_out, double *cov_out, double *chi2_out, int32_t *row_out_inner) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  init_tables();
  kctx k = {&cfg, 0.299792458e-3 * cfg.bz_kg, cfg.sigma * cfg.sigma};
  kstate s;
  int flags = 0;
  s.x = X32[seed_row];
  memcpy(s.p, seed, 5 * sizeof(double));
  reset_cov(&k, &s);
  int row = seed_row;
  for (int32_t g = 0; g < m; g++) {
    if (g > 0) {
      if (!rotate(&s, sector_angle(seg_sector[g]) - sector_angle(seg_sector[g - 1]))) return 0;
      row = NROW; /* the next propagation goes to the segment's first row, wherever x now is */
    }
    for (int64_t i = seg_off[g]; i < seg_off[g + 1]; i++) {
      if (row == NROW) {
        if (!carry_to(&k, &s, X32[rows[i]], &flags)) return 0;
        row = rows[i];
      }
      while (row > rows[i]) {
        row--;
        if (!propagate(&k, &s, X32[row], &flags)) return 0;
      }
      update(&k, &s, y[i], z[i]);
    }
  }
  memcpy(par_out, s.p, 5 * sizeof(double));
  pack_cov(s.C, cov_out);
  *chi2_out = s.chi2;
  *row_out_inner = row;
  return 1;
}

/* Row radii and half-widths as the oracle uses them (binary32). */
void orc_tables(float *x, float *yhi) {
  init_tables();
  memcpy(x, X32, sizeof(X32));
  memcpy(yhi, YHI32, sizeof(YHI32));
}
