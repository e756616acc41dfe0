/*
 * Seeded synthetic TPC cluster generator.
 *
 * This module only simulates detector input: charged helices from the
 * interaction region in a uniform Bz field, intersected with the 159 pad-row
 * planes of the 36 TPC sectors, with Gaussian smearing, row inefficiency and
 * uniform noise (the shape of the Pb-Pb input the ALICE HLT sector tracker
 * processes, Sec. 2; continuous read-out timeframes with z taken from the
 * drift time, Sec. 5).  It contains none of the tracking method's arithmetic:
 * the row crossings are solved in the global frame with a circle/plane
 * intersection, independent of the tracker's x-parametrised propagation.
 *
 * Random numbers come from a counter-based generator: every draw is
 * mix64(key, counter) where mix64 is the SplitMix64 output function
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  Draws are keyed by (seed, domain, object index), so the
 * result does not depend on thread count or iteration order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  float y, z;
  uint16_t row, sector;
  uint32_t id;
} gen_cluster; /* 16 bytes, same layout as the tracker's input cluster */

typedef struct {
  int32_t track;  /* track label, -1 for noise */
  int32_t flags;  /* bit0: local x decreases along the track at this crossing; bits 1+: the leg */
  double y, z;    /* exact (unsmeared) local position; z in the stored coordinate */
  double sphi;    /* sin of the local direction angle */
  double tgl;     /* dz/ds_T in the stored z coordinate */
  double qpt;     /* q/pT in c/GeV */
} gen_truth;

typedef struct {
  uint64_t seed;
  int32_t n_primaries;
  int32_t n_secondaries;
  double pt_min, pt_max; /* GeV/c, power law p^-3 */
  double eta_max;
  double phi_min, phi_max; /* azimuth range, radians (see phi_radius) */
  double phi_radius;       /* 0: the range is that of the initial direction; r > 0: it is the
                              range of the primary's position azimuth where it crosses radius r */
  double sec_r_max;        /* secondaries: vertex uniform in the disk r < sec_r_max */
  uint64_t sector_mask;    /* bit s set: sector s keeps clusters */
  double sigma_y, sigma_z;
  double row_eff;
  double noise_frac; /* noise clusters per track cluster */
  double bz_kg;
  /* continuous read-out timeframe mode */
  int32_t timeframe;
  double tf_length_us;
  double rate_khz;
  double vdrift; /* cm/us */
  double mb_offset; /* track count density ~ 1/(N + mb_offset) */
  double mb_max;    /* on [0, mb_max] */
  int32_t n_threads;
  int32_t legs; /* half-turns of a looper (a circle inside the outermost row radius); 1: the first */
} gen_params;

#define NROWS 159
#define NSEC_AZ 18
#define ZMAX 250.0
static const double X_FIRST = 85.2;
static const double X_LAST = 245.8;
static const double TAN_HALF_SECTOR = 0.17632698070846498; /* tan(10 deg) */
static const double PI = 3.14159265358979323846;

enum { DOM_TRACK = 1, DOM_HIT = 2, DOM_NOISE = 3, DOM_COLL = 4 };

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t make_key(uint64_t seed, uint64_t domain, uint64_t index) {
  return mix64(mix64(seed ^ (domain << 56)) ^ mix64(index + 0x632BE59BD9B4E019ull));
}
/* uniform in [0,1) with 53 random bits */
static inline double uni(uint64_t key, uint64_t ctr) {
  return (double)(mix64(key ^ mix64(ctr)) >> 11) * (1.0 / 9007199254740992.0);
}
/* standard normal by Box-Muller from two draws */
static inline double gauss(uint64_t key, uint64_t ctr) {
  double u1 = 1.0 - uni(key, 2 * ctr);
  double u2 = uni(key, 2 * ctr + 1);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * PI * u2);
}
static inline double pmod(double a, double p) {
  double r = fmod(a, p);
  return r < 0 ? r + p : r;
}

typedef struct {
  double xv, yv;   /* vertex, transverse */
  double phi0;     /* initial direction */
  double pt, q, t; /* t = dz/ds_T = sinh(eta) */
  double tc;       /* collision time, us (timeframe mode) */
} track_t;

/* Pad-row planes sit at the binary32 radii (float)(85.2 + r*(245.8-85.2)/158):
   the tracker stores cluster rows by index and uses these values as x. */
static double row_x(int r) { return (double)(float)(X_FIRST + r * ((X_LAST - X_FIRST) / (NROWS - 1))); }

/* Draw the kinematics of track i (primary or secondary). */
static void sample_track(const gen_params *p, int64_t i, int secondary, double tc, track_t *tr) {
  uint64_t key = make_key(p->seed, DOM_TRACK, (uint64_t)i);
  double a2 = 1.0 / (p->pt_min * p->pt_min), b2 = 1.0 / (p->pt_max * p->pt_max);
  double u = uni(key, 0);
  tr->pt = 1.0 / sqrt(a2 - u * (a2 - b2)); /* inverse CDF of p^-3 on [pt_min, pt_max] */
  double eta = -p->eta_max + 2.0 * p->eta_max * uni(key, 1);
  tr->t = sinh(eta);
  tr->phi0 = p->phi_min + (p->phi_max - p->phi_min) * uni(key, 2);
  tr->q = uni(key, 3) < 0.5 ? 1.0 : -1.0;
  if (p->phi_radius > 0.0) {
    /* a circle through the origin reaches radius rho at position azimuth
       phi0 + sign(kappa) * asin(rho * |kappa| / 2) */
    double kappa = -0.299792458e-3 * p->bz_kg * tr->q / tr->pt;
    double arg = p->phi_radius * fabs(kappa) / 2.0;
    if (arg < 1.0) tr->phi0 -= (kappa > 0 ? 1.0 : -1.0) * asin(arg);
  }
  tr->xv = tr->yv = 0.0;
  if (secondary) {
    double r = p->sec_r_max * sqrt(uni(key, 4));
    double a = 2.0 * PI * uni(key, 5);
    tr->xv = r * cos(a);
    tr->yv = r * sin(a);
  }
  tr->tc = tc;
}

/*
 * All row-plane crossings of one track inside the first outgoing half-turn
 * (from the vertex to the point of the circle farthest from the beam axis)
 * and, for a looper, inside legs-1 further half-turns (no energy loss: the
 * particle stays on its helix).  The truth flags hold the leg (0: the first)
 * in bits 1 and up.  The first `cap` clusters (and truth) are written to out
 * (NULL: none); returns the count, which may exceed cap.
 */
static int64_t track_hits(const gen_params *p, const track_t *tr, int64_t label, gen_cluster *out,
                          gen_truth *truth, int64_t cap) {
  const double K = 0.299792458e-3 * p->bz_kg;
  double kappa = -K * tr->q / tr->pt; /* signed curvature dphi/ds */
  double R = 1.0 / fabs(kappa);
  double sgn = kappa > 0 ? 1.0 : -1.0;
  double xc = tr->xv - sin(tr->phi0) / kappa;
  double yc = tr->yv + cos(tr->phi0) / kappa;
  double cn = hypot(xc, yc);
  double beta = atan2(yc, xc);
  double period = 2.0 * PI * R;
  double phi_far = atan2(sgn * xc, -sgn * yc);
  double s_end = pmod((phi_far - tr->phi0) / kappa, period);
  const int legs = (cn + R < X_LAST && p->legs > 1) ? p->legs : 1;
  const double s_max = s_end + (legs - 1) * PI * R;
  const int turns = (int)floor(s_max / period);
  uint64_t key = make_key(p->seed, DOM_HIT, (uint64_t)label);
  double tf_zmax = p->vdrift * p->tf_length_us;
  int64_t n = 0;
  for (int r = 0; r < NROWS; r++) {
    double xr = row_x(r);
    double arg = (xr * xr - cn * cn - R * R) / (2.0 * R * cn);
    if (arg > 1.0 || arg < -1.0) continue;
    double dpsi = acos(arg);
    int cand[6], nc = 0;
    for (int k = 0; k < 2; k++) {
      double psi = beta + (k ? -dpsi : dpsi);
      double th = atan2(yc + R * sin(psi), xc + R * cos(psi));
      int a = (int)floor(pmod(th, 2.0 * PI) / (2.0 * PI / NSEC_AZ));
      for (int d = -1; d <= 1; d++) {
        int s = ((a + d) % NSEC_AZ + NSEC_AZ) % NSEC_AZ, dup = 0;
        for (int j = 0; j < nc; j++) dup |= cand[j] == s;
        if (!dup) cand[nc++] = s;
      }
    }
    for (int ci = 0; ci < nc; ci++) {
      int a = cand[ci];
      double alpha = (a * 20.0 + 10.0) * PI / 180.0;
      double ca = cos(alpha), sa = sin(alpha);
      double A = xc * ca + yc * sa, B = -xc * sa + yc * ca;
      double w = kappa * (xr - A); /* sin of the local direction at the crossing */
      if (fabs(w) >= 1.0) continue;
      for (int sol = 0; sol < 2 * (turns + 1); sol++) {
        const int j = sol >> 1; /* turn */
        double ploc = (sol & 1) ? PI - asin(w) : asin(w);
        double s = pmod((alpha + ploc - tr->phi0) / kappa, period) + j * period;
        if (!(s > 0.0) || s > s_max) continue;
        const int leg = s <= s_end ? 0 : 1 + (int)floor((s - s_end) / (PI * R));
        double yloc = B - cos(ploc) / kappa;
        if (fabs(yloc) > xr * TAN_HALF_SECTOR) continue;
        double z = tr->t * s;
        if (fabs(z) > ZMAX) continue;
        int sector = a + (z >= 0.0 ? 0 : NSEC_AZ);
        if (!((p->sector_mask >> sector) & 1ull)) continue;
        uint64_t ctr = (((uint64_t)j * NROWS + (uint64_t)r) * 64 + (uint64_t)a) * 2 + (uint64_t)(sol & 1);
        if (uni(key, 8 * ctr) >= p->row_eff) continue;
        double zs = z, tgl = tr->t;
        if (p->timeframe) {
          zs = p->vdrift * tr->tc + (ZMAX - fabs(z));
          tgl = z >= 0.0 ? -tr->t : tr->t;
          if (zs >= tf_zmax) continue; /* arrives after the end of the timeframe */
        }
        if (out && n < cap) {
          gen_cluster *c = &out[n];
          c->y = (float)(yloc + p->sigma_y * gauss(key, 8 * ctr + 2));
          c->z = (float)(zs + p->sigma_z * gauss(key, 8 * ctr + 3));
          c->row = (uint16_t)r;
          c->sector = (uint16_t)sector;
          c->id = (uint32_t)label;
          if (truth) {
            gen_truth *g = &truth[n];
            g->track = (int32_t)label;
            g->flags = (cos(ploc) < 0 ? 1 : 0) | (leg << 1);
            g->y = yloc;
            g->z = zs;
            g->sphi = w;
            g->tgl = tgl;
            g->qpt = tr->q / tr->pt;
          }
        }
        n++;
      }
    }
  }
  return n;
}

/* The track list of an event or timeframe (step 1 of gen_run): *tracks is
   malloc'd with *ntr_out entries.  Returns 0, or -1 on allocation failure. */
static int build_tracks(const gen_params *p, track_t **tracks_out, int64_t *ntr_out) {
  int64_t ntr = 0, cap = 0;
  track_t *tracks = NULL;
  if (!p->timeframe) {
    cap = (int64_t)p->n_primaries + p->n_secondaries;
    tracks = (track_t *)malloc(sizeof(track_t) * (size_t)(cap > 0 ? cap : 1));
    if (!tracks) return -1;
    for (int64_t i = 0; i < p->n_primaries; i++) sample_track(p, ntr, 0, 0.0, &tracks[ntr]), ntr++;
    for (int64_t i = 0; i < p->n_secondaries; i++) sample_track(p, ntr, 1, 0.0, &tracks[ntr]), ntr++;
  } else {
    /* Poisson collision times on [0, tf_length), minimum-bias track counts
       N = off*((max+off)/off)^u - off, i.e. density ~ 1/(N+off) on [0, max] */
    double tcoll = 0.0;
    for (int64_t c = 0;; c++) {
      uint64_t key = make_key(p->seed, DOM_COLL, (uint64_t)c);
      tcoll += -log(1.0 - uni(key, 0)) / (p->rate_khz * 1e-3);
      if (tcoll >= p->tf_length_us) break;
      double ratio = (p->mb_max + p->mb_offset) / p->mb_offset;
      int64_t nt = (int64_t)floor(p->mb_offset * pow(ratio, uni(key, 1)) - p->mb_offset);
      int64_t nsec = (int64_t)floor(nt * ((double)p->n_secondaries / (p->n_primaries > 0 ? p->n_primaries : 1)));
      if (ntr + nt + nsec > cap) {
        cap = (ntr + nt + nsec) * 2 + 1024;
        track_t *t2 = (track_t *)realloc(tracks, sizeof(track_t) * (size_t)cap);
        if (!t2) { free(tracks); return -1; }
        tracks = t2;
      }
      for (int64_t i = 0; i < nt; i++) sample_track(p, ntr, 0, tcoll, &tracks[ntr]), ntr++;
      for (int64_t i = 0; i < nsec; i++) sample_track(p, ntr, 1, tcoll, &tracks[ntr]), ntr++;
    }
  }
  *tracks_out = tracks;
  *ntr_out = ntr;
  return 0;
}

/*
 * Generate one event (or one timeframe).  On success *clusters (and *truth
 * when truth != NULL) point to malloc'd arrays of *n entries, released with
 * gen_free.  Returns 0, or -1 on allocation failure / bad parameters.
 */
int gen_run(const gen_params *p, gen_cluster **clusters, gen_truth **truth, int64_t *n_out,
            int64_t *n_tracks_out) {
  if (!p || !clusters || !n_out || p->pt_min <= 0 || p->pt_max <= p->pt_min) return -1;
  /* 1. the track list */
  int64_t ntr = 0;
  track_t *tracks = NULL;
  if (build_tracks(p, &tracks, &ntr) != 0) return -1;
  /* 2. the tracks' clusters, one pass: fixed chunks of tracks, each into
     its own growing buffer, then concatenated in track order (the output
     does not depend on the thread count) */
  const int64_t CH = 1024;
  const int64_t nchunks = (ntr + CH - 1) / CH;
  typedef struct {
    gen_cluster *c;
    gen_truth *t;
    int64_t n, cap;
    int fail;
  } chunk_buf;
  chunk_buf *cb = (chunk_buf *)calloc((size_t)(nchunks > 0 ? nchunks : 1), sizeof(chunk_buf));
  if (!cb) { free(tracks); return -1; }
#pragma omp parallel for schedule(dynamic, 1) num_threads(p->n_threads > 0 ? p->n_threads : 1)
  for (int64_t k = 0; k < nchunks; k++) {
    chunk_buf *b = &cb[k];
    const int64_t i1 = (k + 1) * CH < ntr ? (k + 1) * CH : ntr;
    for (int64_t i = k * CH; i < i1 && !b->fail; i++) {
      for (;;) {
        const int64_t room = b->cap - b->n;
        const int64_t got = track_hits(p, &tracks[i], i, b->c ? b->c + b->n : NULL,
                                       b->t ? b->t + b->n : NULL, room);
        if (got <= room) {
          b->n += got;
          break;
        }
        int64_t nc = 2 * b->cap > b->n + got + 256 ? 2 * b->cap : b->n + got + 256;
        gen_cluster *c2 = (gen_cluster *)realloc(b->c, sizeof(gen_cluster) * (size_t)nc);
        gen_truth *t2 = NULL;
        if (c2) b->c = c2;
        if (truth) {
          t2 = (gen_truth *)realloc(b->t, sizeof(gen_truth) * (size_t)nc);
          if (t2) b->t = t2;
        }
        if (!c2 || (truth && !t2)) {
          b->fail = 1;
          break;
        }
        b->cap = nc;
      }
    }
  }
  int64_t nhit = 0, bad = 0;
  for (int64_t k = 0; k < nchunks; k++) {
    nhit += cb[k].n;
    bad |= cb[k].fail;
  }
  int64_t nnoise = (int64_t)floor(p->noise_frac * (double)nhit + 0.5);
  int nsel = 0;
  int selected[36];
  for (int s = 0; s < 36; s++)
    if ((p->sector_mask >> s) & 1ull) selected[nsel++] = s;
  if (nsel == 0) nnoise = 0;
  int64_t ntot = nhit + nnoise;
  gen_cluster *out = bad ? NULL : (gen_cluster *)malloc(sizeof(gen_cluster) * (size_t)(ntot > 0 ? ntot : 1));
  gen_truth *tru = truth && !bad ? (gen_truth *)malloc(sizeof(gen_truth) * (size_t)(ntot > 0 ? ntot : 1)) : NULL;
  if (!out || (truth && !tru)) {
    free(out); free(tru);
    for (int64_t k = 0; k < nchunks; k++) { free(cb[k].c); free(cb[k].t); }
    free(cb); free(tracks);
    return -1;
  }
  int64_t *coff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nchunks + 1));
  if (!coff) {
    free(out); free(tru);
    for (int64_t k = 0; k < nchunks; k++) { free(cb[k].c); free(cb[k].t); }
    free(cb); free(tracks);
    return -1;
  }
  coff[0] = 0;
  for (int64_t k = 0; k < nchunks; k++) coff[k + 1] = coff[k] + cb[k].n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(p->n_threads > 0 ? p->n_threads : 1)
  for (int64_t k = 0; k < nchunks; k++) {
    if (cb[k].n) memcpy(out + coff[k], cb[k].c, sizeof(gen_cluster) * (size_t)cb[k].n);
    if (tru && cb[k].n) memcpy(tru + coff[k], cb[k].t, sizeof(gen_truth) * (size_t)cb[k].n);
    free(cb[k].c);
    free(cb[k].t);
  }
  free(coff);
  free(cb);
  /* 3. uniform noise clusters in the selected sectors */
  double tf_zmax = p->vdrift * p->tf_length_us;
  for (int64_t k = 0; k < nnoise; k++) {
    uint64_t key = make_key(p->seed, DOM_NOISE, (uint64_t)k);
    int sector = selected[(int)floor(uni(key, 0) * nsel) % nsel];
    int r = (int)floor(uni(key, 1) * NROWS) % NROWS;
    double ymax = row_x(r) * TAN_HALF_SECTOR;
    double y = -ymax + 2.0 * ymax * uni(key, 2);
    double z;
    if (p->timeframe) z = tf_zmax * uni(key, 3);
    else z = (sector < NSEC_AZ ? 1.0 : -1.0) * ZMAX * uni(key, 3);
    gen_cluster *c = &out[nhit + k];
    c->y = (float)y;
    c->z = (float)z;
    c->row = (uint16_t)r;
    c->sector = (uint16_t)sector;
    c->id = 0xFFFFFFFFu;
    if (tru) {
      gen_truth *g = &tru[nhit + k];
      memset(g, 0, sizeof(*g));
      g->track = -1;
      g->y = y;
      g->z = z;
    }
  }
  free(tracks);
  *clusters = out;
  if (truth) *truth = tru;
  *n_out = ntot;
  if (n_tracks_out) *n_tracks_out = ntr;
  return 0;
}

void gen_free(void *ptr) { free(ptr); }

/* Kinematics of every track of an event or timeframe, in label order:
   out[7*i..7*i+6] = {xv, yv, phi0, pt, q, t, tc} (tc: collision time in us,
   0 for events).  With out == NULL only *n_out is set; otherwise at most cap
   tracks are written.  Returns 0, or -1 on failure. */
int gen_track_table(const gen_params *p, double *out, int64_t cap, int64_t *n_out) {
  track_t *tracks = NULL;
  int64_t ntr = 0;
  if (!p || !n_out || build_tracks(p, &tracks, &ntr) != 0) return -1;
  *n_out = ntr;
  for (int64_t i = 0; out && i < ntr && i < cap; i++) {
    const track_t *tr = &tracks[i];
    double *o = out + 7 * i;
    o[0] = tr->xv; o[1] = tr->yv; o[2] = tr->phi0; o[3] = tr->pt; o[4] = tr->q; o[5] = tr->t; o[6] = tr->tc;
  }
  free(tracks);
  return 0;
}

/* Track kinematics for label i (as drawn by gen_run with the same params):
   out = {xv, yv, phi0, pt, q, t, tc}. Returns -1 if i is out of range. */
int gen_track_info(const gen_params *p, int64_t i, double *out7) {
  if (p->timeframe) return -1; /* collision structure not exposed */
  int64_t ntr = (int64_t)p->n_primaries + p->n_secondaries;
  if (i < 0 || i >= ntr) return -1;
  track_t tr;
  sample_track(p, i, i >= p->n_primaries, 0.0, &tr);
  out7[0] = tr.xv; out7[1] = tr.yv; out7[2] = tr.phi0; out7[3] = tr.pt;
  out7[4] = tr.q; out7[5] = tr.t; out7[6] = tr.tc;
  return 0;
}
