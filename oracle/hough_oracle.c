/*
 * CPU ORACLE of the conformal Hough hit filter -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow restatement of the method for checking the CUDA path: nested
 * loops over events, hits and theta columns in int64, no blocking, no fusion.
 * Only tests, the package's smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does. It shares no code, header or
 * constant table with the CUDA library: every constant and table below is
 * defined here, from the paper's definitions.
 *
 * Steps (paper Sec. 2 and Sec. 3):
 *   1. trig tables   c_j = round(2^14 cos th_j), s_j = round(2^14 sin th_j),
 *                    th_j = (j + 1/2) pi / N_theta  (equal-width bins over [0, pi), Sec. 2)
 *   2. map, Eq. (1) with the factor 2 that makes Eq. (2) hold:
 *                    u_q = floor(2 x 2^32 / (x^2 + y^2)), v_q likewise (x, y in um)
 *   3. rho matrix    rho_q(i, j) = u_q(i) c_j + v_q(i) s_j   (matrix R, Sec. 3), scale 2^46 per um
 *   4. vote          k = clamp(floor((rho_q + H) N_rho / (2H)), 0, N_rho - 1), acc[j][k] += 1,
 *                    H = round(0.01 mm^-1 * 1e-3 mm/um * 2^46): rho in [-0.01, 0.01] mm^-1 (Sec. 2)
 *   5. peaks         acc >= T and a 3x3 local maximum (Sec. 2 peak finding with neighbourhood
 *                    suppression); ties: strictly greater than the neighbours that precede the
 *                    cell in raster (theta-major) order, greater or equal to those that follow;
 *                    theta wraps: column -1 is column N_theta-1 and column N_theta is column 0,
 *                    both with rho mirrored (k -> N_rho-1-k); neighbours beyond the rho edges
 *                    are skipped. Peaks are listed in raster order, at most max_peaks stored.
 *   6. select        a hit is kept if, at the theta column of some stored peak, its rho bin lies
 *                    within keep_halfwidth of the peak's rho bin (back-projection data filtering,
 *                    Sec. 2); Eq. (8) R_c and Eq. (9) R_s follow from the kept mask.
 * The peak/tie/wrap rule, the clamping, the bin-centre theta samples and the
 * factor 2 are readings of passages the paper leaves open.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_TRIG_SCALE 16384.0
#define OR_H 703687442LL /* 0.01 mm^-1 in units of 2^-46 um^-1 */
#define OR_COORD_MAX (1LL << 24)
#define OR_MAX_EVENT_HITS 32767

/* status flags (bit values fixed by the library's public interface) */
#define OR_F_BAD_HIT 1
#define OR_F_BAD_OFFSETS 2
#define OR_F_PEAK_OVERFLOW 4
#define OR_F_EVENT_TOO_LARGE 8

typedef struct or_params {
  int32_t n_theta, n_rho, threshold, keep_halfwidth, max_peaks;
  int32_t theta_tiles, events_per_cta, block; /* unused by the oracle */
  int32_t peak_mode;                          /* 0: one-pass 3x3 local maxima, 1: iterative (step 5') */
  int32_t rel_num, rel_den, nms_radius;       /* step 5' */
} or_params;

typedef struct or_peak {
  int16_t theta_bin, rho_bin, votes, flags;
} or_peak;

static const double OR_PI = 3.14159265358979323846;

/* Step 1: trig tables over bin-centre angles. */
void or_tables(int32_t n_theta, int16_t* c, int16_t* s) {
  for (int32_t j = 0; j < n_theta; ++j) {
    double th = (j + 0.5) * OR_PI / n_theta;
    c[j] = (int16_t)llround(OR_TRIG_SCALE * cos(th));
    s[j] = (int16_t)llround(OR_TRIG_SCALE * sin(th));
  }
}

/* floor(a / b) for b > 0 (C division truncates toward zero). */
static int64_t or_floor_div(int64_t a, int64_t b) {
  int64_t q = a / b, r = a % b;
  if (r != 0 && a < 0) q -= 1;
  return q;
}

/* Step 2: conformal map of one hit. Returns 0, or OR_F_BAD_HIT for r = 0 or |x|,|y| > 2^24. */
int32_t or_map_hit(int32_t x, int32_t y, int64_t* uq, int64_t* vq) {
  int64_t X = x, Y = y;
  if (X > OR_COORD_MAX || X < -OR_COORD_MAX || Y > OR_COORD_MAX || Y < -OR_COORD_MAX) return OR_F_BAD_HIT;
  int64_t r2 = X * X + Y * Y;
  if (r2 == 0) return OR_F_BAD_HIT;
  *uq = or_floor_div(2 * X * (1LL << 32), r2);
  *vq = or_floor_div(2 * Y * (1LL << 32), r2);
  return 0;
}

/* Steps 3-4: rho of a mapped hit at one column, then its bin. */
int64_t or_rho(int64_t uq, int64_t vq, int16_t c, int16_t s) { return uq * (int64_t)c + vq * (int64_t)s; }

int32_t or_bin(int64_t rho, int32_t n_rho) {
  int64_t t = rho + OR_H;
  if (t < 0) return 0;
  int64_t k = (t * n_rho) / (2 * OR_H);
  if (k > n_rho - 1) k = n_rho - 1;
  return (int32_t)k;
}

/* Step 5 on a given accumulator [n_theta][n_rho]. Returns the true peak count (may exceed max_peaks). */
int32_t or_peaks(const int16_t* acc, const or_params* p, or_peak* out) {
  const int32_t NT = p->n_theta, NR = p->n_rho;
  int32_t n = 0;
  for (int32_t j = 0; j < NT; ++j) {
    for (int32_t k = 0; k < NR; ++k) {
      int32_t a = acc[(int64_t)j * NR + k];
      if (a < p->threshold) continue;
      int is_peak = 1;
      for (int dj = -1; dj <= 1 && is_peak; ++dj) {
        for (int dk = -1; dk <= 1; ++dk) {
          if (dj == 0 && dk == 0) continue;
          int32_t kk = k + dk, jj = j + dj;
          if (kk < 0 || kk >= NR) continue;
          if (jj == -1) {
            jj = NT - 1;
            kk = NR - 1 - kk;
          } else if (jj == NT) {
            jj = 0;
            kk = NR - 1 - kk;
          }
          int32_t b = acc[(int64_t)jj * NR + kk];
          int precedes = ((int64_t)jj * NR + kk) < ((int64_t)j * NR + k);
          if (precedes ? !(a > b) : !(a >= b)) {
            is_peak = 0;
            break;
          }
        }
      }
      if (!is_peak) continue;
      if (n < p->max_peaks) {
        out[n].theta_bin = (int16_t)j;
        out[n].rho_bin = (int16_t)k;
        out[n].votes = (int16_t)a;
        out[n].flags = 0;
      }
      ++n;
    }
  }
  return n;
}

/* Step 5' (the paper's own peak finder, Sec. 2): a relative threshold on the accumulator's
 * global maximum, then iterative extraction with neighbourhood suppression. A cell qualifies
 * iff acc >= threshold and acc * rel_den >= rel_num * max(acc) (the fraction rel_num/rel_den
 * of the maximum, compared exactly in integers). Repeatedly: the qualifying cell that is not
 * yet suppressed with the most votes (ties: the first in raster order) becomes the next peak,
 * and every cell within nms_radius of it in theta and in rho is suppressed, itself included.
 * theta wraps as in step 5: column j + dj outside [0, N_theta) is column j + dj -+ N_theta with
 * rho mirrored (k -> N_rho-1-k); rows outside [0, N_rho) are skipped. Peaks are listed in
 * extraction order, at most max_peaks stored; returns the true count. */
int32_t or_peaks_iterative(const int16_t* acc, const or_params* p, or_peak* out) {
  const int32_t NT = p->n_theta, NR = p->n_rho, R = p->nms_radius;
  const int64_t ncell = (int64_t)NT * NR;
  uint8_t* gone = (uint8_t*)calloc((size_t)(ncell > 0 ? ncell : 1), 1);
  int32_t amax = 0;
  for (int64_t c = 0; c < ncell; ++c)
    if (acc[c] > amax) amax = acc[c];
  int32_t n = 0;
  for (;;) {
    int64_t best = -1;
    int32_t bv = 0;
    for (int64_t c = 0; c < ncell; ++c) {
      const int32_t a = acc[c];
      if (gone[c] || a < p->threshold || (int64_t)a * p->rel_den < (int64_t)p->rel_num * amax) continue;
      if (best < 0 || a > bv) {
        best = c;
        bv = a;
      }
    }
    if (best < 0) break;
    const int32_t j = (int32_t)(best / NR), k = (int32_t)(best % NR);
    if (n < p->max_peaks) {
      out[n].theta_bin = (int16_t)j;
      out[n].rho_bin = (int16_t)k;
      out[n].votes = (int16_t)bv;
      out[n].flags = 0;
    }
    ++n;
    for (int32_t dj = -R; dj <= R; ++dj) {
      for (int32_t dk = -R; dk <= R; ++dk) {
        int32_t jj = j + dj, kk = k + dk;
        if (kk < 0 || kk >= NR) continue;
        if (jj < 0) {
          jj += NT;
          kk = NR - 1 - kk;
        } else if (jj >= NT) {
          jj -= NT;
          kk = NR - 1 - kk;
        }
        gone[(int64_t)jj * NR + kk] = 1;
      }
    }
  }
  free(gone);
  return n;
}

static uint64_t or_mix64(uint64_t z) { /* SplitMix64 finaliser (Steele, Lea, Flood 2014) */
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Order-free accumulator fingerprint: sum over cells c = j N_rho + k of acc[c] * mix64(c + 1), mod 2^64. */
uint64_t or_checksum(const int16_t* acc, int32_t n_theta, int32_t n_rho) {
  uint64_t h = 0;
  for (int64_t c = 0; c < (int64_t)n_theta * n_rho; ++c) h += (uint64_t)(int64_t)acc[c] * or_mix64((uint64_t)c + 1);
  return h;
}

/* One event: hits xy[2n]. acc [n_theta*n_rho] is scratch/output (required). Returns status flags. */
int32_t or_event(const int32_t* xy, int64_t n, const or_params* p, int16_t* acc, int32_t* npeaks, or_peak* peaks,
                 uint8_t* mask, int32_t* nkept, uint64_t* checksum) {
  const int32_t NT = p->n_theta, NR = p->n_rho;
  int32_t status = 0;
  memset(acc, 0, sizeof(int16_t) * (size_t)NT * NR);
  for (int64_t i = 0; i < n; ++i) mask[i] = 0;
  *npeaks = 0;
  *nkept = 0;
  if (n > OR_MAX_EVENT_HITS) {
    if (checksum) *checksum = 0;
    return OR_F_EVENT_TOO_LARGE;
  }
  int16_t* c = (int16_t*)malloc(sizeof(int16_t) * NT);
  int16_t* s = (int16_t*)malloc(sizeof(int16_t) * NT);
  int64_t* uq = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int64_t* vq = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  uint8_t* ok = (uint8_t*)malloc(n > 0 ? n : 1);
  or_tables(NT, c, s);
  for (int64_t i = 0; i < n; ++i) {
    int32_t f = or_map_hit(xy[2 * i], xy[2 * i + 1], &uq[i], &vq[i]);
    ok[i] = (f == 0);
    status |= f;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!ok[i]) continue;
    for (int32_t j = 0; j < NT; ++j) {
      int32_t k = or_bin(or_rho(uq[i], vq[i], c[j], s[j]), NR);
      acc[(int64_t)j * NR + k] += 1;
    }
  }
  if (checksum) *checksum = or_checksum(acc, NT, NR);
  int32_t np = p->peak_mode == 1 ? or_peaks_iterative(acc, p, peaks) : or_peaks(acc, p, peaks);
  *npeaks = np;
  if (np > p->max_peaks) status |= OR_F_PEAK_OVERFLOW;
  int32_t stored = np < p->max_peaks ? np : p->max_peaks;
  int32_t kept = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!ok[i]) continue;
    for (int32_t q = 0; q < stored; ++q) {
      int32_t j = peaks[q].theta_bin;
      int32_t k = or_bin(or_rho(uq[i], vq[i], c[j], s[j]), NR);
      int32_t d = k - peaks[q].rho_bin;
      if (d < 0) d = -d;
      if (d <= p->keep_halfwidth) {
        mask[i] = 1;
        break;
      }
    }
    kept += mask[i];
  }
  *nkept = kept;
  free(c);
  free(s);
  free(uq);
  free(vq);
  free(ok);
  return status;
}

/* ---- batch driver: events split over threads, same per-event code ---- */
typedef struct or_job {
  const int32_t* xy;
  const int64_t* off;
  const or_params* p;
  int16_t* acc; /* n_events * NT * NR, or NULL */
  int32_t* npeaks;
  or_peak* peaks; /* n_events * max_peaks */
  uint8_t* mask;
  int32_t* nkept;
  uint64_t* checksum; /* or NULL */
  int64_t begin, end;
  int32_t status;
} or_job;

static void* or_worker(void* arg) {
  or_job* jb = (or_job*)arg;
  const or_params* p = jb->p;
  size_t cells = (size_t)p->n_theta * p->n_rho;
  int16_t* scratch = jb->acc ? NULL : (int16_t*)malloc(sizeof(int16_t) * cells);
  or_peak* pk = (or_peak*)malloc(sizeof(or_peak) * (size_t)(p->max_peaks > 0 ? p->max_peaks : 1));
  for (int64_t e = jb->begin; e < jb->end; ++e) {
    int64_t a = jb->off[e], n = jb->off[e + 1] - a;
    int16_t* acc = jb->acc ? jb->acc + (size_t)e * cells : scratch;
    uint64_t cs = 0;
    jb->status |= or_event(jb->xy + 2 * a, n, p, acc, &jb->npeaks[e], pk, jb->mask + a, &jb->nkept[e],
                           jb->checksum ? &cs : NULL);
    if (jb->checksum) jb->checksum[e] = cs;
    int32_t stored = jb->npeaks[e] < p->max_peaks ? jb->npeaks[e] : p->max_peaks;
    or_peak* dst = jb->peaks + (size_t)e * p->max_peaks;
    memcpy(dst, pk, sizeof(or_peak) * (size_t)stored);
    memset(dst + stored, 0, sizeof(or_peak) * (size_t)(p->max_peaks - stored));
  }
  free(scratch);
  free(pk);
  return NULL;
}

/* Whole batch. Offsets must satisfy off[0] = 0 <= off[1] <= ... <= off[n_events] = n_hits, else
 * OR_F_BAD_OFFSETS is returned and nothing is computed. Returns the OR of all status flags. */
int32_t or_run(const int32_t* xy, int64_t n_hits, const int64_t* off, int64_t n_events, const or_params* p,
               int16_t* acc, int32_t* npeaks, or_peak* peaks, uint8_t* mask, int32_t* nkept, uint64_t* checksum,
               int32_t n_threads) {
  if (off[0] != 0 || off[n_events] != n_hits) return OR_F_BAD_OFFSETS;
  for (int64_t e = 0; e < n_events; ++e)
    if (off[e + 1] < off[e]) return OR_F_BAD_OFFSETS;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 512) n_threads = 512;
  if (n_events < n_threads) n_threads = (int32_t)(n_events > 0 ? n_events : 1);
  or_job jobs[512];
  pthread_t th[512];
  for (int32_t t = 0; t < n_threads; ++t) {
    or_job j = {xy, off, p, acc, npeaks, peaks, mask, nkept, checksum, n_events * t / n_threads,
                n_events * (t + 1) / n_threads, 0};
    jobs[t] = j;
  }
  for (int32_t t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, or_worker, &jobs[t]);
  or_worker(&jobs[0]);
  int32_t status = jobs[0].status;
  for (int32_t t = 1; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    status |= jobs[t].status;
  }
  return status;
}

int64_t or_const_H(void) { return OR_H; }

/* Step 7 (Eq. 2, circle recovery): the circle through the origin that peak (j, k) stands for,
 * taken at the bin centres th = (j + 1/2) pi / N_theta and rho = (-1 + (2k + 1) / N_rho) * 0.01
 * mm^-1: centre x_c = cos(th) / rho, y_c = sin(th) / rho (mm), radius r_c = 1 / |rho| (mm), and
 * the transverse momentum pT = 0.3 * B * r_c (MeV/c for B in tesla and r_c in mm; the 0.3 of the
 * usual pT [GeV/c] = 0.3 B [T] R [m], the convention the synthetic events are drawn with).
 * out[4 * q + 0..3] = x_c, y_c, r_c, pT for the n stored peaks of one event. */
void or_circles(const or_peak* pk, int32_t n, int32_t n_theta, int32_t n_rho, double b_tesla, double* out) {
  for (int32_t q = 0; q < n; ++q) {
    const double th = ((double)pk[q].theta_bin + 0.5) * OR_PI / (double)n_theta;
    const double rho = (-1.0 + (2.0 * (double)pk[q].rho_bin + 1.0) / (double)n_rho) * 0.01;
    out[4 * q + 0] = cos(th) / rho;
    out[4 * q + 1] = sin(th) / rho;
    out[4 * q + 2] = 1.0 / fabs(rho);
    out[4 * q + 3] = 0.3 * b_tesla * (1.0 / fabs(rho));
  }
}
