/*
 * Seeded synthetic 2D drift-chamber events (input generator only).
 *
 * Stands in for the simulated STCF MDC samples of the paper's Sec. 4, which are
 * not available here. It holds none of the Hough method's arithmetic: it only
 * places hits. Both the CUDA path and the CPU oracle consume its output.
 *
 * Geometry: 48 axial layers at r_l = 200 + 13 l mm with n_l = 128 + 4 l cells,
 * wire l,k at phi = 2 pi (k + 1/2) / n_l, wire coordinates rounded to integer um.
 * A track from the origin with transverse momentum pT [MeV/c] in a 1 T field is
 * a circle of radius R = pT / 0.3 mm through the origin, centred at azimuth
 * phi_c = phi0 - q pi/2. It crosses layer l (if r_l <= 2R) at
 * phi_c + q acos(r_l / 2R) on the way out; a track with 2R < r_47 curls and
 * also crosses every layer it reaches at phi_c - q acos(r_l / 2R) on the way
 * back (further turns repeat the same cells). A hit is the wire of the crossed
 * cell. Noise is an independent Bernoulli(occupancy) draw per cell. Cells are
 * de-duplicated; a track label beats a noise label and the lower track index
 * beats a higher one. Hits are emitted in (layer, cell) order.
 *
 * Random numbers come from a counter-based SplitMix64-style hash keyed by
 * (seed, event, stream, counter), so any event can be regenerated alone.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HG_LAYERS 48
#define HG_CELLS 10656
#define HG_MAX_TRACKS 64
#define HG_STREAM_EVENT 0u
#define HG_STREAM_NOISE 0xFFFFu

typedef struct hg_config {
  uint64_t seed;
  int32_t tracks_mode; /* 0 fixed tracks_a; 1 uniform int [tracks_a, tracks_b]; 2 Poisson(tracks_mean) capped at tracks_b */
  int32_t tracks_a;
  int32_t tracks_b;
  int32_t pt_mode; /* 0 uniform [pt_a,pt_b]; 1 log-uniform [pt_a,pt_b]; 2 with prob pt_frac log-uniform [pt_a2,pt_b2] else log-uniform [pt_a,pt_b] */
  double tracks_mean;
  double pt_a, pt_b, pt_frac, pt_a2, pt_b2;
  int32_t noise_mode; /* 0 fixed noise_a; 1 uniform [noise_a, noise_b] per event */
  int32_t reserved;
  double noise_a, noise_b;
} hg_config;

static const double HG_PI = 3.14159265358979323846;

static inline uint64_t hg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static inline uint64_t hg_key(uint64_t seed, uint64_t event, uint64_t stream) {
  uint64_t k = hg_mix64(seed ^ hg_mix64(event * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL));
  return hg_mix64(k ^ (stream * 0xD6E8FEB86659FD93ULL + 0x2545F4914F6CDD1DULL));
}

static inline double hg_unif(uint64_t key, uint64_t ctr) {
  uint64_t x = hg_mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- geometry ---- */
static int32_t g_layer_first[HG_LAYERS + 1];
static int32_t g_wire_x[HG_CELLS], g_wire_y[HG_CELLS];
static pthread_once_t g_geom_once = PTHREAD_ONCE_INIT;

static void hg_init_geometry(void) {
  int32_t c = 0;
  for (int l = 0; l < HG_LAYERS; ++l) {
    int n = 128 + 4 * l;
    double r_um = 1000.0 * (200.0 + 13.0 * l);
    g_layer_first[l] = c;
    for (int k = 0; k < n; ++k, ++c) {
      double phi = 2.0 * HG_PI * (k + 0.5) / n;
      g_wire_x[c] = (int32_t)llround(r_um * cos(phi));
      g_wire_y[c] = (int32_t)llround(r_um * sin(phi));
    }
  }
  g_layer_first[HG_LAYERS] = c;
}

static inline int hg_cell_of(int l, double phi) {
  int n = 128 + 4 * l;
  double t = fmod(phi, 2.0 * HG_PI);
  if (t < 0) t += 2.0 * HG_PI;
  int k = (int)floor(t * n / (2.0 * HG_PI));
  if (k >= n) k = n - 1;
  if (k < 0) k = 0;
  return g_layer_first[l] + k;
}

typedef struct hg_track {
  double pt;
  double phi0;
  int32_t q;
} hg_track;

static double hg_loguniform(double u, double a, double b) { return exp(log(a) + u * (log(b) - log(a))); }

/* Draws the tracks of one event; returns how many. */
static int hg_draw_tracks(const hg_config* cfg, uint64_t ev, hg_track* tr) {
  uint64_t ke = hg_key(cfg->seed, ev, HG_STREAM_EVENT);
  int n = 0;
  if (cfg->tracks_mode == 0) {
    n = cfg->tracks_a;
  } else if (cfg->tracks_mode == 1) {
    int span = cfg->tracks_b - cfg->tracks_a + 1;
    n = cfg->tracks_a + (int)floor(hg_unif(ke, 0) * span);
    if (n > cfg->tracks_b) n = cfg->tracks_b;
  } else {
    double u = hg_unif(ke, 0);
    double p = exp(-cfg->tracks_mean), F = p;
    while (u > F && n < cfg->tracks_b) {
      ++n;
      p *= cfg->tracks_mean / n;
      F += p;
    }
  }
  if (n > HG_MAX_TRACKS) n = HG_MAX_TRACKS;
  if (n < 0) n = 0;
  for (int t = 0; t < n; ++t) {
    uint64_t kt = hg_key(cfg->seed, ev, 1 + (uint64_t)t);
    double u_pt = hg_unif(kt, 0), u_q = hg_unif(kt, 1), u_phi = hg_unif(kt, 2), u_mix = hg_unif(kt, 3);
    double pt;
    if (cfg->pt_mode == 0)
      pt = cfg->pt_a + u_pt * (cfg->pt_b - cfg->pt_a);
    else if (cfg->pt_mode == 1)
      pt = hg_loguniform(u_pt, cfg->pt_a, cfg->pt_b);
    else
      pt = (u_mix < cfg->pt_frac) ? hg_loguniform(u_pt, cfg->pt_a2, cfg->pt_b2) : hg_loguniform(u_pt, cfg->pt_a, cfg->pt_b);
    tr[t].pt = pt;
    tr[t].q = (u_q < 0.5) ? 1 : -1;
    tr[t].phi0 = 2.0 * HG_PI * u_phi;
  }
  return n;
}

static double hg_event_noise(const hg_config* cfg, uint64_t ev) {
  if (cfg->noise_mode == 0) return cfg->noise_a;
  uint64_t ke = hg_key(cfg->seed, ev, HG_STREAM_EVENT);
  return cfg->noise_a + hg_unif(ke, 1) * (cfg->noise_b - cfg->noise_a);
}

/* Fills label[HG_CELLS]: -2 empty, -1 noise, t >= 0 track t. */
static void hg_event_labels(const hg_config* cfg, uint64_t ev, int32_t* label) {
  hg_track tr[HG_MAX_TRACKS];
  int nt = hg_draw_tracks(cfg, ev, tr);
  for (int c = 0; c < HG_CELLS; ++c) label[c] = -2;
  const double r_last = 200.0 + 13.0 * (HG_LAYERS - 1);
  for (int t = 0; t < nt; ++t) {
    double R = tr[t].pt / 0.3;
    double phic = tr[t].phi0 - tr[t].q * 0.5 * HG_PI;
    int curls = (2.0 * R < r_last);
    for (int l = 0; l < HG_LAYERS; ++l) {
      double r = 200.0 + 13.0 * l;
      if (r > 2.0 * R) break;
      double a = acos(r / (2.0 * R));
      int c1 = hg_cell_of(l, phic + tr[t].q * a);
      if (label[c1] < 0) label[c1] = t;
      if (curls) {
        int c2 = hg_cell_of(l, phic - tr[t].q * a);
        if (label[c2] < 0) label[c2] = t;
      }
    }
  }
  double occ = hg_event_noise(cfg, ev);
  uint64_t kn = hg_key(cfg->seed, ev, HG_STREAM_NOISE);
  for (int c = 0; c < HG_CELLS; ++c) {
    double u = hg_unif(kn, (uint64_t)c);
    if (u < occ && label[c] == -2) label[c] = -1;
  }
}

/* ---- threaded drivers ---- */
typedef struct hg_job {
  const hg_config* cfg;
  int64_t ev0, begin, end;
  int64_t* counts;
  const int64_t* off;
  int32_t* xy;
  int32_t* truth;
} hg_job;

static void* hg_count_worker(void* arg) {
  hg_job* j = (hg_job*)arg;
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * HG_CELLS);
  for (int64_t e = j->begin; e < j->end; ++e) {
    hg_event_labels(j->cfg, (uint64_t)(j->ev0 + e), label);
    int64_t n = 0;
    for (int c = 0; c < HG_CELLS; ++c) n += (label[c] != -2);
    j->counts[e] = n;
  }
  free(label);
  return NULL;
}

static void* hg_fill_worker(void* arg) {
  hg_job* j = (hg_job*)arg;
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * HG_CELLS);
  int64_t base = j->off[0];
  for (int64_t e = j->begin; e < j->end; ++e) {
    hg_event_labels(j->cfg, (uint64_t)(j->ev0 + e), label);
    int64_t w = j->off[e] - base, stop = j->off[e + 1] - base;
    for (int c = 0; c < HG_CELLS && w < stop; ++c) {
      if (label[c] == -2) continue;
      j->xy[2 * w] = g_wire_x[c];
      j->xy[2 * w + 1] = g_wire_y[c];
      if (j->truth) j->truth[w] = label[c];
      ++w;
    }
  }
  free(label);
  return NULL;
}

static int hg_run(void* (*fn)(void*), hg_job proto, int64_t n_events, int n_threads) {
  pthread_once(&g_geom_once, hg_init_geometry);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_events < n_threads) n_threads = (int)(n_events > 0 ? n_events : 1);
  hg_job jobs[256];
  pthread_t th[256];
  for (int i = 0; i < n_threads; ++i) {
    jobs[i] = proto;
    jobs[i].begin = n_events * i / n_threads;
    jobs[i].end = n_events * (i + 1) / n_threads;
  }
  for (int i = 1; i < n_threads; ++i)
    if (pthread_create(&th[i], NULL, fn, &jobs[i]) != 0) return -1;
  fn(&jobs[0]);
  for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
  return 0;
}

/* Hit count of events [ev0, ev0 + n_events) into counts[n_events]. */
int hg_count(const hg_config* cfg, int64_t ev0, int64_t n_events, int64_t* counts, int n_threads) {
  hg_job p = {cfg, ev0, 0, 0, counts, NULL, NULL, NULL};
  return hg_run(hg_count_worker, p, n_events, n_threads);
}

/* Hits of events [ev0, ev0 + n_events): event e fills rows [off[e]-off[0], off[e+1]-off[0])
 * of xy (int32 (x, y) pairs in um) and truth (track index, or -1 for noise; may be NULL). */
int hg_fill(const hg_config* cfg, int64_t ev0, int64_t n_events, const int64_t* off, int32_t* xy, int32_t* truth,
            int n_threads) {
  hg_job p = {cfg, ev0, 0, 0, NULL, off, xy, truth};
  return hg_run(hg_fill_worker, p, n_events, n_threads);
}

/* Truth tracks of one event: returns the count (<= cap written). */
int hg_event_tracks(const hg_config* cfg, int64_t ev, double* pt, int32_t* q, double* phi0, int cap) {
  hg_track tr[HG_MAX_TRACKS];
  int n = hg_draw_tracks(cfg, (uint64_t)ev, tr);
  for (int t = 0; t < n && t < cap; ++t) {
    pt[t] = tr[t].pt;
    q[t] = tr[t].q;
    phi0[t] = tr[t].phi0;
  }
  return n;
}

/* Wire table (HG_CELLS entries) and per-layer first-cell index (HG_LAYERS + 1 entries). */
int hg_geometry(int32_t* wire_x, int32_t* wire_y, int32_t* layer_first) {
  pthread_once(&g_geom_once, hg_init_geometry);
  if (wire_x) memcpy(wire_x, g_wire_x, sizeof g_wire_x);
  if (wire_y) memcpy(wire_y, g_wire_y, sizeof g_wire_y);
  if (layer_first) memcpy(layer_first, g_layer_first, sizeof g_layer_first);
  return HG_CELLS;
}
