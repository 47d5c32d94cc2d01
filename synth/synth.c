/*
 * Seeded synthetic sensor data: analytic scenes rendered into pinhole depth/RGB frames and spinning-LiDAR scans.
 *
 * This file is an input producer only. It shares nothing with the fusion method: it renders ground-truth ranges of
 * boxes, spheres and planes, adds seeded noise, and writes plain arrays. Both the CPU oracle and the CUDA library
 * consume its output.
 *
 * Randomness is counter-based: every random number is splitmix64 of (seed, frame, element, stream), so the output does
 * not depend on thread count or scheduling. Normal deviates use the Box-Muller transform.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------ random numbers */

static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t mix4(uint64_t seed, uint64_t frame, uint64_t elem, uint64_t stream) {
  uint64_t h = splitmix64(seed);
  h = splitmix64(h ^ frame);
  h = splitmix64(h ^ elem);
  return splitmix64(h ^ stream);
}

/* uniform in (0, 1] */
static double uniform01(uint64_t seed, uint64_t frame, uint64_t elem, uint64_t stream) {
  return ((double)(mix4(seed, frame, elem, stream) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

static double normal01(uint64_t seed, uint64_t frame, uint64_t elem) {
  double u1 = uniform01(seed, frame, elem, 1);
  double u2 = uniform01(seed, frame, elem, 2);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ------------------------------------------------------------------------------------------------ scene */

/* Primitive kinds. ROOM: the ray is inside an axis-aligned box and hits where it leaves it. BOX: solid axis-aligned
 * box seen from outside. SPHERE: solid sphere. GROUND: the plane z = 0 seen from above. */
enum { PRIM_ROOM = 0, PRIM_BOX = 1, PRIM_SPHERE = 2, PRIM_GROUND = 3 };

/* One primitive = 14 doubles: kind, p[0..5] (box lo/hi or sphere centre+radius), colour A rgb, colour B rgb (0..255),
 * checker_period (metres, 0 = plain colour A). */
#define PRIM_STRIDE 14

typedef struct {
  const double* prims;
  int n_prims;
} scene_t;

/* Nearest hit of the ray o + s*d, s > s_min. Returns the primitive index or -1; *s_out receives s. */
static int ray_hit(const scene_t* sc, const double o[3], const double d[3], double s_min, double* s_out) {
  double best = INFINITY;
  int best_i = -1;
  for (int i = 0; i < sc->n_prims; ++i) {
    const double* p = sc->prims + (size_t)i * PRIM_STRIDE;
    int kind = (int)p[0];
    double s = INFINITY;
    if (kind == PRIM_ROOM || kind == PRIM_BOX) {
      double t_enter = -INFINITY, t_exit = INFINITY;
      int miss = 0;
      for (int a = 0; a < 3; ++a) {
        double lo = p[1 + a], hi = p[4 + a];
        if (d[a] == 0.0) {
          if (o[a] < lo || o[a] > hi) miss = 1;
          continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t_enter) t_enter = ta;
        if (tb < t_exit) t_exit = tb;
      }
      if (miss || t_enter > t_exit) continue;
      s = (kind == PRIM_ROOM) ? t_exit : t_enter;
    } else if (kind == PRIM_SPHERE) {
      double oc[3] = {o[0] - p[1], o[1] - p[2], o[2] - p[3]};
      double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double b = 2.0 * (d[0] * oc[0] + d[1] * oc[1] + d[2] * oc[2]);
      double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - p[4] * p[4];
      double disc = b * b - 4.0 * a * c;
      if (disc < 0.0) continue;
      s = (-b - sqrt(disc)) / (2.0 * a);
    } else if (kind == PRIM_GROUND) {
      if (d[2] >= 0.0) continue;
      s = -o[2] / d[2];
    }
    if (s > s_min && s < best) {
      best = s;
      best_i = i;
    }
  }
  *s_out = best;
  return best_i;
}

static void prim_colour(const double* p, const double x[3], uint8_t rgb[3]) {
  const double* col = p + 7;
  double period = p[13];
  if (period > 0.0) {
    long k = (long)floor(x[0] / period) + (long)floor(x[1] / period) + (long)floor(x[2] / period);
    if (k & 1) col = p + 10;
  }
  for (int c = 0; c < 3; ++c) rgb[c] = (uint8_t)col[c];
}

/* ------------------------------------------------------------------------------------------------ pinhole frames */

typedef struct {
  scene_t sc;
  int width, height;
  double fx, fy, cx, cy;
  double T[16]; /* world <- camera, row-major 4x4 */
  double noise_coef; /* depth noise sigma = noise_coef * z^2 */
  double dropout;    /* probability that a pixel reads 0 */
  uint64_t seed, frame;
  float* depth;
  uint8_t* rgb;
  int row0, row1;
} depth_job_t;

static void* depth_worker(void* arg) {
  depth_job_t* j = (depth_job_t*)arg;
  for (int v = j->row0; v < j->row1; ++v) {
    for (int u = 0; u < j->width; ++u) {
      size_t pix = (size_t)v * j->width + u;
      /* camera ray with unit z component, so the hit parameter is the z-depth */
      double qc[3] = {((double)u - j->cx) / j->fx, ((double)v - j->cy) / j->fy, 1.0};
      double d[3], o[3] = {j->T[3], j->T[7], j->T[11]};
      for (int r = 0; r < 3; ++r) d[r] = j->T[4 * r + 0] * qc[0] + j->T[4 * r + 1] * qc[1] + j->T[4 * r + 2] * qc[2];
      double s;
      int hit = ray_hit(&j->sc, o, d, 1e-9, &s);
      float z = 0.0f;
      uint8_t col[3] = {0, 0, 0};
      if (hit >= 0) {
        double x[3] = {o[0] + s * d[0], o[1] + s * d[1], o[2] + s * d[2]};
        prim_colour(j->sc.prims + (size_t)hit * PRIM_STRIDE, x, col);
        double zn = s;
        if (j->noise_coef > 0.0) zn += j->noise_coef * s * s * normal01(j->seed, j->frame, pix);
        if (j->dropout > 0.0 && uniform01(j->seed, j->frame, pix, 3) <= j->dropout) zn = 0.0;
        z = (float)zn;
      }
      if (j->depth) j->depth[pix] = z;
      if (j->rgb) memcpy(j->rgb + 3 * pix, col, 3);
    }
  }
  return NULL;
}

/* Render one pinhole frame. depth: H*W float32 z-depth in metres (0 = no return). rgb: H*W*3 uint8 or NULL. */
int synth_render_depth(const double* prims, int n_prims, int width, int height, double fx, double fy, double cx,
                       double cy, const double* T_wc, double noise_coef, double dropout, uint64_t seed, uint64_t frame,
                       float* depth, uint8_t* rgb, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  depth_job_t jobs[256];
  int created[256] = {0};
  int rows_per = (height + n_threads - 1) / n_threads;
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    depth_job_t* j = &jobs[t];
    j->sc.prims = prims;
    j->sc.n_prims = n_prims;
    j->width = width;
    j->height = height;
    j->fx = fx; j->fy = fy; j->cx = cx; j->cy = cy;
    memcpy(j->T, T_wc, sizeof(j->T));
    j->noise_coef = noise_coef;
    j->dropout = dropout;
    j->seed = seed;
    j->frame = frame;
    j->depth = depth;
    j->rgb = rgb;
    j->row0 = t * rows_per;
    j->row1 = j->row0 + rows_per > height ? height : j->row0 + rows_per;
    if (j->row0 >= j->row1) break;
    created[t] = pthread_create(&th[t], NULL, depth_worker, j) == 0;
    if (!created[t]) depth_worker(j);
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (created[t]) pthread_join(th[t], NULL);
  return 0;
}

/* ------------------------------------------------------------------------------------------------ LiDAR scans */

typedef struct {
  scene_t sc;
  int n_beams, n_azimuth;
  double elev_min, elev_max; /* radians */
  double T[16];              /* world <- sensor */
  double range_noise, r_min, r_max;
  uint64_t seed, frame;
  float* xyz;
  int col0, col1;
} lidar_job_t;

static void* lidar_worker(void* arg) {
  lidar_job_t* j = (lidar_job_t*)arg;
  for (int a = j->col0; a < j->col1; ++a) {
    double az = 6.283185307179586 * (double)a / (double)j->n_azimuth;
    for (int b = 0; b < j->n_beams; ++b) {
      size_t idx = (size_t)a * j->n_beams + b; /* column-major: all beams of one azimuth are consecutive */
      double el = j->n_beams > 1 ? j->elev_min + (j->elev_max - j->elev_min) * (double)b / (double)(j->n_beams - 1)
                                 : j->elev_min;
      double ds[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
      double d[3], o[3] = {j->T[3], j->T[7], j->T[11]};
      for (int r = 0; r < 3; ++r) d[r] = j->T[4 * r + 0] * ds[0] + j->T[4 * r + 1] * ds[1] + j->T[4 * r + 2] * ds[2];
      double s;
      int hit = ray_hit(&j->sc, o, d, 1e-9, &s);
      float* out = j->xyz + 3 * idx;
      if (hit < 0) {
        out[0] = out[1] = out[2] = NAN;
        continue;
      }
      double r = s + j->range_noise * normal01(j->seed, j->frame, idx);
      if (!(r >= j->r_min && r <= j->r_max)) {
        out[0] = out[1] = out[2] = NAN;
        continue;
      }
      out[0] = (float)(r * ds[0]);
      out[1] = (float)(r * ds[1]);
      out[2] = (float)(r * ds[2]);
    }
  }
  return NULL;
}

/* Render one spinning-LiDAR scan into xyz (n_beams*n_azimuth x 3 float32, sensor frame; NaN = no return).
 * Point index = azimuth * n_beams + beam. Directions are unit vectors in the sensor frame (x forward, z up). */
int synth_render_lidar(const double* prims, int n_prims, int n_beams, int n_azimuth, double elev_min_deg,
                       double elev_max_deg, const double* T_ws, double range_noise, double r_min, double r_max,
                       uint64_t seed, uint64_t frame, float* xyz, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  lidar_job_t jobs[256];
  int created[256] = {0};
  int cols_per = (n_azimuth + n_threads - 1) / n_threads;
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    lidar_job_t* j = &jobs[t];
    j->sc.prims = prims;
    j->sc.n_prims = n_prims;
    j->n_beams = n_beams;
    j->n_azimuth = n_azimuth;
    j->elev_min = elev_min_deg * 0.017453292519943295;
    j->elev_max = elev_max_deg * 0.017453292519943295;
    memcpy(j->T, T_ws, sizeof(j->T));
    j->range_noise = range_noise;
    j->r_min = r_min;
    j->r_max = r_max;
    j->seed = seed;
    j->frame = frame;
    j->xyz = xyz;
    j->col0 = t * cols_per;
    j->col1 = j->col0 + cols_per > n_azimuth ? n_azimuth : j->col0 + cols_per;
    if (j->col0 >= j->col1) break;
    created[t] = pthread_create(&th[t], NULL, lidar_worker, j) == 0;
    if (!created[t]) lidar_worker(j);
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (created[t]) pthread_join(th[t], NULL);
  return 0;
}
