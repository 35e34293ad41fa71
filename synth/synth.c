/*
 * Seeded synthetic scenes, trajectories and sensor images.
 *
 * This module produces INPUTS only: analytic scenes (inward room box, solid
 * boxes, spheres, vertical cylinders, planes), camera / LiDAR poses on a
 * smooth spline, and depth / range images made by exact FP64 ray casting with
 * a counter-based noise model.  It holds none of the integration method's
 * arithmetic and is shared by the oracle tests and by the CUDA path's tests
 * and benchmark, which each do their own processing of what it returns.
 *
 * Sensor models follow the paper's problem statement (Sec. III): a depth
 * image D: Omega -> d where Omega is the pinhole image plane (z-depth per
 * pixel) or the LiDAR beam angles (range per beam).
 *
 * Pixel-centre convention: pixel (i, j) has its centre at image coordinates
 * (u, v) = (i, j); its ray in the camera frame is ((i-cu)/fu, (j-cv)/fv, 1),
 * so the ray parameter at a hit is the z-depth.  LiDAR cell (k, j) covers
 * azimuth [theta_start + k/alpha, theta_start + (k+1)/alpha) and polar angle
 * [phi_start + j/beta, ...); its beam is cast through the cell centre.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based hash
 * of (seed, frame, pixel, stream); normals by the Box-Muller transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_ROOM 0     /* inward axis-aligned box: p[0..2] min, p[3..5] max */
#define SYN_BOX 1      /* solid axis-aligned box: p[0..2] min, p[3..5] max  */
#define SYN_SPHERE 2   /* p[0..2] centre, p[3] radius                       */
#define SYN_CYL 3      /* vertical capped cylinder: p[0],p[1] centre xy,
                          p[2] radius, p[3] z0, p[4] z1                      */
#define SYN_PLANE 4    /* p[0..2] unit normal n, p[3] offset: n.x = p[3]    */
#define SYN_NPAR 9     /* doubles per primitive: kind + 8 parameters        */

static const double kEps = 1e-9;

static uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* uniform in (0, 1) from a 64-bit hash */
static double u01(uint64_t h) { return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static uint64_t ctr_hash(uint64_t seed, uint64_t frame, uint64_t pixel, uint64_t stream) {
  return sm64(sm64(sm64(sm64(seed) ^ frame) ^ pixel) ^ stream);
}

static double ctr_normal(uint64_t seed, uint64_t frame, uint64_t pixel) {
  double a = u01(ctr_hash(seed, frame, pixel, 1));
  double b = u01(ctr_hash(seed, frame, pixel, 2));
  return sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
}

/* ---------------------------------------------------------------- ray cast */

static double hit_room(const double* p, const double o[3], const double d[3]) {
  double t = INFINITY;
  for (int k = 0; k < 3; ++k) {
    double tk = INFINITY;
    if (d[k] > 0) tk = (p[3 + k] - o[k]) / d[k];
    else if (d[k] < 0) tk = (p[k] - o[k]) / d[k];
    if (tk < t) t = tk;
  }
  return t > kEps ? t : INFINITY;
}

static double hit_box(const double* p, const double o[3], const double d[3]) {
  double tn = -INFINITY, tf = INFINITY;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) {
      if (o[k] < p[k] || o[k] > p[3 + k]) return INFINITY;
      continue;
    }
    double t1 = (p[k] - o[k]) / d[k], t2 = (p[3 + k] - o[k]) / d[k];
    if (t1 > t2) { double s = t1; t1 = t2; t2 = s; }
    if (t1 > tn) tn = t1;
    if (t2 < tf) tf = t2;
  }
  if (tn > tf || tf <= kEps) return INFINITY;
  return tn > kEps ? tn : INFINITY; /* origin inside a solid: ignore it */
}

/* smallest root > eps of a t^2 + 2 b t + c = 0, numerically stable form */
static double small_root(double a, double b, double c) {
  double disc = b * b - a * c;
  if (disc < 0 || a == 0) return INFINITY;
  double sq = sqrt(disc);
  double q = (b > 0) ? -(b + sq) : (-b + sq);
  double t0 = q / a, t1 = (q != 0) ? c / q : INFINITY;
  if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
  if (t0 > kEps) return t0;
  if (t1 > kEps) return INFINITY; /* origin inside the solid */
  return INFINITY;
}

static double hit_sphere(const double* p, const double o[3], const double d[3]) {
  double oc[3] = {o[0] - p[0], o[1] - p[1], o[2] - p[2]};
  double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
  double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - p[3] * p[3];
  return small_root(a, b, c);
}

static double hit_cyl(const double* p, const double o[3], const double d[3]) {
  double best = INFINITY;
  double ox = o[0] - p[0], oy = o[1] - p[1], r2 = p[2] * p[2];
  /* origin inside the solid: ignore it */
  if (ox * ox + oy * oy <= r2 && o[2] >= p[3] && o[2] <= p[4]) return INFINITY;
  double a = d[0] * d[0] + d[1] * d[1];
  if (a > 0) {
    double b = ox * d[0] + oy * d[1];
    double c = ox * ox + oy * oy - r2;
    double disc = b * b - a * c;
    if (disc >= 0) {
      double sq = sqrt(disc);
      double ts[2] = {(-b - sq) / a, (-b + sq) / a};
      for (int i = 0; i < 2; ++i) {
        double t = ts[i];
        if (t > kEps && t < best) {
          double z = o[2] + t * d[2];
          if (z >= p[3] && z <= p[4]) best = t;
        }
      }
    }
  }
  if (d[2] != 0) {
    double zc[2] = {p[3], p[4]};
    for (int i = 0; i < 2; ++i) {
      double t = (zc[i] - o[2]) / d[2];
      if (t > kEps && t < best) {
        double x = ox + t * d[0], y = oy + t * d[1];
        if (x * x + y * y <= r2) best = t;
      }
    }
  }
  return best;
}

static double hit_plane(const double* p, const double o[3], const double d[3]) {
  double den = p[0] * d[0] + p[1] * d[1] + p[2] * d[2];
  if (fabs(den) < 1e-15) return INFINITY;
  double t = (p[3] - (p[0] * o[0] + p[1] * o[1] + p[2] * o[2])) / den;
  return t > kEps ? t : INFINITY;
}

static double hit_prim(const double* q, const double o[3], const double d[3]) {
  const double* p = q + 1;
  switch ((int)q[0]) {
    case SYN_ROOM: return hit_room(p, o, d);
    case SYN_BOX: return hit_box(p, o, d);
    case SYN_SPHERE: return hit_sphere(p, o, d);
    case SYN_CYL: return hit_cyl(p, o, d);
    case SYN_PLANE: return hit_plane(p, o, d);
    default: return INFINITY;
  }
}

/* Bounding sphere of a bounded solid (boxes, spheres, cylinders): centre c,
 * squared radius; returns 0 for unbounded primitives (rooms, planes). */
static int bound(const double* q, double c[3], double* r2) {
  const double* p = q + 1;
  switch ((int)q[0]) {
    case SYN_BOX:
      for (int k = 0; k < 3; ++k) c[k] = 0.5 * (p[k] + p[3 + k]);
      *r2 = 0.25 * ((p[3] - p[0]) * (p[3] - p[0]) + (p[4] - p[1]) * (p[4] - p[1]) + (p[5] - p[2]) * (p[5] - p[2]));
      return 1;
    case SYN_SPHERE:
      c[0] = p[0]; c[1] = p[1]; c[2] = p[2];
      *r2 = p[3] * p[3];
      return 1;
    case SYN_CYL: {
      const double h = 0.5 * (p[4] - p[3]);
      c[0] = p[0]; c[1] = p[1]; c[2] = 0.5 * (p[3] + p[4]);
      *r2 = p[2] * p[2] + h * h;
      return 1;
    }
    default:
      return 0;
  }
}

/* First hit parameter t > 0 of o + t d against every primitive, or INFINITY.
 * Bounded solids whose bounding sphere the ray misses (or meets only beyond
 * the best hit so far) are skipped; the exact tests decide everything else. */
double synth_cast(const double* prims, int32_t n, const double o[3], const double d[3]) {
  double best = INFINITY;
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  for (int32_t i = 0; i < n; ++i) {
    const double* q = prims + (size_t)i * SYN_NPAR;
    const double* p = q + 1;
    double c[3], r2;
    if (bound(q, c, &r2)) {
      const double oc[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
      const double ocd = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
      const double oc2 = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2];
      if (oc2 > r2 * 1.0000001 + 1e-12) {  /* origin outside the sphere */
        if (ocd <= 0) continue;                                /* sphere behind the ray */
        if (oc2 - ocd * ocd / dd > r2 * 1.0000001 + 1e-12) continue;  /* ray misses it */
        const double tnear = (ocd - sqrt(r2 * dd)) / dd;       /* lower bound on any hit */
        if (tnear > best) continue;
      }
    }
    const double t = hit_prim(q, o, d);
    if (t < best) best = t;
  }
  return best;
}

/* --------------------------------------------------- 2D grid acceleration */

/* Uniform grid over the xy extent of the bounded solids: each cell lists the
 * solids whose xy bounding box (grown by 1e-6 m) overlaps it; rooms and
 * planes are tested for every ray.  A ray walks the cells its xy projection
 * crosses and stops once its best hit lies before the next cell; the exact
 * hit tests decide, so images equal those of the exhaustive caster. */
typedef struct {
  double x0, y0, cell;
  int nx, ny;
  int* start;   /* [nx*ny + 1] */
  int* items;
  int* unb;     /* unbounded primitives */
  int n_unb;
} grid2;

static int xy_box(const double* q, double b[4]) {
  const double* p = q + 1;
  switch ((int)q[0]) {
    case SYN_BOX: b[0] = p[0]; b[1] = p[1]; b[2] = p[3]; b[3] = p[4]; return 1;
    case SYN_SPHERE: b[0] = p[0] - p[3]; b[1] = p[1] - p[3]; b[2] = p[0] + p[3]; b[3] = p[1] + p[3]; return 1;
    case SYN_CYL: b[0] = p[0] - p[2]; b[1] = p[1] - p[2]; b[2] = p[0] + p[2]; b[3] = p[1] + p[2]; return 1;
    default: return 0;
  }
}

static void grid_free(grid2* g) {
  free(g->start);
  free(g->items);
  free(g->unb);
}

static int grid_build(grid2* g, const double* prims, int32_t n) {
  memset(g, 0, sizeof(*g));
  double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
  int nb = 0;
  g->unb = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) {
    double b[4];
    if (!xy_box(prims + (size_t)i * SYN_NPAR, b)) { g->unb[g->n_unb++] = i; continue; }
    ++nb;
    if (b[0] < lo[0]) lo[0] = b[0];
    if (b[1] < lo[1]) lo[1] = b[1];
    if (b[2] > hi[0]) hi[0] = b[2];
    if (b[3] > hi[1]) hi[1] = b[3];
  }
  if (nb == 0) { g->nx = g->ny = 0; g->start = NULL; g->items = NULL; return 0; }
  const double ext = fmax(hi[0] - lo[0], hi[1] - lo[1]);
  g->cell = fmax(ext / 48.0, 0.25);
  g->x0 = lo[0] - 1e-3;
  g->y0 = lo[1] - 1e-3;
  g->nx = (int)((hi[0] - g->x0) / g->cell) + 1;
  g->ny = (int)((hi[1] - g->y0) / g->cell) + 1;
  const int nc = g->nx * g->ny;
  g->start = (int*)calloc((size_t)nc + 1, sizeof(int));
  for (int pass = 0; pass < 2; ++pass) {
    int* fill = NULL;
    if (pass == 1) {
      for (int c = 0; c < nc; ++c) g->start[c + 1] += g->start[c];
      g->items = (int*)malloc(sizeof(int) * (g->start[nc] > 0 ? g->start[nc] : 1));
      fill = (int*)calloc((size_t)nc, sizeof(int));
    }
    for (int32_t i = 0; i < n; ++i) {
      double b[4];
      if (!xy_box(prims + (size_t)i * SYN_NPAR, b)) continue;
      int cx0 = (int)floor((b[0] - 1e-6 - g->x0) / g->cell), cx1 = (int)floor((b[2] + 1e-6 - g->x0) / g->cell);
      int cy0 = (int)floor((b[1] - 1e-6 - g->y0) / g->cell), cy1 = (int)floor((b[3] + 1e-6 - g->y0) / g->cell);
      if (cx0 < 0) cx0 = 0;
      if (cy0 < 0) cy0 = 0;
      if (cx1 >= g->nx) cx1 = g->nx - 1;
      if (cy1 >= g->ny) cy1 = g->ny - 1;
      for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) {
          const int c = cy * g->nx + cx;
          if (pass == 0) g->start[c + 1]++;
          else g->items[g->start[c] + fill[c]++] = i;
        }
    }
    free(fill);
  }
  return 1;
}

/* mark[i] == stamp: primitive i already tested for this ray */
static double grid_cast(const grid2* g, const double* prims, const double o[3], const double d[3],
                        int* mark, int stamp) {
  double best = INFINITY;
  for (int k = 0; k < g->n_unb; ++k) {
    const double t = hit_prim(prims + (size_t)g->unb[k] * SYN_NPAR, o, d);
    if (t < best) best = t;
  }
  if (g->nx == 0) return best;
  /* clip the ray's xy projection to the grid rectangle */
  double t0 = 0.0, t1 = INFINITY;
  const double lo[2] = {g->x0, g->y0}, hi[2] = {g->x0 + g->nx * g->cell, g->y0 + g->ny * g->cell};
  for (int k = 0; k < 2; ++k) {
    if (d[k] == 0.0) {
      if (o[k] < lo[k] || o[k] > hi[k]) return best;
      continue;
    }
    double a = (lo[k] - o[k]) / d[k], b = (hi[k] - o[k]) / d[k];
    if (a > b) { const double s = a; a = b; b = s; }
    if (a > t0) t0 = a;
    if (b < t1) t1 = b;
  }
  if (!(t0 <= t1) || t0 >= best) return best;
  const double px = o[0] + t0 * d[0], py = o[1] + t0 * d[1];
  int cx = (int)floor((px - g->x0) / g->cell), cy = (int)floor((py - g->y0) / g->cell);
  if (cx < 0) cx = 0;
  if (cx >= g->nx) cx = g->nx - 1;
  if (cy < 0) cy = 0;
  if (cy >= g->ny) cy = g->ny - 1;
  const int sx = d[0] > 0 ? 1 : (d[0] < 0 ? -1 : 0), sy = d[1] > 0 ? 1 : (d[1] < 0 ? -1 : 0);
  double tx = INFINITY, ty = INFINITY, dtx = INFINITY, dty = INFINITY;
  if (sx) { tx = (g->x0 + (cx + (sx > 0)) * g->cell - o[0]) / d[0]; dtx = g->cell / fabs(d[0]); }
  if (sy) { ty = (g->y0 + (cy + (sy > 0)) * g->cell - o[1]) / d[1]; dty = g->cell / fabs(d[1]); }
  for (;;) {
    const int c = cy * g->nx + cx;
    for (int k = g->start[c]; k < g->start[c + 1]; ++k) {
      const int i = g->items[k];
      if (mark[i] == stamp) continue;
      mark[i] = stamp;
      const double t = hit_prim(prims + (size_t)i * SYN_NPAR, o, d);
      if (t < best) best = t;
    }
    const double tn = tx < ty ? tx : ty;
    /* a hit before the next cell cannot be beaten by solids met later
       (their hits lie at or beyond the cell boundary, up to the 1e-6 margin) */
    if (best < tn - 1e-5 || tn > t1) break;
    if (tx < ty) { cx += sx; tx += dtx; } else { cy += sy; ty += dty; }
    if (cx < 0 || cx >= g->nx || cy < 0 || cy >= g->ny) break;
  }
  return best;
}

/* ------------------------------------------------------------- renderers */

/*
 * Pinhole z-depth image, row-major float32[H][W].  T is the camera-to-world
 * pose (row-major 4x4).  Noise: z += N(0,1) * sigma_z2 * z^2; then with
 * probability invalid_frac the pixel is set to 0; depths above max_depth (or
 * <= 0, or no hit) are written as 0 (invalid).
 */
void synth_render_pinhole(const double* prims, int32_t n, const double T[16], double fu, double fv,
                          double cu, double cv, int32_t W, int32_t H, double sigma_z2,
                          double invalid_frac, double max_depth, uint64_t seed, uint64_t frame,
                          float* out) {
  const double o[3] = {T[3], T[7], T[11]};
  grid2 g;
  grid_build(&g, prims, n);
#pragma omp parallel for schedule(dynamic, 4)
  for (int32_t j = 0; j < H; ++j) {
    int* mark = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    for (int32_t i = 0; i < W; ++i) {
      double rc[3] = {((double)i - cu) / fu, ((double)j - cv) / fv, 1.0};
      double dw[3];
      for (int k = 0; k < 3; ++k) dw[k] = T[4 * k + 0] * rc[0] + T[4 * k + 1] * rc[1] + T[4 * k + 2] * rc[2];
      double z = grid_cast(&g, prims, o, dw, mark, i + 1);
      uint64_t pix = (uint64_t)j * (uint64_t)W + (uint64_t)i;
      if (isfinite(z) && sigma_z2 > 0) z += ctr_normal(seed, frame, pix) * sigma_z2 * z * z;
      if (invalid_frac > 0 && u01(ctr_hash(seed, frame, pix, 3)) < invalid_frac) z = 0;
      if (!isfinite(z) || z <= 0 || z > max_depth) z = 0;
      out[pix] = (float)z;
    }
    free(mark);
  }
  grid_free(&g);
}

/*
 * Spherical LiDAR range image, row-major float32[n_el][n_az]; row 0 is the
 * smallest polar angle (topmost beam).  Beam (k, j) direction in the sensor
 * frame: theta = theta_start + (k+0.5)*2pi/n_az (azimuth about +z),
 * phi = phi_start + (j+0.5)*el_fov/n_el (polar angle from +z),
 * b = (sin phi cos theta, sin phi sin theta, cos phi).  Noise N(0, sigma);
 * ranges outside [min_range, max_range] are written as 0.
 */
void synth_render_lidar(const double* prims, int32_t n, const double T[16], int32_t n_az,
                        int32_t n_el, double theta_start, double phi_start, double el_fov,
                        double min_range, double max_range, double sigma, uint64_t seed,
                        uint64_t frame, float* out) {
  const double o[3] = {T[3], T[7], T[11]};
  grid2 g;
  grid_build(&g, prims, n);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < n_el; ++j) {
    double phi = phi_start + ((double)j + 0.5) * (el_fov / (double)n_el);
    int* mark = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    for (int32_t k = 0; k < n_az; ++k) {
      double th = theta_start + ((double)k + 0.5) * (6.283185307179586 / (double)n_az);
      double b[3] = {sin(phi) * cos(th), sin(phi) * sin(th), cos(phi)};
      double dw[3];
      for (int q = 0; q < 3; ++q) dw[q] = T[4 * q + 0] * b[0] + T[4 * q + 1] * b[1] + T[4 * q + 2] * b[2];
      double r = grid_cast(&g, prims, o, dw, mark, k + 1);
      uint64_t pix = (uint64_t)j * (uint64_t)n_az + (uint64_t)k;
      if (isfinite(r) && sigma > 0) r += ctr_normal(seed, frame, pix) * sigma;
      if (!isfinite(r) || r < min_range || r > max_range) r = 0;
      out[pix] = (float)r;
    }
    free(mark);
  }
  grid_free(&g);
}

/* ----------------------------------------------------------------- scenes */

typedef struct { uint64_t s; } rng_t;
static double rng_u(rng_t* r) { r->s += 0x9E3779B97F4A7C15ull; return u01(sm64(r->s)); }
static double rng_range(rng_t* r, double lo, double hi) { return lo + (hi - lo) * rng_u(r); }

static double* put(double* q, int kind, const double* p, int np) {
  memset(q, 0, sizeof(double) * SYN_NPAR);
  q[0] = kind;
  for (int i = 0; i < np; ++i) q[1 + i] = p[i];
  return q + SYN_NPAR;
}

/*
 * Room scene: inward box [0,sx]x[0,sy]x[0,sz], n_boxes solid boxes with edges
 * U[edge_lo, edge_hi] and centres uniform such that the box lies inside the
 * room, n_spheres spheres with radius U[r_lo, r_hi] inside the room.
 * Returns the number of primitives written (1 + n_boxes + n_spheres).
 */
int32_t synth_room_scene(uint64_t seed, double sx, double sy, double sz, int32_t n_boxes,
                         int32_t n_spheres, double edge_lo, double edge_hi, double r_lo,
                         double r_hi, double* out) {
  rng_t r = {sm64(seed ^ 0x526f6f6dull)};
  double* q = out;
  double room[6] = {0, 0, 0, sx, sy, sz};
  q = put(q, SYN_ROOM, room, 6);
  double dims[3] = {sx, sy, sz};
  for (int32_t b = 0; b < n_boxes; ++b) {
    double p[6];
    for (int k = 0; k < 3; ++k) {
      double e = rng_range(&r, edge_lo, edge_hi);
      if (e > dims[k]) e = dims[k];
      double c = rng_range(&r, 0.5 * e, dims[k] - 0.5 * e);
      p[k] = c - 0.5 * e;
      p[3 + k] = c + 0.5 * e;
    }
    q = put(q, SYN_BOX, p, 6);
  }
  for (int32_t s = 0; s < n_spheres; ++s) {
    double rad = rng_range(&r, r_lo, r_hi);
    double p[4];
    for (int k = 0; k < 3; ++k) p[k] = rng_range(&r, rad, dims[k] - rad);
    p[3] = rad;
    q = put(q, SYN_SPHERE, p, 4);
  }
  return 1 + n_boxes + n_spheres;
}

/*
 * Outdoor scene: ground plane z = 0 over [0,sx]x[0,sy], n_boxes boxes resting
 * on the ground (edges U[edge_lo, edge_hi], height capped at sz), n_cyl
 * vertical cylinders (radius U[r_lo, r_hi], height U[h_lo, h_hi]) on the
 * ground.  Returns the number of primitives.
 */
int32_t synth_outdoor_scene(uint64_t seed, double sx, double sy, double sz, int32_t n_boxes,
                            int32_t n_cyl, double edge_lo, double edge_hi, double r_lo,
                            double r_hi, double h_lo, double h_hi, double* out) {
  rng_t r = {sm64(seed ^ 0x4f7574ull)};
  double* q = out;
  double ground[4] = {0, 0, 1, 0};
  q = put(q, SYN_PLANE, ground, 4);
  for (int32_t b = 0; b < n_boxes; ++b) {
    double ex = rng_range(&r, edge_lo, edge_hi), ey = rng_range(&r, edge_lo, edge_hi);
    double ez = rng_range(&r, edge_lo, edge_hi);
    if (ez > sz) ez = sz;
    double cx = rng_range(&r, 0.5 * ex, sx - 0.5 * ex), cy = rng_range(&r, 0.5 * ey, sy - 0.5 * ey);
    double p[6] = {cx - 0.5 * ex, cy - 0.5 * ey, 0.0, cx + 0.5 * ex, cy + 0.5 * ey, ez};
    q = put(q, SYN_BOX, p, 6);
  }
  for (int32_t c = 0; c < n_cyl; ++c) {
    double rad = rng_range(&r, r_lo, r_hi), h = rng_range(&r, h_lo, h_hi);
    if (h > sz) h = sz;
    double p[5] = {rng_range(&r, rad, sx - rad), rng_range(&r, rad, sy - rad), rad, 0.0, h};
    q = put(q, SYN_CYL, p, 5);
  }
  return 1 + n_boxes + n_cyl;
}

/* Distance from point x to the surface of the solid primitives (rooms and
 * planes ignored); negative inside.  Used to keep trajectories clear. */
static double clearance(const double* prims, int32_t n, const double x[3]) {
  double best = INFINITY;
  for (int32_t i = 0; i < n; ++i) {
    const double* q = prims + (size_t)i * SYN_NPAR;
    const double* p = q + 1;
    double dist = INFINITY;
    if ((int)q[0] == SYN_BOX) {
      double out2 = 0, inside = -INFINITY;
      int in = 1;
      for (int k = 0; k < 3; ++k) {
        double lo = p[k] - x[k], hi = x[k] - p[3 + k];
        double e = lo > hi ? lo : hi;
        if (e > 0) { out2 += e * e; in = 0; }
        if (e > inside) inside = e;
      }
      dist = in ? inside : sqrt(out2);
    } else if ((int)q[0] == SYN_SPHERE) {
      double dx = x[0] - p[0], dy = x[1] - p[1], dz = x[2] - p[2];
      dist = sqrt(dx * dx + dy * dy + dz * dz) - p[3];
    } else if ((int)q[0] == SYN_CYL) {
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double radial = sqrt(dx * dx + dy * dy) - p[2];
      double vert = (x[2] < p[3]) ? p[3] - x[2] : (x[2] > p[4] ? x[2] - p[4] : -INFINITY);
      if (radial <= 0 && vert < 0) dist = radial > vert ? radial : vert;
      else dist = sqrt((radial > 0 ? radial * radial : 0) + (vert > 0 ? vert * vert : 0));
    }
    if (dist < best) best = dist;
  }
  return best;
}

/* Catmull-Rom position and tangent at global parameter u in [0, n_way-1]. */
static void spline_eval(double way[][2], int n_way, double u, double P[2], double D[2]) {
  int nseg = n_way - 1;
  int seg = (int)floor(u);
  if (seg >= nseg) seg = nseg - 1;
  if (seg < 0) seg = 0;
  double t = u - seg;
  int i0 = seg - 1 < 0 ? 0 : seg - 1, i1 = seg, i2 = seg + 1, i3 = seg + 2 > nseg ? nseg : seg + 2;
  for (int k = 0; k < 2; ++k) {
    double p0 = way[i0][k], p1 = way[i1][k], p2 = way[i2][k], p3 = way[i3][k];
    double a = 2 * p1, b = -p0 + p2, c = 2 * p0 - 5 * p1 + 4 * p2 - p3, d = -p0 + 3 * p1 - 3 * p2 + p3;
    P[k] = 0.5 * (a + b * t + c * t * t + d * t * t * t);
    D[k] = 0.5 * (b + 2 * c * t + 3 * d * t * t);
  }
}

/*
 * Smooth trajectory: uniform Catmull-Rom spline through n_way seeded
 * waypoints in [lo_xy, hi_xy]^2 at height z, sampled at n_samples uniform
 * parameter values.  Waypoints are drawn one at a time and re-drawn (up to
 * 500 times each) until the waypoint and the straight segment from the
 * previous one keep `clear` metres from every solid; whole sets are re-drawn
 * (up to 200 times) until the spline itself, checked at 2000 points, keeps
 * the clearance, else the set with the fewest violations is used.  The path
 * does not depend on n_samples.  Yaw follows the tangent, pitch 0.  Each pose
 * is a row-major 4x4 camera-to-world matrix with camera axes x right, y down,
 * z forward.  Returns the number of spline check points that violate the
 * clearance (0 for a clear path), or < 0 on bad arguments.
 */
int32_t synth_trajectory(uint64_t seed, const double* prims, int32_t n, int32_t n_way,
                         double lo_xy, double hi_xy, double z, double clear, int32_t n_samples,
                         double* out_T) {
  rng_t r = {sm64(seed ^ 0x5472616aull)};
  double way[64][2], best[64][2];
  int best_bad = -1;
  if (n_way < 2 || n_way > 64 || n_samples < 2) return -2;
  for (int attempt = 0; attempt < 200 && best_bad != 0; ++attempt) {
    for (int w = 0; w < n_way; ++w) {
      for (int tries = 0; tries < 500; ++tries) {
        way[w][0] = rng_range(&r, lo_xy, hi_xy);
        way[w][1] = rng_range(&r, lo_xy, hi_xy);
        double x[3] = {way[w][0], way[w][1], z};
        if (clearance(prims, n, x) < clear) continue;
        int ok = 1;
        if (w > 0) {
          double dx = way[w][0] - way[w - 1][0], dy = way[w][1] - way[w - 1][1];
          int steps = 1 + (int)(sqrt(dx * dx + dy * dy) / 0.05);
          for (int s = 1; s < steps && ok; ++s) {
            double y[3] = {way[w - 1][0] + dx * s / steps, way[w - 1][1] + dy * s / steps, z};
            if (clearance(prims, n, y) < clear) ok = 0;
          }
        }
        if (ok) break;
      }
    }
    int bad = 0;
    for (int s = 0; s < 2000; ++s) {
      double P[2], D[2];
      spline_eval(way, n_way, (double)s * (n_way - 1) / 1999.0, P, D);
      double x[3] = {P[0], P[1], z};
      if (clearance(prims, n, x) < clear) ++bad;
    }
    if (best_bad < 0 || bad < best_bad) {
      best_bad = bad;
      memcpy(best, way, sizeof(way));
    }
  }
  for (int32_t s = 0; s < n_samples; ++s) {
    double P[2], D[2];
    spline_eval(best, n_way, (double)s * (double)(n_way - 1) / (double)(n_samples - 1), P, D);
    double nrm = sqrt(D[0] * D[0] + D[1] * D[1]);
    double cy = nrm > 1e-12 ? D[0] / nrm : 1.0, sy = nrm > 1e-12 ? D[1] / nrm : 0.0;
    double* T = out_T + (size_t)s * 16;
    /* columns: x_cam = (sy, -cy, 0), y_cam = (0, 0, -1), z_cam = (cy, sy, 0) */
    T[0] = sy;  T[1] = 0;  T[2] = cy;  T[3] = P[0];
    T[4] = -cy; T[5] = 0;  T[6] = sy;  T[7] = P[1];
    T[8] = 0;   T[9] = -1; T[10] = 0;  T[11] = z;
    T[12] = 0;  T[13] = 0; T[14] = 0;  T[15] = 1;
  }
  return best_bad;
}
