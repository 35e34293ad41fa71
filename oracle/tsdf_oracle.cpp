/*
 * CPU oracle for projective TSDF integration — TEST INFRASTRUCTURE ONLY.
 *
 * This is the plain, slow, obviously-correct restatement of the method that
 * the CUDA path is checked against.  Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (nvblox, Sec. IV-B "Frame Integration"):
 *   - blocks in view: for every valid pixel the segment of its ray that lies
 *     within the truncation band [d - tau, d + tau] is traversed through the
 *     block grid (Amanatides & Woo voxel traversal, as Sec. IV-B cites) and
 *     every block it passes through is allocated (D = 0, W = 0) if missing;
 *   - voxel update: every voxel of every block in this frame's band set is
 *     projected into the image (Eq. 1; pinhole Eq. 2, LiDAR Eq. 3), the depth
 *     is sampled (nearest pixel for a camera, guarded bilinear for LiDAR),
 *     d_p = d - d_v is formed, voxels with d_p < -tau are skipped, d_p is
 *     clamped to +tau, and the weighted running average is applied with the
 *     weight f_w (constant 1 by default; optional sensor-error models),
 *     weights added up to max_weight (Sec. IV-B);
 *   - occupancy layer (Sec. IV-B, second functor), optional: the same voxels
 *     instead add a constant log-odds, negative in front of the surface
 *     (d_p > 0), positive otherwise; a decay step (Sec. V-E: dynamic content
 *     of an occupancy layer fades over time) moves every voxel's log-odds
 *     toward 0 by a fixed amount without crossing 0.
 *
 * Storage: std::unordered_map from integer block coordinates to a block of
 * 8x8x8 voxels holding D (double) and W (double), voxel index
 * x + 8 y + 64 z inside the block.
 *
 * Precision contract.  Every VALUE (d_v, s, D, W, bilinear depth) is FP64.
 * Every DISCRETE decision (which blocks a ray segment passes through, which
 * pixel a voxel projects to, sample validity, the d_p >= -tau test, LiDAR
 * cell choice and the fg/bg guard) is taken with a prescribed sequence of
 * IEEE single-precision operations, written out below with explicit fmaf and
 * compiled with -ffp-contract=off, so that a GPU kernel that takes the same
 * decisions in FP32 can be compared bit-exactly on block sets and weights.
 * The sequence is:
 *   host FP64: R, t from T_LC; B = 8 v; anchor a = floor(t / B);
 *     Rcl = (float) R^T;  tloc_i = (float)((R_0i e_0 + R_1i e_1) + R_2i e_2)
 *     with e_k = a_k B - t_k;  M = (float)(R / B);  o_k = (float)((t_k - a_k B) / B);
 *     tau_f = (float)(trunc_voxels * v).
 *   voxel: rel = (b - a) * 8 + l;  q = ((float)rel + 0.5f) * v;
 *     p_i = fmaf(Rcl_i0, q_0, fmaf(Rcl_i1, q_1, fmaf(Rcl_i2, q_2, tloc_i))).
 *   pinhole: z = p_2 > 0;  iz = 1/z;  u = fmaf(p_0 * iz, fu, cu);
 *     pixel = (int)(u + 0.5f) after checking 0 <= u + 0.5f < W (same for v).
 *   ray segment: r = ((i - cu)/fu, (j - cv)/fv, 1) (camera) or the beam
 *     direction from FP64 cos/sin tables (LiDAR); dir_k = M_k . r (fmaf chain);
 *     cells along z (or range) in [max(d - tau_f, 0), d + tau_f] by the
 *     traversal in dda() below.
 * Where a decision needs atan2 (LiDAR, Eq. 3) it uses atan2_dec(): octant
 * reduction, the half-angle identity atan t = 2 atan(t / (1 + sqrt(1 + t^2)))
 * applied twice, then the Maclaurin (Gregory) series of atan through t^13.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <unordered_map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Key {
  int64_t x, y, z;
  bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
  bool operator<(const Key& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

struct Block {
  double D[512];
  double W[512];
  double C[512][3];  // colour layer: running average of r, g, b
};

struct Counters {
  int64_t candidates = 0;     // cells emitted by all ray traversals (with repeats)
  int64_t band_blocks = 0;    // |B_f|
  int64_t new_blocks = 0;     // blocks allocated by this frame
  int64_t voxels_updated = 0; // (voxel, frame) pairs that passed the update test
  int64_t truncated_rays = 0; // traversals cut at kMaxCells
};

constexpr int kMaxCells = 32;

struct Oracle {
  float v;
  int trunc;
  float wmax;
  double vd, Bd, taud;
  float tauf;
  int lidar_nearest = 0;
  float guard_f;  // LiDAR fg/bg guard threshold (metres)
  // occupancy layer (Sec. IV-B, second functor): D holds the log-odds, W
  // the number of updates
  int occupancy = 0;
  double l_occ = 0.0, l_free = 0.0;
  // weighting function of the TSDF update
  int weighting = 0;
  double dropoff = 0.0;
  std::unordered_map<Key, std::unique_ptr<Block>, KeyHash> blocks;
  Counters last;
  int64_t total_updates = 0;
  std::vector<Key> last_band;
};

/* ------------------------------------------------------------ pose (A0) */

struct Pose {
  double R[3][3], t[3];      // T_LC: sensor-to-layer rotation and translation
  int64_t a[3];              // anchor block (block containing the sensor origin)
  float Rcl[3][3], tloc[3];  // FP32 voxel-to-sensor transform, anchor-local
  float M[3][3], o[3];       // FP32 layer rotation in block units, origin in block units
};

Pose make_pose(const double* T, double Bd) {
  Pose P;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) P.R[i][j] = T[4 * i + j];
    P.t[i] = T[4 * i + 3];
  }
  double e[3];
  for (int k = 0; k < 3; ++k) {
    P.a[k] = (int64_t)std::floor(P.t[k] / Bd);
    e[k] = (double)P.a[k] * Bd - P.t[k];
  }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) P.Rcl[i][j] = (float)P.R[j][i];
    P.tloc[i] = (float)((P.R[0][i] * e[0] + P.R[1][i] * e[1]) + P.R[2][i] * e[2]);
    for (int j = 0; j < 3; ++j) P.M[i][j] = (float)(P.R[i][j] / Bd);
    P.o[i] = (float)((P.t[i] - (double)P.a[i] * Bd) / Bd);
  }
  return P;
}

/* p_C = T_CL p_L = R^T (p_L - t), FP64 (the value path of Eq. 1) */
void to_sensor64(const Pose& P, const double pL[3], double pC[3]) {
  double d[3] = {pL[0] - P.t[0], pL[1] - P.t[1], pL[2] - P.t[2]};
  for (int k = 0; k < 3; ++k) pC[k] = P.R[0][k] * d[0] + P.R[1][k] * d[1] + P.R[2][k] * d[2];
}

/* ------------------------------------------------- block traversal (A2) */

/*
 * Cells of the block grid (anchor-relative integer coordinates) passed by the
 * segment p(s) = o + s dir, s in [s0, s1], in block units: Amanatides & Woo
 * traversal with z-absolute crossing parameters, ties between axes taken in
 * x, y, z order, at most kMaxCells cells.
 */
int dda(const float o[3], const float dir[3], float s0, float s1, int32_t cells[][3],
        int* truncated) {
  int c[3], step[3];
  float inv[3], tmax[3];
  *truncated = 0;
  float start[3];
  for (int k = 0; k < 3; ++k) {
    start[k] = std::fmaf(s0, dir[k], o[k]);
    // keys hold 21-bit coordinates: a segment that starts 2^18 blocks or
    // more from the sensor's block is outside the map's range and dropped
    if (!(std::fabs(start[k]) < 262144.0f)) return 0;
  }
  for (int k = 0; k < 3; ++k) {
    c[k] = (int)std::floor(start[k]);
    step[k] = dir[k] > 0.0f ? 1 : (dir[k] < 0.0f ? -1 : 0);
    inv[k] = step[k] != 0 ? 1.0f / dir[k] : 0.0f;
  }
  auto crossing = [&](int k) -> float {
    if (step[k] == 0) return INFINITY;
    float bnd = (float)(step[k] > 0 ? c[k] + 1 : c[k]);
    return (bnd - o[k]) * inv[k];
  };
  for (int k = 0; k < 3; ++k) tmax[k] = crossing(k);
  int n = 0;
  for (int k = 0; k < 3; ++k) cells[n][k] = c[k];
  ++n;
  while (true) {
    int k = 0;
    if (tmax[1] < tmax[k]) k = 1;
    if (tmax[2] < tmax[k]) k = 2;
    if (!(tmax[k] <= s1)) break;
    if (n == kMaxCells) { *truncated = 1; break; }
    c[k] += step[k];
    tmax[k] = crossing(k);
    for (int q = 0; q < 3; ++q) cells[n][q] = c[q];
    ++n;
  }
  return n;
}

/* ------------------------------------------- FP32 atan2 for decisions */

float atan2_dec(float y, float x) {
  const float ax = std::fabs(x), ay = std::fabs(y);
  const float mx = std::fmax(ax, ay), mn = std::fmin(ax, ay);
  if (mx == 0.0f) return 0.0f;
  const float t = mn / mx;
  const float t1 = t / (1.0f + std::sqrt(std::fmaf(t, t, 1.0f)));
  const float t2 = t1 / (1.0f + std::sqrt(std::fmaf(t1, t1, 1.0f)));
  const float z = t2 * t2;
  // Maclaurin coefficients (-1)^n / (2n + 1), n = 6 .. 1, each an IEEE quotient
  float p = 1.0f / 13.0f;
  p = std::fmaf(p, z, -(1.0f / 11.0f));
  p = std::fmaf(p, z, 1.0f / 9.0f);
  p = std::fmaf(p, z, -(1.0f / 7.0f));
  p = std::fmaf(p, z, 1.0f / 5.0f);
  p = std::fmaf(p, z, -(1.0f / 3.0f));
  p = std::fmaf(p, z, 1.0f);
  float a = 4.0f * (t2 * p);
  if (ay > ax) a = (float)(M_PI / 2) - a;
  if (x < 0.0f) a = (float)M_PI - a;
  if (y < 0.0f) a = -a;
  return a;
}

/* -------------------------------------------------------- shared steps */

void insert_band(Oracle& m, const Pose& P, const std::vector<std::vector<Key>>& per_thread,
                 std::vector<Block*>& band, std::vector<uint8_t>& fresh) {
  std::vector<Key> keys;
  for (auto& v : per_thread) keys.insert(keys.end(), v.begin(), v.end());
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  m.last.band_blocks = (int64_t)keys.size();
  band.clear();
  fresh.clear();
  for (const Key& k : keys) {
    auto it = m.blocks.find(k);
    if (it == m.blocks.end()) {
      auto b = std::make_unique<Block>();
      for (int i = 0; i < 512; ++i) {
        b->D[i] = 0.0;
        b->W[i] = 0.0;
        b->C[i][0] = b->C[i][1] = b->C[i][2] = 0.0;
      }
      band.push_back(b.get());
      m.blocks.emplace(k, std::move(b));
      m.last.new_blocks++;
    } else {
      band.push_back(it->second.get());
    }
  }
  m.last_band = keys;
  (void)P;
}

/* Running weighted average with constant weight 1, weights added up to the
 * maximum; the average uses the unclamped sum W + 1 (Sec. IV-B). */
inline void tsdf_update(double& D, double& W, double s, double w, double wmax) {
  if (!(W + w > 0.0)) return;  // zero weight on an unobserved voxel
  D = (W * D + w * s) / (W + w);
  W = std::min(W + w, wmax);
}

/* Weighting function f_w (Sec. IV-B: constant or from the sensor's error
 * model): mode 0 constant 1; 1 inverse square of the voxel depth d_v; 2
 * constant with a linear drop-off behind the surface, from 1 at
 * d_p = -delta to 0 at d_p = -tau; 3 inverse square times that drop-off.
 * dp is the projective distance before truncation. */
inline double weight(int mode, double dv, double dp, double delta, double tau) {
  double w = (mode == 1 || mode == 3) ? 1.0 / (dv * dv) : 1.0;
  if ((mode == 2 || mode == 3) && dp < -delta) w *= (tau + dp) / (tau - delta);
  return w;
}

/* Colour functor: running average of the pixel's r, g, b with weight 1,
 * weights added up to the maximum (the TSDF rule applied per channel). */
inline void color_update(double* C, double& W, uint32_t rgba, double wmax) {
  const double c[3] = {(double)(rgba & 255u), (double)((rgba >> 8) & 255u), (double)((rgba >> 16) & 255u)};
  for (int k = 0; k < 3; ++k) C[k] = (W * C[k] + c[k]) / (W + 1.0);
  W = std::min(W + 1.0, wmax);
}

/* Occupancy functor (Sec. IV-B): running addition of a constant negative
 * log-odds where the voxel lies in front of the measured surface (d_p > 0)
 * and a constant positive one otherwise (-tau <= d_p <= 0; the voxels more
 * than tau behind it were skipped as unobserved). */
inline void occupancy_update(double& L, double& N, bool in_front, double l_occ, double l_free) {
  L += in_front ? l_free : l_occ;
  N += 1.0;
}

/* Occupancy decay (Sec. V-E, the paper gives no rule): log-odds above 0
 * (occupied) drop by decay_occ, log-odds below 0 (free) rise by decay_free,
 * neither crossing 0, so every voxel drifts back to the prior p = 0.5. */
inline void occupancy_decay(double& L, double decay_occ, double decay_free) {
  if (L > 0.0) L = std::max(L - decay_occ, 0.0);
  else if (L < 0.0) L = std::min(L + decay_free, 0.0);
}

}  // namespace

extern "C" {

void* orc_create(float voxel_size, int32_t truncation_voxels, float max_weight) {
  auto* m = new Oracle();
  m->v = voxel_size;
  m->trunc = truncation_voxels;
  m->wmax = max_weight;
  m->vd = (double)voxel_size;
  m->Bd = 8.0 * m->vd;
  m->taud = (double)truncation_voxels * m->vd;
  m->tauf = (float)m->taud;
  m->guard_f = m->tauf;
  return m;
}

void orc_destroy(void* h) { delete static_cast<Oracle*>(h); }

/* Weighting function of the TSDF update (see weight()); dropoff is the
 * distance behind the surface where the drop-off starts (<= 0: one voxel). */
void orc_set_weighting(void* h, int32_t mode, float dropoff) {
  auto* m = static_cast<Oracle*>(h);
  m->weighting = mode;
  m->dropoff = dropoff > 0.0f ? (double)dropoff : m->vd;
}

/* Occupancy layer: voxels accumulate log-odds l_occ (on or behind the
 * surface, within tau) or l_free (in front of it) instead of the TSDF; the
 * exported D is the log-odds and W the number of updates. */
void orc_set_occupancy(void* h, float l_occ, float l_free) {
  auto* m = static_cast<Oracle*>(h);
  m->occupancy = 1;
  m->l_occ = (double)l_occ;
  m->l_free = (double)l_free;
}

/* One decay step of an occupancy layer over every allocated voxel (the
 * update counts are kept).  Returns -1 if the layer is not an occupancy
 * layer or a step is negative. */
int32_t orc_decay_occupancy(void* h, float decay_occ, float decay_free) {
  auto* m = static_cast<Oracle*>(h);
  if (!m->occupancy || !(decay_occ >= 0.0f) || !(decay_free >= 0.0f)) return -1;
  for (auto& kv : m->blocks)
    for (int l = 0; l < 512; ++l) occupancy_decay(kv.second->D[l], decay_occ, decay_free);
  return 0;
}

/* LiDAR sampling: nearest != 0 selects nearest-cell sampling (a test mode);
 * guard is the fg/bg threshold of the bilinear mode in metres (<= 0: tau). */
void orc_set_lidar_sampling(void* h, int32_t nearest, float guard) {
  auto* m = static_cast<Oracle*>(h);
  m->lidar_nearest = nearest;
  m->guard_f = guard > 0.0f ? guard : m->tauf;
}

/*
 * Integrate one pinhole z-depth image (row-major float[H][W]; d <= 0 or
 * non-finite = invalid) taken at pose T_LC (row-major 4x4, sensor-to-layer).
 */
}  // extern "C"

namespace {

/* One pinhole frame; with rgba != nullptr the frame feeds the colour layer:
 * voxels within the truncation band on either side of the surface
 * (-tau <= d_p <= tau) average the colour of their pixel, weight 1. */
int32_t integrate_pinhole(Oracle& m, const float* depth, const uint32_t* rgba, int32_t W, int32_t H,
                          float fu, float fv, float cu, float cv, const double* T) {
  const Pose P = make_pose(T, m.Bd);
  // block coordinates are 21-bit: the sensor's block must lie within 2^19
  for (int c = 0; c < 3; ++c)
    if (!(P.a[c] > -524288 && P.a[c] < 524288)) return -1;
  m.last = Counters();
  const float tau = m.tauf;

  // A1-A2: band segment of every valid pixel through the block grid.
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  std::vector<std::vector<Key>> per_thread(nthreads);
  std::vector<int64_t> cand(nthreads, 0), trunc_rays(nthreads, 0);
#pragma omp parallel for schedule(static)
  for (int32_t j = 0; j < H; ++j) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int32_t cells[kMaxCells][3];
    for (int32_t i = 0; i < W; ++i) {
      const float d = depth[(size_t)j * W + i];
      if (!(d > 0.0f && d <= 3.402823466e38f)) continue;
      const float rx = ((float)i - cu) / fu, ry = ((float)j - cv) / fv;
      float dir[3];
      for (int k = 0; k < 3; ++k) dir[k] = std::fmaf(P.M[k][0], rx, std::fmaf(P.M[k][1], ry, P.M[k][2]));
      const float s0 = std::fmax(d - tau, 0.0f), s1 = d + tau;
      int tr = 0;
      const int n = dda(P.o, dir, s0, s1, cells, &tr);
      trunc_rays[tid] += tr;
      cand[tid] += n;
      for (int c = 0; c < n; ++c)
        per_thread[tid].push_back(Key{P.a[0] + cells[c][0], P.a[1] + cells[c][1], P.a[2] + cells[c][2]});
    }
  }
  for (int t = 0; t < nthreads; ++t) { m.last.candidates += cand[t]; m.last.truncated_rays += trunc_rays[t]; }

  // A3: allocate missing blocks; B_f is this frame's band set.
  std::vector<Block*> band;
  std::vector<uint8_t> fresh;
  insert_band(m, P, per_thread, band, fresh);
  const std::vector<Key> keys = m.last_band;

  // A4-A6: every voxel of every block in B_f.
  int64_t updated = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : updated)
  for (int64_t bi = 0; bi < (int64_t)band.size(); ++bi) {
    Block* blk = band[bi];
    const Key& b = keys[bi];
    for (int lz = 0; lz < 8; ++lz)
      for (int ly = 0; ly < 8; ++ly)
        for (int lx = 0; lx < 8; ++lx) {
          const int l = lx + 8 * ly + 64 * lz;
          const int64_t rel[3] = {(b.x - P.a[0]) * 8 + lx, (b.y - P.a[1]) * 8 + ly, (b.z - P.a[2]) * 8 + lz};
          // decision arithmetic (FP32)
          float q[3], p[3];
          for (int k = 0; k < 3; ++k) q[k] = ((float)rel[k] + 0.5f) * m.v;
          for (int k = 0; k < 3; ++k)
            p[k] = std::fmaf(P.Rcl[k][0], q[0], std::fmaf(P.Rcl[k][1], q[1], std::fmaf(P.Rcl[k][2], q[2], P.tloc[k])));
          if (!(p[2] > 0.0f)) continue;
          const float iz = 1.0f / p[2];
          const float u = std::fmaf(p[0] * iz, fu, cu) + 0.5f;
          const float v = std::fmaf(p[1] * iz, fv, cv) + 0.5f;
          if (!(u >= 0.0f && u < (float)W && v >= 0.0f && v < (float)H)) continue;
          const float d = depth[(size_t)(int)v * W + (int)u];
          if (!(d > 0.0f && d <= 3.402823466e38f)) continue;
          if (d - p[2] < -tau) continue;
          if (rgba) {
            if (d - p[2] > tau) continue;  // colour only near the surface
            const uint32_t c = rgba[(size_t)(int)v * W + (int)u];
            color_update(blk->C[l], blk->W[l], c, (double)m.wmax);
            ++updated;
            continue;
          }
          // value arithmetic (FP64): d_v is the voxel's z-depth in the camera
          const int64_t g[3] = {b.x * 8 + lx, b.y * 8 + ly, b.z * 8 + lz};
          const double pL[3] = {((double)g[0] + 0.5) * m.vd, ((double)g[1] + 0.5) * m.vd,
                                ((double)g[2] + 0.5) * m.vd};
          double pC[3];
          to_sensor64(P, pL, pC);
          if (m.occupancy) {
            occupancy_update(blk->D[l], blk->W[l], d - p[2] > 0.0f, m.l_occ, m.l_free);
          } else {
            const double dp = (double)d - pC[2];
            tsdf_update(blk->D[l], blk->W[l], std::min(dp, m.taud),
                        weight(m.weighting, pC[2], dp, m.dropoff, m.taud), (double)m.wmax);
          }
          ++updated;
        }
  }
  m.last.voxels_updated = updated;
  m.total_updates += updated;
  return 0;
}

}  // namespace

extern "C" {

/*
 * Integrate one pinhole z-depth image (row-major float[H][W]; d <= 0 or
 * non-finite = invalid) taken at pose T_LC (row-major 4x4, sensor-to-layer).
 */
int32_t orc_integrate_pinhole(void* h, const float* depth, int32_t W, int32_t H, float fu,
                              float fv, float cu, float cv, const double* T) {
  return integrate_pinhole(*static_cast<Oracle*>(h), depth, nullptr, W, H, fu, fv, cu, cv, T);
}

/* Integrate a registered depth + colour pair (rgba: row-major uint32 [H][W],
 * r in the low byte, then g, b; the top byte is ignored) into the colour
 * layer: the exported D is unused, W counts the colour updates and
 * orc_export_color returns the averaged colours. */
int32_t orc_integrate_color(void* h, const float* depth, const uint32_t* rgba, int32_t W, int32_t H,
                            float fu, float fv, float cu, float cv, const double* T) {
  return integrate_pinhole(*static_cast<Oracle*>(h), depth, rgba, W, H, fu, fv, cu, cv, T);
}

/*
 * Integrate one LiDAR range image (row-major float[n_el][n_az], row 0 = the
 * smallest polar angle; ranges outside [min_range, max_range] or non-finite
 * are invalid).  Columns cover the full azimuth circle from theta_start;
 * rows cover polar angles [phi_start, phi_start + el_fov].
 */
int32_t orc_integrate_lidar(void* h, const float* range, int32_t n_az, int32_t n_el,
                            float theta_start, float phi_start, float el_fov, float min_range,
                            float max_range, const double* T) {
  Oracle& m = *static_cast<Oracle*>(h);
  const Pose P = make_pose(T, m.Bd);
  // block coordinates are 21-bit: the sensor's block must lie within 2^19
  for (int c = 0; c < 3; ++c)
    if (!(P.a[c] > -524288 && P.a[c] < 524288)) return -1;
  m.last = Counters();
  const float tau = m.tauf;
  auto valid = [&](float d) { return d >= min_range && d <= max_range; };

  // beam-centre direction tables (FP64 -> FP32)
  std::vector<float> ct(n_az), st(n_az), cp(n_el), sp(n_el);
  for (int k = 0; k < n_az; ++k) {
    double th = (double)theta_start + ((double)k + 0.5) * (6.283185307179586 / (double)n_az);
    ct[k] = (float)std::cos(th);
    st[k] = (float)std::sin(th);
  }
  for (int j = 0; j < n_el; ++j) {
    double ph = (double)phi_start + ((double)j + 0.5) * ((double)el_fov / (double)n_el);
    cp[j] = (float)std::cos(ph);
    sp[j] = (float)std::sin(ph);
  }
  // pixels per radian (Eq. 3)
  const float alpha = (float)((double)n_az / 6.283185307179586);
  const float beta = (float)((double)n_el / (double)el_fov);

  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  std::vector<std::vector<Key>> per_thread(nthreads);
  std::vector<int64_t> cand(nthreads, 0), trunc_rays(nthreads, 0);
#pragma omp parallel for schedule(static)
  for (int32_t j = 0; j < n_el; ++j) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int32_t cells[kMaxCells][3];
    for (int32_t k = 0; k < n_az; ++k) {
      const float d = range[(size_t)j * n_az + k];
      if (!valid(d)) continue;
      const float bx = sp[j] * ct[k], by = sp[j] * st[k], bz = cp[j];
      float dir[3];
      for (int q = 0; q < 3; ++q) dir[q] = std::fmaf(P.M[q][0], bx, std::fmaf(P.M[q][1], by, P.M[q][2] * bz));
      const float s0 = std::fmax(d - tau, 0.0f), s1 = d + tau;
      int tr = 0;
      const int n = dda(P.o, dir, s0, s1, cells, &tr);
      trunc_rays[tid] += tr;
      cand[tid] += n;
      for (int c = 0; c < n; ++c)
        per_thread[tid].push_back(Key{P.a[0] + cells[c][0], P.a[1] + cells[c][1], P.a[2] + cells[c][2]});
    }
  }
  for (int t = 0; t < nthreads; ++t) { m.last.candidates += cand[t]; m.last.truncated_rays += trunc_rays[t]; }

  std::vector<Block*> band;
  std::vector<uint8_t> fresh;
  insert_band(m, P, per_thread, band, fresh);
  const std::vector<Key> keys = m.last_band;

  int64_t updated = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : updated)
  for (int64_t bi = 0; bi < (int64_t)band.size(); ++bi) {
    Block* blk = band[bi];
    const Key& b = keys[bi];
    for (int lz = 0; lz < 8; ++lz)
      for (int ly = 0; ly < 8; ++ly)
        for (int lx = 0; lx < 8; ++lx) {
          const int l = lx + 8 * ly + 64 * lz;
          const int64_t rel[3] = {(b.x - P.a[0]) * 8 + lx, (b.y - P.a[1]) * 8 + ly, (b.z - P.a[2]) * 8 + lz};
          float q[3], p[3];
          for (int c = 0; c < 3; ++c) q[c] = ((float)rel[c] + 0.5f) * m.v;
          for (int c = 0; c < 3; ++c)
            p[c] = std::fmaf(P.Rcl[c][0], q[0], std::fmaf(P.Rcl[c][1], q[1], std::fmaf(P.Rcl[c][2], q[2], P.tloc[c])));
          // Eq. 3 in FP32 decision arithmetic: r, azimuth, polar angle
          const float r = std::sqrt(std::fmaf(p[0], p[0], std::fmaf(p[1], p[1], p[2] * p[2])));
          if (!(r > 0.0f)) continue;
          const float rho = std::sqrt(std::fmaf(p[0], p[0], p[1] * p[1]));
          const float th = atan2_dec(p[1], p[0]);
          const float ph = atan2_dec(rho, p[2]);
          const float u = (th - theta_start) * alpha;
          const float v = (ph - phi_start) * beta;
          float dsamp32;
          double dsamp64;
          if (m.lidar_nearest) {
            const float ku = std::floor(u), jv = std::floor(v);
            if (!(jv >= 0.0f && jv <= (float)(n_el - 1))) continue;
            if (!(ku >= -1.0f && ku <= (float)n_az)) continue;
            const int kk = (((int)ku % n_az) + n_az) % n_az, jj = (int)jv;
            dsamp32 = range[(size_t)jj * n_az + kk];
            if (!valid(dsamp32)) continue;
            dsamp64 = dsamp32;
          } else {
            // guarded bilinear over the four beam centres around (u, v)
            const float uu = u - 0.5f, vv = v - 0.5f;
            const float k0f = std::floor(uu), j0f = std::floor(vv);
            if (!(j0f >= 0.0f && j0f <= (float)(n_el - 2))) continue;
            if (!(k0f >= -1.0f && k0f <= (float)n_az)) continue;
            const float fx = uu - k0f, fy = vv - j0f;
            const int k0 = (((int)k0f % n_az) + n_az) % n_az, k1 = (k0 + 1) % n_az, j0 = (int)j0f;
            const float d00 = range[(size_t)j0 * n_az + k0], d10 = range[(size_t)j0 * n_az + k1];
            const float d01 = range[(size_t)(j0 + 1) * n_az + k0], d11 = range[(size_t)(j0 + 1) * n_az + k1];
            if (!(valid(d00) && valid(d10) && valid(d01) && valid(d11))) continue;
            const float hi = std::fmax(std::fmax(d00, d10), std::fmax(d01, d11));
            const float lo = std::fmin(std::fmin(d00, d10), std::fmin(d01, d11));
            if (hi - lo > m.guard_f) continue;
            const float top = std::fmaf(fx, d10 - d00, d00);
            const float bot = std::fmaf(fx, d11 - d01, d01);
            dsamp32 = std::fmaf(fy, bot - top, top);
            const double fxd = fx, fyd = fy;
            dsamp64 = (1.0 - fyd) * ((1.0 - fxd) * d00 + fxd * d10) + fyd * ((1.0 - fxd) * d01 + fxd * d11);
          }
          if (dsamp32 - r < -tau) continue;
          // value arithmetic (FP64): d_v is the voxel's range from the sensor
          const int64_t g[3] = {b.x * 8 + lx, b.y * 8 + ly, b.z * 8 + lz};
          const double pL[3] = {((double)g[0] + 0.5) * m.vd, ((double)g[1] + 0.5) * m.vd,
                                ((double)g[2] + 0.5) * m.vd};
          double pC[3];
          to_sensor64(P, pL, pC);
          const double r64 = std::sqrt(pC[0] * pC[0] + pC[1] * pC[1] + pC[2] * pC[2]);
          if (m.occupancy) {
            occupancy_update(blk->D[l], blk->W[l], dsamp32 - r > 0.0f, m.l_occ, m.l_free);
          } else {
            const double dp = dsamp64 - r64;
            tsdf_update(blk->D[l], blk->W[l], std::min(dp, m.taud),
                        weight(m.weighting, r64, dp, m.dropoff, m.taud), (double)m.wmax);
          }
          ++updated;
        }
  }
  m.last.voxels_updated = updated;
  m.total_updates += updated;
  return 0;
}

int64_t orc_num_blocks(void* h) { return (int64_t) static_cast<Oracle*>(h)->blocks.size(); }

/* Export all blocks sorted by (x, y, z): keys [n][3], D [n][512], W [n][512]. */
int64_t orc_export(void* h, int32_t* keys, double* D, double* W, int64_t cap) {
  Oracle& m = *static_cast<Oracle*>(h);
  std::vector<Key> ks;
  ks.reserve(m.blocks.size());
  for (auto& kv : m.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  if ((int64_t)ks.size() > cap) return -1;
  for (size_t i = 0; i < ks.size(); ++i) {
    keys[3 * i + 0] = (int32_t)ks[i].x;
    keys[3 * i + 1] = (int32_t)ks[i].y;
    keys[3 * i + 2] = (int32_t)ks[i].z;
    const Block* b = m.blocks[ks[i]].get();
    if (D) std::memcpy(D + 512 * i, b->D, sizeof(b->D));
    if (W) std::memcpy(W + 512 * i, b->W, sizeof(b->W));
  }
  return (int64_t)ks.size();
}

/* Colours of all blocks, sorted like orc_export: rgb [n][512][3]. */
int64_t orc_export_color(void* h, double* rgb, int64_t cap) {
  Oracle& m = *static_cast<Oracle*>(h);
  std::vector<Key> ks;
  for (auto& kv : m.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  if ((int64_t)ks.size() > cap) return -1;
  for (size_t i = 0; i < ks.size(); ++i)
    std::memcpy(rgb + (size_t)1536 * i, m.blocks[ks[i]]->C, sizeof(double) * 1536);
  return (int64_t)ks.size();
}

/* Band set of the last integrated frame, sorted: keys [n][3]. */
int64_t orc_last_band(void* h, int32_t* keys, int64_t cap) {
  Oracle& m = *static_cast<Oracle*>(h);
  if ((int64_t)m.last_band.size() > cap) return -1;
  for (size_t i = 0; i < m.last_band.size(); ++i) {
    keys[3 * i + 0] = (int32_t)m.last_band[i].x;
    keys[3 * i + 1] = (int32_t)m.last_band[i].y;
    keys[3 * i + 2] = (int32_t)m.last_band[i].z;
  }
  return (int64_t)m.last_band.size();
}

/* Counters of the last frame: candidates, band blocks, new blocks, voxel
 * updates, truncated traversals; out[5] = total updates so far. */
void orc_counters(void* h, int64_t* out) {
  Oracle& m = *static_cast<Oracle*>(h);
  out[0] = m.last.candidates;
  out[1] = m.last.band_blocks;
  out[2] = m.last.new_blocks;
  out[3] = m.last.voxels_updated;
  out[4] = m.last.truncated_rays;
  out[5] = m.total_updates;
}

/* The FP32 decision atan2, exposed so that tests can bound its error. */
float orc_atan2_dec(float y, float x) { return atan2_dec(y, x); }

/* The block traversal alone, exposed so that tests can check it against a
 * brute-force slab test: returns the number of cells written to cells[n][3]. */
int32_t orc_dda(const float* o, const float* dir, float s0, float s1, int32_t* cells) {
  int tr = 0;
  return dda(o, dir, s0, s1, reinterpret_cast<int32_t(*)[3]>(cells), &tr);
}

}  // extern "C"
