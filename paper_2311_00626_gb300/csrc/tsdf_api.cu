// Host side of the GB300 TSDF library: the C ABI declared in include/tsdf.h.
//
// Per frame the host only prepares the pose (FP64, Sec. III's T_LC inverted
// into T_CL, anchored at the block that holds the sensor origin and rounded
// once to FP32) and enqueues two kernels: the band allocator and the
// per-voxel integrator (Sec. IV-B).  Nothing here touches voxel data.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "tsdf.h"
#include "tsdf_internal.cuh"

using gbt::BatchParams;
using gbt::EsdfDev;
using gbt::FrameDev;
using gbt::MapDev;

struct LidarTable {
  int32_t n_az, n_el;
  float theta_start, phi_start, el_fov;
  float* dev;  // float2 [n_az] (cos, sin azimuth) then float2 [n_el] (cos, sin polar)
  int lsb;     // smallest last-place exponent of a nonzero beam direction component (fast_rcp_ok)
};

struct tsdf_map {
  MapDev dev;
  int device;
  uint32_t cap;
  int64_t max_blocks;
  int storage;
  float v, wmax;
  int32_t trunc;
  double vd, Bd;
  int n_ctas_integrate;
  int tile_h;  // allocation tile height, 0 = automatic
  int launch_mode;     // TSDF_LAUNCH_SPLIT or TSDF_LAUNCH_FUSED
  int32_t wait_extra;  // map_wait_test: extra CTAs the fused launch's grid-wide wait expects
  int64_t frames;
  unsigned long long status_seen;  // device status bits observed by the host
  std::vector<LidarTable> tables;
  // second mask / work-list / control set: with it the allocation of one
  // sub-batch runs on `aux` while the previous sub-batch integrates
  uint32_t* mask1;
  uint32_t* list1;
  unsigned int* ctl1;
  cudaStream_t aux;
  cudaEvent_t ev_alloc[4], ev_int[4], ev_start;
  // host-input batches: copy stream and per-sub-batch copy events (lazy)
  cudaStream_t copy;
  cudaEvent_t ev_copy[4];
  // diagnostics: per call (alloc start, alloc end, integrate start, integrate end)
  bool timing;
  std::vector<cudaEvent_t> events;
  size_t n_timed;
  // ESDF layer, allocated by the first map_esdf_update
  bool esdf_on;
  EsdfDev esdf;
  tsdf_esdf_opts esdf_opts;
  uint32_t esdf_gen;      // generation of the last update set / tlist built
  uint32_t* esdf_host;    // pinned copy of esdf.cnt
  // meshing scratch, allocated by the first map_mesh
  bool mesh_on;
  gbt::MeshDev mesh;
  uint32_t mesh_gen;
};

namespace {

constexpr int64_t kDefaultBlocks = 1 << 18;
constexpr size_t kTimedCalls = 4096;
constexpr int32_t kMaxBatchFrames = 1 << 16;

tsdf_status cuda_fail() {
  cudaGetLastError();
  return TSDF_ERR_CUDA;
}

tsdf_status status_from_bits(unsigned long long bits) {
  if (bits & (gbt::kStPoolFull | gbt::kStHashFull | gbt::kStListFull)) return TSDF_ERR_CAPACITY;
  if (bits & gbt::kStTimeout) return TSDF_ERR_TIMEOUT;
  return TSDF_OK;
}

bool finite_all(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// T must be a rigid transform: finite, rotation block orthonormal.
bool rigid(const double* T) {
  if (!finite_all(T, 16)) return false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double d = 0;
      for (int k = 0; k < 3; ++k) d += T[4 * k + i] * T[4 * k + j];
      if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-5) return false;
    }
  return true;
}

// Pose preparation (FP64 -> FP32), shared by both sensor kinds.  With
// T = T_LC = [R | t]: anchor a = floor(t / B); voxel-to-sensor rotation
// R^T and translation R^T (a B - t) in anchor-local metres; ray rotation
// R / B and sensor origin (t - a B) / B in anchor-relative block units.
bool prepare_pose(double Bd, const double* T, FrameDev& F) {
  double R[3][3], t[3], e[3];
  int64_t a[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) R[i][j] = T[4 * i + j];
    t[i] = T[4 * i + 3];
  }
  for (int k = 0; k < 3; ++k) {
    a[k] = (int64_t)std::floor(t[k] / Bd);
    if (!(a[k] > -524288 && a[k] < 524288)) return false;
    e[k] = (double)a[k] * Bd - t[k];
  }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) F.Rcl[3 * i + j] = (float)R[j][i];
    F.tloc[i] = (float)((R[0][i] * e[0] + R[1][i] * e[1]) + R[2][i] * e[2]);
    for (int j = 0; j < 3; ++j) F.M[3 * i + j] = (float)(R[i][j] / Bd);
    F.o[i] = (float)((t[i] - (double)a[i] * Bd) / Bd);
    F.a[i] = (int32_t)a[i];
  }
  return true;
}

bool valid_pinhole(const tsdf_pinhole* c) {
  return c && c->width > 0 && c->height > 0 && (int64_t)c->width * c->height < (1ll << 30) &&
         std::isfinite(c->fu) && std::isfinite(c->fv) && std::isfinite(c->cu) &&
         std::isfinite(c->cv) && c->fu != 0.0f && c->fv != 0.0f;
}

bool valid_lidar(const tsdf_lidar* c) {
  return c && c->n_az > 0 && c->n_el > 1 && (int64_t)c->n_az * c->n_el < (1ll << 30) &&
         std::isfinite(c->theta_start) && std::isfinite(c->phi_start) &&
         std::isfinite(c->el_fov) && c->el_fov > 0.0f && std::isfinite(c->min_range) &&
         std::isfinite(c->max_range) && c->min_range <= c->max_range;
}

// Exponent of the last place of a nonzero FP32 value (subnormals: -149).
int lsb_exp(float x) {
  int e = 0;
  std::frexp(x, &e);  // |x| = f 2^e, f in [0.5, 1)
  return std::max(e - 24, -149);
}

constexpr double kTwo126 = 8.507059173023462e37;  // 2^126

// Range check for the kernels' fast reciprocal (rcp_dec<true>, exact for
// |x| in [2^-126, 2^126]).  Every value a frame's decisions invert is an
// FMA chain of FP32 terms, sum_k a_k b_k + c: a traversal direction
// component d = M_k0 r_x + (M_k1 r_y + M_k2) (pinhole, r the pixel's ray)
// or M_k0 b_x + (M_k1 b_y + RN(M_k2 b_z)) (LiDAR, b the beam direction), and
// a voxel depth z = R_20 q_x + (R_21 q_y + (R_22 q_z + t_2)) (pinhole
// projection; q the voxel centre, |q| >= v / 2).  The exact sum is a
// multiple of 2^L, L the smallest last-place exponent among the products
// (lsb a + lsb b) and the addend, and each rounding in the chain keeps it
// so, hence a nonzero result has magnitude >= 2^L.  With L >= -126 and the
// magnitudes bounded below 2^126 every nonzero value is in range; zeros are
// never inverted (a zero direction component has no crossing, z <= 0 fails
// the projection test).  lidar_lsb: the table's smallest beam-component
// last-place exponent.
bool fast_rcp_ok(const FrameDev& F, double v, int lidar_lsb) {
  int lsb_m = INT_MAX;
  double max_m = 0.0;
  for (int i = 0; i < 9; ++i)
    if (F.M[i] != 0.0f) {
      lsb_m = std::min(lsb_m, lsb_exp(F.M[i]));
      max_m = std::max(max_m, (double)std::fabs(F.M[i]));
    }
  if (lsb_m == INT_MAX) return false;
  if (F.kind == TSDF_SENSOR_PINHOLE) {
    // pixel ray components r = (i - c) / f, as the allocation kernel forms
    // them: monotone in i (every rounding is), so the largest |r| is at an
    // image edge and the smallest nonzero |r| next to the principal point;
    // those few pixels bound the whole image
    int lsb_r = INT_MAX;
    double max_r = 1.0;
    auto bound = [&](int n, float c, float f) {
      const double cl = std::floor((double)c);
      const int cand[6] = {0, n - 1, (int)std::max(-1.0, std::min((double)n, cl - 1.0)),
                           (int)std::max(-1.0, std::min((double)n, cl)),
                           (int)std::max(-1.0, std::min((double)n, cl + 1.0)),
                           (int)std::max(-1.0, std::min((double)n, cl + 2.0))};
      for (int i : cand) {
        if (i < 0 || i >= n) continue;
        const float r = ((float)i - c) / f;
        if (r != 0.0f) lsb_r = std::min(lsb_r, lsb_exp(r));
        max_r = std::max(max_r, (double)std::fabs(r));
      }
    };
    bound(F.width, F.cu, F.fu);
    bound(F.height, F.cv, F.fv);
    const int L = std::min(lsb_m, lsb_r == INT_MAX ? lsb_m : lsb_m + lsb_r);
    if (L < -126 || 3.0 * max_m * max_r * (1.0 + 1e-6) >= kTwo126) return false;
    // projection: z of a voxel centre
    int lsb_rc = INT_MAX;
    double max_rc = 0.0;
    for (int j = 6; j < 9; ++j)
      if (F.Rcl[j] != 0.0f) {
        lsb_rc = std::min(lsb_rc, lsb_exp(F.Rcl[j]));
        max_rc = std::max(max_rc, (double)std::fabs(F.Rcl[j]));
      }
    const float half_v = 0.5f * (float)v;  // the smallest |q| (q = (rel + 1/2) v, rel an integer)
    if (!(half_v >= 1.17549435e-38f)) return false;
    int L2 = lsb_rc == INT_MAX ? INT_MAX : lsb_rc + lsb_exp(half_v);
    if (F.tloc[2] != 0.0f) L2 = std::min(L2, lsb_exp(F.tloc[2]));
    const double max_q = (16777216.0 + 16.0) * (double)(float)v * (1.0 + 1e-6);  // |rel| < 2^24 + 8
    if (L2 < -126 || 3.0 * max_rc * max_q + std::fabs((double)F.tloc[2]) >= kTwo126) return false;
    return true;
  }
  const int L = lidar_lsb == INT_MAX ? lsb_m : lsb_m + lidar_lsb;  // beam components are at most 1
  return L >= -126 && 3.0 * max_m * (1.0 + 1e-6) < kTwo126;
}

// Whether every band segment of frame F provably meets fewer than
// kMaxCells blocks, so the allocation kernel may walk without the cap.  A
// segment spans s1 - s0 <= 2 tau of depth or range (plus at most d 2^-23 from
// rounding its two ends, under 0.06 blocks at the distances walked) along a
// direction of length |r| / B in blocks per unit, r = (rx, ry, 1) for a
// pinhole pixel (largest at an image corner) and a unit beam for a LiDAR:
// L <= (2 tau / B) |r| = (trunc / 4) |r| blocks.  Along each axis the FP32
// traversal crosses at most |dp_k| + 2 boundaries (the three roundings of a
// crossing parameter and the rounded start point move a boundary test by
// less than one cell), so a segment meets at most 7 + sqrt(3) (L + 0.06)
// cells; L <= 8 keeps that under 22.
bool short_walks_ok(const FrameDev& F, int32_t trunc) {
  double r2 = 1.0;
  if (F.kind == TSDF_SENSOR_PINHOLE) {
    const double ax = std::max(std::fabs(-(double)F.cu / (double)F.fu),
                               std::fabs(((double)F.width - 1.0 - (double)F.cu) / (double)F.fu));
    const double ay = std::max(std::fabs(-(double)F.cv / (double)F.fv),
                               std::fabs(((double)F.height - 1.0 - (double)F.cv) / (double)F.fv));
    r2 += ax * ax + ay * ay;
  }
  return 0.25 * (double)trunc * std::sqrt(r2) * (1.0 + 1e-3) <= 8.0;
}

// Beam-centre direction tables of a LiDAR (Eq. 3 inverted at the cell
// centres), computed in FP64 and rounded once; uploaded on first use.
tsdf_status lidar_table(tsdf_map* m, const tsdf_lidar* c, const float** out, int* lsb) {
  for (const LidarTable& t : m->tables)
    if (t.n_az == c->n_az && t.n_el == c->n_el && t.theta_start == c->theta_start &&
        t.phi_start == c->phi_start && t.el_fov == c->el_fov) {
      *out = t.dev;
      *lsb = t.lsb;
      return TSDF_OK;
    }
  std::vector<float> h(2 * ((size_t)c->n_az + c->n_el));
  for (int k = 0; k < c->n_az; ++k) {
    const double th = (double)c->theta_start + ((double)k + 0.5) * (6.283185307179586 / (double)c->n_az);
    h[2 * k] = (float)std::cos(th);
    h[2 * k + 1] = (float)std::sin(th);
  }
  for (int j = 0; j < c->n_el; ++j) {
    const double ph = (double)c->phi_start + ((double)j + 0.5) * ((double)c->el_fov / (double)c->n_el);
    h[2 * (c->n_az + j)] = (float)std::cos(ph);
    h[2 * (c->n_az + j) + 1] = (float)std::sin(ph);
  }
  // beam direction components the traversal uses: sin(polar) cos / sin(azimuth)
  // (FP32 products, as the kernel forms them) and cos(polar)
  int low = INT_MAX;
  auto note = [&low](float x) {
    if (x != 0.0f) low = std::min(low, lsb_exp(x));
  };
  for (int j = 0; j < c->n_el; ++j) {
    const float sp = h[2 * (c->n_az + j) + 1];
    note(h[2 * (c->n_az + j)]);
    for (int k = 0; k < c->n_az; ++k) {
      note(sp * h[2 * k]);
      note(sp * h[2 * k + 1]);
    }
  }
  LidarTable t{c->n_az, c->n_el, c->theta_start, c->phi_start, c->el_fov, nullptr, low};
  if (cudaMalloc(&t.dev, h.size() * sizeof(float)) != cudaSuccess) return cuda_fail();
  if (cudaMemcpy(t.dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(t.dev);
    return cuda_fail();
  }
  m->tables.push_back(t);
  *out = t.dev;
  *lsb = t.lsb;
  return TSDF_OK;
}

// A colour map takes pinhole frames with a colour image; other maps take no
// colour image.
tsdf_status fill_frame(tsdf_map* m, int map_index, int kind, const tsdf_pinhole* ph,
                       const tsdf_lidar* li, const float* depth, const uint32_t* rgba,
                       const double* T, FrameDev& F) {
  std::memset(&F, 0, sizeof(F));
  int lidar_lsb = INT_MAX;
  if (!depth || !T || !rigid(T)) return TSDF_ERR_ARG;
  const bool color = m->storage == gbt::kStorageColor;
  if (color != (rgba != nullptr) || (color && kind != TSDF_SENSOR_PINHOLE)) return TSDF_ERR_ARG;
  F.kind = kind;
  F.map = map_index;
  F.depth = depth;
  F.rgba = rgba;
  if (kind == TSDF_SENSOR_PINHOLE) {
    if (!valid_pinhole(ph)) return TSDF_ERR_ARG;
    F.width = ph->width;
    F.height = ph->height;
    F.fu = ph->fu;
    F.fv = ph->fv;
    F.cu = ph->cu;
    F.cv = ph->cv;
  } else if (kind == TSDF_SENSOR_LIDAR) {
    if (!valid_lidar(li)) return TSDF_ERR_ARG;
    F.width = li->n_az;
    F.height = li->n_el;
    F.theta_start = li->theta_start;
    F.phi_start = li->phi_start;
    F.alpha = (float)((double)li->n_az / 6.283185307179586);  // pixels per radian
    F.beta = (float)((double)li->n_el / (double)li->el_fov);
    F.min_range = li->min_range;
    F.max_range = li->max_range;
    tsdf_status st = lidar_table(m, li, &F.tab, &lidar_lsb);
    if (st != TSDF_OK) return st;
  } else {
    return TSDF_ERR_ARG;
  }
  if (!prepare_pose(m->Bd, T, F)) return TSDF_ERR_ARG;
  F.fast_rcp = fast_rcp_ok(F, m->vd, lidar_lsb) ? 1 : 0;
  F.short_walks = short_walks_ok(F, m->trunc) ? 1 : 0;
  return TSDF_OK;
}

size_t voxel_size_bytes(int storage) {
  return storage == gbt::kStorageColor ? 16 : storage == TSDF_STORAGE_FP32 ? 8 : 4;  // FP16, fixed 16, occupancy
}

int alloc_ctas(const FrameDev& F, int tile_h) {
  return ((F.width + gbt::kTileW - 1) / gbt::kTileW) * ((F.height + tile_h - 1) / tile_h);
}

int pick_tile_h(int64_t pixels) {
  return pixels >= gbt::kBigTilePixels ? gbt::kTileHBig : gbt::kTileHSmall;
}

bool on_device(const tsdf_map* m) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == m->device;
}

// Next free event quadruple when timing is enabled, else nullptr.
cudaEvent_t* timing_slot(tsdf_map* m) {
  if (!m->timing || m->n_timed >= kTimedCalls) return nullptr;
  return &m->events[4 * m->n_timed++];
}

// Device view of map m using mask / list / control set `set` (0 or 1).
MapDev view_set(const tsdf_map* m, int set) {
  MapDev d = m->dev;
  if (set) {
    d.mask = m->mask1;
    d.list = m->list1;
    d.ctl = m->ctl1;
  }
  return d;
}

tsdf_status integrate_one(tsdf_map* m, int kind, const tsdf_pinhole* ph, const tsdf_lidar* li,
                          const float* depth, const uint32_t* rgba, const double* T, void* stream) {
  if (!m) return TSDF_ERR_ARG;
  if (!on_device(m)) return TSDF_ERR_STATE;
  if (status_from_bits(m->status_seen) != TSDF_OK) return status_from_bits(m->status_seen);
  BatchParams<1, 1> p;
  std::memset(&p, 0, sizeof(p));
  p.n_frames = 1;
  p.n_maps = 1;
  p.maps[0] = m->dev;
  tsdf_status st = fill_frame(m, 0, kind, ph, li, depth, rgba, T, p.fr[0]);
  if (st != TSDF_OK) return st;
  p.fr[0].blk_begin = 0;
  p.fr[0].bit = 0;
  p.fast_rcp = p.fr[0].fast_rcp;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t* ev = timing_slot(m);
  if (ev) cudaEventRecord(ev[0], s);
  const int th = m->tile_h ? m->tile_h : pick_tile_h((int64_t)p.fr[0].width * p.fr[0].height);
  // one frame per call: each launch may be scheduled while the stream's
  // previous kernel finishes (both kernels wait for it before touching memory)
  p.overlap = 1;
  if (gbt::launch_band_alloc(p, alloc_ctas(p.fr[0], th), th, s) != cudaSuccess) return cuda_fail();
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  if (gbt::launch_integrate(p, m->n_ctas_integrate, s) != cudaSuccess) return cuda_fail();
  if (ev) cudaEventRecord(ev[3], s);
  m->frames += 1;
  return TSDF_OK;
}

tsdf_status read_counters(const tsdf_map* m, unsigned long long c[gbt::kNumCounters]) {
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail();
  if (cudaMemcpy(c, m->dev.counters, sizeof(unsigned long long) * gbt::kNumCounters,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail();
  const_cast<tsdf_map*>(m)->status_seen |= c[gbt::kCntStatus];
  return TSDF_OK;
}

void free_map(tsdf_map* m) {
  cudaFree(m->mask1);
  cudaFree(m->list1);
  cudaFree(m->ctl1);
  cudaFree(m->dev.dirty);
  if (m->mesh_on) {
    cudaFree(m->mesh.list);
    cudaFree(m->mesh.stamp);
    cudaFree(m->mesh.cnt);
  }
  if (m->esdf_on) {
    cudaFree(m->esdf.st);
    cudaFree(m->esdf.st2);
    cudaFree(m->esdf.list[0]);
    cudaFree(m->esdf.list[1]);
    cudaFree(m->esdf.tlist[0]);
    cudaFree(m->esdf.tlist[1]);
    cudaFree(m->esdf.nbr);
    cudaFree(m->esdf.clist);
    cudaFree(m->esdf.stamp_s);
    cudaFree(m->esdf.stamp_t);
    cudaFree(m->esdf.tchanged);
    cudaFree(m->esdf.bits);
    cudaFree(m->esdf.cnt);
    cudaFree(m->esdf.stats);
    cudaFreeHost(m->esdf_host);
  }
  if (m->aux) cudaStreamDestroy(m->aux);
  if (m->copy) cudaStreamDestroy(m->copy);
  for (int i = 0; i < 4; ++i)
    if (m->ev_copy[i]) cudaEventDestroy(m->ev_copy[i]);
  for (int i = 0; i < 4; ++i) {
    if (m->ev_alloc[i]) cudaEventDestroy(m->ev_alloc[i]);
    if (m->ev_int[i]) cudaEventDestroy(m->ev_int[i]);
  }
  if (m->ev_start) cudaEventDestroy(m->ev_start);
  cudaFree(m->dev.keys);
  cudaFree(m->dev.vals);
  cudaFree(m->dev.mask);
  cudaFree(m->dev.pool);
  cudaFree(m->dev.block_keys);
  cudaFree(m->dev.counters);
  cudaFree(m->dev.list);
  cudaFree(m->dev.ctl);
  for (LidarTable& t : m->tables) cudaFree(t.dev);
  for (cudaEvent_t e : m->events) cudaEventDestroy(e);
  delete m;
}

}  // namespace

extern "C" {

tsdf_status map_create_ex(float voxel_size, int32_t truncation_voxels, float max_weight,
                          const tsdf_map_opts* opts, tsdf_map** out) {
  if (!out || !(voxel_size > 0.0f) || !std::isfinite(voxel_size) || truncation_voxels <= 0 ||
      !(max_weight > 0.0f) || !std::isfinite(max_weight))
    return TSDF_ERR_ARG;
  tsdf_map_opts o{TSDF_STORAGE_FP32, kDefaultBlocks, 0, 0, 0.0f, 0, 0, TSDF_LAYER_TSDF, 0.0f, 0.0f,
                  TSDF_WEIGHT_CONSTANT, 0.0f};
  if (opts) o = *opts;
  if (o.weighting < 0 || o.weighting > 3 || !std::isfinite(o.dropoff)) return TSDF_ERR_ARG;
  if ((o.weighting & TSDF_WEIGHT_DROPOFF) &&
      !((o.dropoff > 0.0f ? o.dropoff : voxel_size) < (float)((double)truncation_voxels * voxel_size)))
    return TSDF_ERR_ARG;  // the drop-off must start in front of -tau
  if (o.layer != TSDF_LAYER_TSDF && o.layer != TSDF_LAYER_OCCUPANCY && o.layer != TSDF_LAYER_COLOR)
    return TSDF_ERR_ARG;
  if (!std::isfinite(o.l_occ) || !std::isfinite(o.l_free)) return TSDF_ERR_ARG;
  if (o.layer == TSDF_LAYER_OCCUPANCY) {
    o.storage = gbt::kStorageOcc;
    if (o.l_occ == 0.0f && o.l_free == 0.0f) {
      o.l_occ = 0.85f;
      o.l_free = -0.4f;
    }
  }
  if (o.layer == TSDF_LAYER_COLOR) {
    o.storage = gbt::kStorageColor;
    o.weighting = TSDF_WEIGHT_CONSTANT;
  }
  if (o.alloc_tile_h != 0 && o.alloc_tile_h != gbt::kTileHSmall && o.alloc_tile_h != gbt::kTileHBig)
    return TSDF_ERR_ARG;
  if (o.integrate_ctas_per_sm < 0) return TSDF_ERR_ARG;
  if (o.launch_mode != TSDF_LAUNCH_SPLIT && o.launch_mode != TSDF_LAUNCH_FUSED) return TSDF_ERR_ARG;
  if (o.storage != TSDF_STORAGE_FP32 && o.storage != TSDF_STORAGE_FP16 && o.storage != TSDF_STORAGE_FIXED16 &&
      o.storage != gbt::kStorageOcc && o.storage != gbt::kStorageColor)
    return TSDF_ERR_ARG;
  if ((o.storage == gbt::kStorageOcc) != (o.layer == TSDF_LAYER_OCCUPANCY) ||
      (o.storage == gbt::kStorageColor) != (o.layer == TSDF_LAYER_COLOR))
    return TSDF_ERR_ARG;  // internal storage kinds go with their layer
  if (o.max_blocks <= 0) o.max_blocks = kDefaultBlocks;
  if (o.max_blocks > (1ll << 27)) return TSDF_ERR_ARG;
  int64_t cap = 1;
  while (cap < std::max<int64_t>(2 * o.max_blocks, o.hash_capacity)) cap <<= 1;
  if (cap > (1ll << 30)) return TSDF_ERR_ARG;

  tsdf_map* m = new tsdf_map();
  std::memset(&m->dev, 0, sizeof(m->dev));
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return cuda_fail();
  }
  m->cap = (uint32_t)cap;
  m->max_blocks = o.max_blocks;
  m->storage = o.storage;
  m->v = voxel_size;
  m->wmax = max_weight;
  m->trunc = truncation_voxels;
  m->vd = (double)voxel_size;
  m->Bd = 8.0 * m->vd;
  m->frames = 0;
  m->status_seen = 0;
  m->timing = false;
  m->n_timed = 0;
  MapDev& d = m->dev;
  d.cap_mask = (uint32_t)(cap - 1);
  d.max_blocks = (int32_t)o.max_blocks;
  d.list_cap = (uint32_t)o.max_blocks;
  d.storage = o.storage;
  d.lidar_nearest = o.lidar_nearest ? 1 : 0;
  d.walk_stats = 0;
  d.v = voxel_size;
  d.tau = (float)((double)truncation_voxels * m->vd);
  d.inv_tau = 1.0f / d.tau;
  d.x16_scale = (float)((double)gbt::kX16Steps / (double)d.tau);
  d.x16_unit = (float)((double)d.tau / (double)gbt::kX16Steps);
  d.wmax = max_weight;
  d.guard = o.lidar_guard > 0.0f ? o.lidar_guard : d.tau;
  d.l_occ = o.l_occ;
  d.l_free = o.l_free;
  d.weighting = o.weighting;
  d.dropoff = o.dropoff > 0.0f ? o.dropoff : voxel_size;
  const size_t voxel_bytes = voxel_size_bytes(o.storage);
  bool ok = cudaMalloc(&d.keys, sizeof(unsigned long long) * cap) == cudaSuccess &&
            cudaMalloc(&d.vals, sizeof(int32_t) * cap) == cudaSuccess &&
            cudaMalloc(&d.mask, sizeof(uint32_t) * cap) == cudaSuccess &&
            cudaMalloc(&d.pool, voxel_bytes * gbt::kBlockVoxels * o.max_blocks) == cudaSuccess &&
            cudaMalloc(&d.block_keys, sizeof(unsigned long long) * o.max_blocks) == cudaSuccess &&
            cudaMalloc(&d.counters, sizeof(unsigned long long) * gbt::kNumCounters) == cudaSuccess &&
            cudaMalloc(&d.list, sizeof(uint32_t) * o.max_blocks) == cudaSuccess &&
            cudaMalloc(&d.ctl, sizeof(unsigned int) * 4) == cudaSuccess &&
            cudaMalloc(&m->mask1, sizeof(uint32_t) * cap) == cudaSuccess &&
            cudaMalloc(&m->list1, sizeof(uint32_t) * o.max_blocks) == cudaSuccess &&
            cudaMalloc(&m->ctl1, sizeof(unsigned int) * 4) == cudaSuccess &&
            cudaMalloc(&d.dirty, (size_t)o.max_blocks) == cudaSuccess &&
            cudaStreamCreateWithFlags(&m->aux, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < 4; ++i)
    ok = cudaEventCreateWithFlags(&m->ev_alloc[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&m->ev_int[i], cudaEventDisableTiming) == cudaSuccess;
  if (ok)
    ok = gbt::launch_reset(d, m->cap, 0) == cudaSuccess &&
         cudaMemsetAsync(m->mask1, 0, sizeof(uint32_t) * cap, 0) == cudaSuccess &&
         cudaMemsetAsync(m->ctl1, 0, sizeof(unsigned int) * 4, 0) == cudaSuccess &&
         cudaMemsetAsync(d.dirty, 0, (size_t)o.max_blocks, 0) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    free_map(m);
    return cuda_fail();
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  int per_sm = gbt::integrate_ctas_per_sm(o.storage);
  if (o.integrate_ctas_per_sm > 0) per_sm = std::min(per_sm, o.integrate_ctas_per_sm);
  m->n_ctas_integrate = std::max(1, sms) * per_sm;
  m->tile_h = o.alloc_tile_h;
  m->launch_mode = o.launch_mode;
  m->wait_extra = 0;
  *out = m;
  return TSDF_OK;
}

tsdf_status map_create(float voxel_size, int32_t truncation_voxels, float max_weight,
                       tsdf_map** out) {
  return map_create_ex(voxel_size, truncation_voxels, max_weight, nullptr, out);
}

tsdf_status integrate_depth(tsdf_map* map, const float* depth_dev, const tsdf_pinhole* intr,
                            const double T_world_cam[16], void* cuda_stream) {
  return integrate_one(map, TSDF_SENSOR_PINHOLE, intr, nullptr, depth_dev, nullptr, T_world_cam,
                       cuda_stream);
}

tsdf_status integrate_color(tsdf_map* map, const float* depth_dev, const uint32_t* color_dev,
                            const tsdf_pinhole* intr, const double T_world_cam[16],
                            void* cuda_stream) {
  if (!map || !color_dev || map->storage != gbt::kStorageColor) return TSDF_ERR_ARG;
  return integrate_one(map, TSDF_SENSOR_PINHOLE, intr, nullptr, depth_dev, color_dev, T_world_cam,
                       cuda_stream);
}

tsdf_status integrate_lidar(tsdf_map* map, const float* range_dev, const tsdf_lidar* intr,
                            const double T_world_lidar[16], void* cuda_stream) {
  return integrate_one(map, TSDF_SENSOR_LIDAR, nullptr, intr, range_dev, nullptr, T_world_lidar,
                       cuda_stream);
}

}  // extern "C"

namespace {

// Checks the maps and frames of a batch and prepares every frame (FP32 pose
// constants, sensor tables) before anything is enqueued.
tsdf_status prepare_batch(tsdf_map* const* maps, int32_t n_maps, const tsdf_frame_desc* frames, int32_t n,
                          std::vector<FrameDev>& fr) {
  if (!maps || !frames || n_maps <= 0 || n_maps > gbt::kMaxMaps || n <= 0 || n > kMaxBatchFrames)
    return TSDF_ERR_ARG;
  for (int i = 0; i < n_maps; ++i) {
    if (!maps[i]) return TSDF_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (maps[j] == maps[i]) return TSDF_ERR_ARG;
    if (maps[i]->storage != maps[0]->storage) return TSDF_ERR_ARG;
    if (!on_device(maps[i])) return TSDF_ERR_STATE;
    if (status_from_bits(maps[i]->status_seen) != TSDF_OK) return status_from_bits(maps[i]->status_seen);
  }
  fr.resize(n);
  for (int f = 0; f < n; ++f) {
    const tsdf_frame_desc& fd = frames[f];
    if (fd.map < 0 || fd.map >= n_maps) return TSDF_ERR_ARG;
    tsdf_status st = fill_frame(maps[fd.map], fd.map, fd.kind, &fd.pinhole, &fd.lidar,
                                fd.depth_dev, fd.color_dev, fd.T_world_sensor, fr[f]);
    if (st != TSDF_OK) return st;
  }
  return TSDF_OK;
}

// Called before sub-batch b (frames f0 .. f0 + nf - 1) is filled in and its
// allocation is enqueued on stream sa; may rewrite the frames' image
// pointers and make sa wait for copies.
using SubBatchHook = tsdf_status (*)(void* ctx, int b, int f0, int nf, cudaStream_t sa);

// Sub-batches of up to 32 frames, each one allocation launch and one
// integration launch.  With more than one, sub-batch b uses mask / list set
// b % 2 and its allocation runs on the lead map's auxiliary stream,
// overlapping the integration of sub-batch b - 1 on the caller's stream; it
// waits for the integration of b - 2, which used the same set.
tsdf_status run_batch(tsdf_map* const* maps, int32_t n_maps, std::vector<FrameDev>& fr, int32_t n,
                      cudaStream_t s, SubBatchHook hook, void* ctx) {
  // the params block is large; keep it off the stack
  static thread_local BatchParams<gbt::kMaxFrames, gbt::kMaxMaps> p;
  // single-map batches launch the one-map kernels (map fields become constants)
  static thread_local BatchParams<gbt::kMaxFrames, 1> p1;
  tsdf_map* lead = maps[0];
  const int n_sub = (n + gbt::kMaxFrames - 1) / gbt::kMaxFrames;
  if (lead->launch_mode == TSDF_LAUNCH_FUSED && n_maps == 1) {
    // one cooperative launch per sub-batch, on the caller's stream
    for (int b = 0; b < n_sub; ++b) {
      const int f0 = b * gbt::kMaxFrames, nf = std::min(gbt::kMaxFrames, n - f0);
      if (hook) {
        tsdf_status st = hook(ctx, b, f0, nf, s);
        if (st != TSDF_OK) return st;
      }
      std::memset(&p1, 0, sizeof(p1));
      p1.n_frames = nf;
      p1.n_maps = 1;
      p1.maps[0] = view_set(lead, 0);
      int64_t pixels = 0;
      for (int f = 0; f < nf; ++f) {
        p1.fr[f] = fr[f0 + f];
        p1.fr[f].bit = f;
        pixels += (int64_t)p1.fr[f].width * p1.fr[f].height;
      }
      const int th = lead->tile_h ? lead->tile_h : pick_tile_h(pixels);
      int ctas = 0;
      for (int f = 0; f < nf; ++f) {
        p1.fr[f].blk_begin = ctas;
        ctas += alloc_ctas(p1.fr[f], th);
      }
      p1.alloc_ctas = ctas;
      p1.wait_extra = lead->wait_extra;
      p1.fast_rcp = 1;
      for (int f = 0; f < nf; ++f) p1.fast_rcp &= p1.fr[f].fast_rcp;
      cudaEvent_t* ev = timing_slot(lead);
      if (ev) cudaEventRecord(ev[0], s);
      cudaError_t err = gbt::launch_fused(p1, th, s);
      if (err == cudaErrorNotSupported) {  // not a fused batch: the two kernels
        cudaGetLastError();
        p1.overlap = 1;
        if (gbt::launch_band_alloc(p1, ctas, th, s) != cudaSuccess) return cuda_fail();
        if (ev) {
          cudaEventRecord(ev[1], s);
          cudaEventRecord(ev[2], s);
        }
        if (gbt::launch_integrate(p1, lead->n_ctas_integrate, s) != cudaSuccess) return cuda_fail();
        if (ev) cudaEventRecord(ev[3], s);
        if (cudaEventRecord(lead->ev_int[b & 3], s) != cudaSuccess) return cuda_fail();
        continue;
      }
      if (err != cudaSuccess) return cuda_fail();
      if (ev) {  // the whole launch counts as allocation time
        cudaEventRecord(ev[1], s);
        cudaEventRecord(ev[2], s);
        cudaEventRecord(ev[3], s);
      }
      // host-image staging reuses this sub-batch's slot after this event
      if (cudaEventRecord(lead->ev_int[b & 3], s) != cudaSuccess) return cuda_fail();
    }
    return TSDF_OK;
  }
  const bool piped = n_sub > 1;
  if (piped && (cudaEventRecord(lead->ev_start, s) != cudaSuccess ||
                cudaStreamWaitEvent(lead->aux, lead->ev_start, 0) != cudaSuccess))
    return cuda_fail();
  for (int b = 0; b < n_sub; ++b) {
    const int f0 = b * gbt::kMaxFrames, nf = std::min(gbt::kMaxFrames, n - f0);
    cudaStream_t sa = piped ? lead->aux : s;
    if (piped && b >= 2 && cudaStreamWaitEvent(sa, lead->ev_int[(b - 2) & 3], 0) != cudaSuccess)
      return cuda_fail();
    if (hook) {
      tsdf_status st = hook(ctx, b, f0, nf, sa);
      if (st != TSDF_OK) return st;
    }
    std::memset(&p, 0, sizeof(p));
    p.n_frames = nf;
    p.n_maps = n_maps;
    for (int i = 0; i < n_maps; ++i) p.maps[i] = view_set(maps[i], piped ? (b & 1) : 0);
    int64_t pixels = 0;
    p.fast_rcp = 1;
    for (int f = 0; f < nf; ++f) {
      p.fr[f] = fr[f0 + f];
      p.fr[f].bit = f;
      p.fast_rcp &= p.fr[f].fast_rcp;
      pixels += (int64_t)p.fr[f].width * p.fr[f].height;
    }
    const int th = lead->tile_h ? lead->tile_h : pick_tile_h(pixels);
    int ctas = 0;
    for (int f = 0; f < nf; ++f) {
      p.fr[f].blk_begin = ctas;
      ctas += alloc_ctas(p.fr[f], th);
    }
    cudaEvent_t* ev = timing_slot(lead);
    if (ev) cudaEventRecord(ev[0], sa);
    if (n_maps == 1) {
      p1.n_frames = p.n_frames;
      p1.n_maps = 1;
      p1.fast_rcp = p.fast_rcp;
      p1.maps[0] = p.maps[0];
      std::memcpy(p1.fr, p.fr, sizeof(p.fr));
    }
    // a single sub-batch runs both kernels back to back on one stream: each
    // may be scheduled while its predecessor drains (see integrate_one)
    p.overlap = p1.overlap = piped ? 0 : 1;
    if ((n_maps == 1 ? gbt::launch_band_alloc(p1, ctas, th, sa) : gbt::launch_band_alloc(p, ctas, th, sa)) !=
        cudaSuccess)
      return cuda_fail();
    if (ev) cudaEventRecord(ev[1], sa);
    if (piped && (cudaEventRecord(lead->ev_alloc[b & 3], sa) != cudaSuccess ||
                  cudaStreamWaitEvent(s, lead->ev_alloc[b & 3], 0) != cudaSuccess))
      return cuda_fail();
    if (ev) cudaEventRecord(ev[2], s);
    if ((n_maps == 1 ? gbt::launch_integrate(p1, lead->n_ctas_integrate, s)
                     : gbt::launch_integrate(p, lead->n_ctas_integrate, s)) != cudaSuccess)
      return cuda_fail();
    if (ev) cudaEventRecord(ev[3], s);
    if (piped && cudaEventRecord(lead->ev_int[b & 3], s) != cudaSuccess) return cuda_fail();
  }
  return TSDF_OK;
}

// Host-input batches: the images of sub-batch b are copied from host memory
// into slot b % slots of the caller's staging buffer on the lead map's copy
// stream (one copy per run of frames contiguous in host memory), after the
// integration of sub-batch b - slots, which read that slot; the sub-batch's
// allocation waits for its copies.  With more slots the copies run further
// ahead of the kernels.
struct HostStaging {
  tsdf_map* lead;
  std::vector<FrameDev>* fr;
  char* base;
  int64_t half;                  // bytes per slot of the staging buffer
  int slots;                     // 2 .. 4
  std::vector<int64_t> off;      // per frame: depth offset in its half (colour follows)
  std::vector<int64_t> bytes;    // per frame: depth bytes
};

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

tsdf_status stage_sub_batch(void* ctx, int b, int f0, int nf, cudaStream_t sa) {
  HostStaging& h = *static_cast<HostStaging*>(ctx);
  tsdf_map* lead = h.lead;
  std::vector<FrameDev>& fr = *h.fr;
  cudaStream_t c = lead->copy;
  if (b >= h.slots && cudaStreamWaitEvent(c, lead->ev_int[(b - h.slots) & 3], 0) != cudaSuccess)
    return cuda_fail();
  char* half = h.base + (int64_t)(b % h.slots) * h.half;
  // copy runs of frames whose images are contiguous both on the host and in the half
  int f = f0;
  while (f < f0 + nf) {
    const char* src = reinterpret_cast<const char*>(fr[f].depth);
    int64_t len = h.bytes[f];
    int g = f + 1;
    while (g < f0 + nf && !fr[g].rgba && !fr[f].rgba &&
           reinterpret_cast<const char*>(fr[g].depth) == src + len && h.off[g] == h.off[f] + len) {
      len += h.bytes[g];
      ++g;
    }
    if (cudaMemcpyAsync(half + h.off[f], src, (size_t)len, cudaMemcpyHostToDevice, c) != cudaSuccess)
      return cuda_fail();
    for (int k = f; k < g; ++k) {
      if (fr[k].rgba &&
          cudaMemcpyAsync(half + h.off[k] + h.bytes[k], fr[k].rgba, (size_t)h.bytes[k], cudaMemcpyHostToDevice,
                          c) != cudaSuccess)
        return cuda_fail();
      fr[k].depth = reinterpret_cast<const float*>(half + h.off[k]);
      if (fr[k].rgba) fr[k].rgba = reinterpret_cast<const uint32_t*>(half + h.off[k] + h.bytes[k]);
    }
    f = g;
  }
  if (cudaEventRecord(lead->ev_copy[b & 3], c) != cudaSuccess ||
      cudaStreamWaitEvent(sa, lead->ev_copy[b & 3], 0) != cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

}  // namespace

extern "C" {

tsdf_status integrate_batch(tsdf_map* const* maps, int32_t n_maps, const tsdf_frame_desc* frames,
                            int32_t n, void* cuda_stream) {
  static thread_local std::vector<FrameDev> fr;
  tsdf_status st = prepare_batch(maps, n_maps, frames, n, fr);
  if (st != TSDF_OK) return st;
  st = run_batch(maps, n_maps, fr, n, (cudaStream_t)cuda_stream, nullptr, nullptr);
  if (st != TSDF_OK) return st;
  for (int f = 0; f < n; ++f) maps[frames[f].map]->frames += 1;
  return TSDF_OK;
}

tsdf_status integrate_batch_host(tsdf_map* const* maps, int32_t n_maps, const tsdf_frame_desc* frames,
                                 int32_t n, void* staging_dev, int64_t staging_bytes, void* cuda_stream) {
  static thread_local std::vector<FrameDev> fr;
  tsdf_status st = prepare_batch(maps, n_maps, frames, n, fr);
  if (st != TSDF_OK) return st;
  if (!staging_dev || staging_bytes <= 0 || (reinterpret_cast<uintptr_t>(staging_dev) & 255u)) return TSDF_ERR_ARG;
  HostStaging h;
  h.lead = maps[0];
  h.fr = &fr;
  h.base = static_cast<char*>(staging_dev);
  h.off.resize(n);
  h.bytes.resize(n);
  int64_t need = 0;
  for (int f0 = 0; f0 < n; f0 += gbt::kMaxFrames) {
    int64_t o = 0;
    for (int f = f0; f < std::min(n, f0 + gbt::kMaxFrames); ++f) {
      h.bytes[f] = (int64_t)fr[f].width * fr[f].height * 4;
      h.off[f] = o;
      o += align256(h.bytes[f]) * (fr[f].rgba ? 2 : 1);
    }
    need = std::max(need, o);
  }
  h.half = align256(need);
  if (2 * h.half > staging_bytes) return TSDF_ERR_ARG;  // two sub-batches must fit
  h.slots = (int)std::min<int64_t>(4, staging_bytes / h.half);
  tsdf_map* lead = maps[0];
  if (!lead->copy) {
    bool ok = cudaStreamCreateWithFlags(&lead->copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < 4; ++i)
      ok = cudaEventCreateWithFlags(&lead->ev_copy[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_fail();
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the copies start after the caller's earlier work on the stream (which may
  // still read the staging buffer)
  if (cudaEventRecord(lead->ev_start, s) != cudaSuccess ||
      cudaStreamWaitEvent(lead->copy, lead->ev_start, 0) != cudaSuccess)
    return cuda_fail();
  st = run_batch(maps, n_maps, fr, n, s, stage_sub_batch, &h);
  if (st != TSDF_OK) return st;
  for (int f = 0; f < n; ++f) maps[frames[f].map]->frames += 1;
  return TSDF_OK;
}

tsdf_status stage_frames(const void* const* src_host, void* const* dst_dev, const int64_t* bytes, int32_t n,
                         void* cuda_stream) {
  if (n < 0 || (n > 0 && (!src_host || !dst_dev || !bytes))) return TSDF_ERR_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (!src_host[i] || !dst_dev[i] || bytes[i] < 0) return TSDF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (int32_t i = 0; i < n; ++i)
    if (bytes[i] > 0 &&
        cudaMemcpyAsync(dst_dev[i], src_host[i], (size_t)bytes[i], cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cuda_fail();
  return TSDF_OK;
}

tsdf_status query_voxels(const tsdf_map* map, const float* pts_dev, int64_t n, float* dist_dev,
                         float* weight_dev, void* cuda_stream) {
  if (!map || n < 0 || (n > 0 && (!pts_dev || !dist_dev || !weight_dev))) return TSDF_ERR_ARG;
  if (map->storage == gbt::kStorageColor) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  if (gbt::launch_query(map->dev, pts_dev, n, dist_dev, weight_dev, (cudaStream_t)cuda_stream) !=
      cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

tsdf_status query_color(const tsdf_map* map, const float* pts_dev, int64_t n, float* rgb_dev,
                        float* weight_dev, void* cuda_stream) {
  if (!map || n < 0 || (n > 0 && (!pts_dev || !rgb_dev || !weight_dev))) return TSDF_ERR_ARG;
  if (map->storage != gbt::kStorageColor) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  if (gbt::launch_query_color(map->dev, pts_dev, n, rgb_dev, weight_dev, (cudaStream_t)cuda_stream) !=
      cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

tsdf_status map_sync(tsdf_map* map) {
  if (!map) return TSDF_ERR_ARG;
  unsigned long long c[gbt::kNumCounters];
  tsdf_status st = read_counters(map, c);
  if (st != TSDF_OK) return st;
  return status_from_bits(map->status_seen);
}

tsdf_status map_num_blocks(const tsdf_map* map, int64_t* out) {
  if (!map || !out) return TSDF_ERR_ARG;
  unsigned long long c[gbt::kNumCounters];
  tsdf_status st = read_counters(map, c);
  if (st != TSDF_OK) return st;
  *out = (int64_t)std::min<unsigned long long>(c[gbt::kCntBlocks], (unsigned long long)map->max_blocks);
  return TSDF_OK;
}

tsdf_status map_stats(const tsdf_map* map, int64_t out[9]) {
  if (!map || !out) return TSDF_ERR_ARG;
  unsigned long long c[gbt::kNumCounters];
  tsdf_status st = read_counters(map, c);
  if (st != TSDF_OK) return st;
  out[0] = (int64_t)std::min<unsigned long long>(c[gbt::kCntBlocks], (unsigned long long)map->max_blocks);
  out[1] = (int64_t)c[gbt::kCntUpdates];
  out[2] = map->frames;
  out[3] = (int64_t)map->status_seen;
  out[4] = (int64_t)c[gbt::kCntVisits];
  out[5] = (int64_t)c[gbt::kCntLaunches];
  out[6] = (int64_t)c[gbt::kCntSegments];
  out[7] = (int64_t)c[gbt::kCntCells];
  out[8] = (int64_t)c[gbt::kCntPairs];
  return TSDF_OK;
}

tsdf_status map_walk_stats(tsdf_map* map, int32_t enable) {
  if (!map) return TSDF_ERR_ARG;
  map->dev.walk_stats = enable ? 1 : 0;
  return TSDF_OK;
}

tsdf_status map_timing(tsdf_map* map, int32_t enable) {
  if (!map) return TSDF_ERR_ARG;
  if (enable && map->events.empty()) {
    map->events.resize(4 * kTimedCalls);
    for (cudaEvent_t& e : map->events)
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail();
  }
  map->timing = enable != 0;
  map->n_timed = 0;
  return TSDF_OK;
}

tsdf_status map_kernel_times(tsdf_map* map, double out_ms[2], int64_t* calls) {
  if (!map || !out_ms || !calls) return TSDF_ERR_ARG;
  out_ms[0] = out_ms[1] = 0.0;
  for (size_t i = 0; i < map->n_timed; ++i) {
    cudaEvent_t* e = &map->events[4 * i];
    float a = 0.0f, b = 0.0f;
    if (cudaEventSynchronize(e[3]) != cudaSuccess || cudaEventSynchronize(e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&a, e[0], e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, e[2], e[3]) != cudaSuccess)
      return cuda_fail();
    out_ms[0] += a;
    out_ms[1] += b;
  }
  *calls = (int64_t)map->n_timed;
  map->n_timed = 0;
  return TSDF_OK;
}

namespace {

// Shared body of map_export and map_export_color: rgb_host is used only for
// colour maps, dist_host only for the others.
tsdf_status export_blocks(const tsdf_map* map, int32_t* keys_host, float* dist_host, float* rgb_host,
                          float* weight_host, int64_t n) {
  if (!map || !keys_host) return TSDF_ERR_ARG;
  int64_t nb = 0;
  tsdf_status st = map_num_blocks(map, &nb);
  if (st != TSDF_OK) return st;
  if (n != nb) return TSDF_ERR_ARG;
  if (nb == 0) return TSDF_OK;
  std::vector<unsigned long long> bk(nb);
  if (cudaMemcpy(bk.data(), map->dev.block_keys, sizeof(unsigned long long) * nb,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail();
  const size_t voxel_bytes = voxel_size_bytes(map->storage);
  std::vector<unsigned char> pool;
  if (dist_host || rgb_host || weight_host) {
    pool.resize(voxel_bytes * gbt::kBlockVoxels * nb);
    if (cudaMemcpy(pool.data(), map->dev.pool, pool.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail();
  }
  std::vector<int64_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  auto coords = [&](int64_t i, int axis) { return gbt::key_coord(bk[i], axis); };
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    for (int ax = 0; ax < 3; ++ax)
      if (coords(a, ax) != coords(b, ax)) return coords(a, ax) < coords(b, ax);
    return false;
  });
  const float tau = map->dev.tau;
  for (int64_t r = 0; r < nb; ++r) {
    const int64_t i = order[r];
    for (int ax = 0; ax < 3; ++ax) keys_host[3 * r + ax] = coords(i, ax);
    if (pool.empty()) continue;
    for (int l = 0; l < gbt::kBlockVoxels; ++l) {
      float D, W;
      if (map->storage == gbt::kStorageColor) {
        const float4 c = reinterpret_cast<const float4*>(pool.data())[(size_t)i * 512 + l];
        if (rgb_host) {
          float* out = rgb_host + ((size_t)r * 512 + l) * 3;
          out[0] = c.x;
          out[1] = c.y;
          out[2] = c.z;
        }
        D = 0.0f;
        W = c.w;
      } else if (map->storage == gbt::kStorageOcc) {
        D = reinterpret_cast<const float*>(pool.data())[(size_t)i * 512 + l];
        W = 0.0f;
      } else if (map->storage == TSDF_STORAGE_FP16) {
        const __half2 h = reinterpret_cast<const __half2*>(pool.data())[(size_t)i * 512 + l];
        D = __low2float(h) * tau;
        W = __high2float(h);
      } else if (map->storage == TSDF_STORAGE_FIXED16) {
        const uint32_t word = reinterpret_cast<const uint32_t*>(pool.data())[(size_t)i * 512 + l];
        D = gbt::x16_dist(word, map->dev.x16_unit);
        W = gbt::x16_weight(word);
      } else {
        const float2 f = reinterpret_cast<const float2*>(pool.data())[(size_t)i * 512 + l];
        D = f.x;
        W = f.y;
      }
      if (dist_host) dist_host[(size_t)r * 512 + l] = D;
      if (weight_host) weight_host[(size_t)r * 512 + l] = W;
    }
  }
  return TSDF_OK;
}

}  // namespace

tsdf_status map_export(const tsdf_map* map, int32_t* keys_host, float* dist_host,
                       float* weight_host, int64_t n) {
  return export_blocks(map, keys_host, dist_host, nullptr, weight_host, n);
}

tsdf_status map_export_color(const tsdf_map* map, int32_t* keys_host, float* rgb_host,
                             float* weight_host, int64_t n) {
  if (!map || map->storage != gbt::kStorageColor) return TSDF_ERR_ARG;
  return export_blocks(map, keys_host, nullptr, rgb_host, weight_host, n);
}

tsdf_status map_decay_occupancy(tsdf_map* map, float decay_occ, float decay_free,
                                void* cuda_stream) {
  if (!map || map->storage != gbt::kStorageOcc || !(decay_occ >= 0.0f) || !(decay_free >= 0.0f) ||
      !std::isfinite(decay_occ) || !std::isfinite(decay_free))
    return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  if (gbt::launch_decay(map->dev, decay_occ, decay_free, (cudaStream_t)cuda_stream) != cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

// ------------------------------------------------------------------ ESDF

namespace {

bool esdf_layer_ok(const tsdf_map* m) {
  return m->storage == TSDF_STORAGE_FP32 || m->storage == TSDF_STORAGE_FP16 ||
         m->storage == TSDF_STORAGE_FIXED16 || m->storage == gbt::kStorageOcc;
}

tsdf_status esdf_alloc(tsdf_map* m, const tsdf_esdf_opts& o) {
  EsdfDev& e = m->esdf;
  std::memset(&e, 0, sizeof(e));
  const size_t nb = (size_t)m->max_blocks;
  bool ok = cudaMalloc(&e.st, sizeof(uint32_t) * 512 * nb) == cudaSuccess &&
            cudaMalloc(&e.st2, sizeof(uint32_t) * 512 * nb) == cudaSuccess &&
            cudaMalloc(&e.list[0], sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.list[1], sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.tlist[0], sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.tlist[1], sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.nbr, sizeof(int32_t) * 6 * nb) == cudaSuccess &&
            cudaMalloc(&e.clist, sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.stamp_s, sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.stamp_t, sizeof(uint32_t) * nb) == cudaSuccess &&
            cudaMalloc(&e.tchanged, nb) == cudaSuccess &&
            cudaMalloc(&e.bits, sizeof(uint32_t) * 2 * gbt::kEsdfBitWords) == cudaSuccess &&
            cudaMalloc(&e.cnt, sizeof(uint32_t) * 8) == cudaSuccess &&
            cudaMalloc(&e.stats, sizeof(unsigned long long) * 4) == cudaSuccess &&
            cudaMallocHost(&m->esdf_host, sizeof(uint32_t) * 8) == cudaSuccess;
  if (ok)
    ok = cudaMemset(e.st, 0, sizeof(uint32_t) * 512 * nb) == cudaSuccess &&
         cudaMemset(e.stamp_s, 0, sizeof(uint32_t) * nb) == cudaSuccess &&
         cudaMemset(e.stamp_t, 0, sizeof(uint32_t) * nb) == cudaSuccess &&
         cudaMemset(e.cnt, 0, sizeof(uint32_t) * 8) == cudaSuccess &&
         cudaMemset(e.stats, 0, sizeof(unsigned long long) * 4) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  m->esdf_on = true;  // free_map releases whatever was allocated
  if (!ok) return cuda_fail();
  e.site_eps = o.site_eps;
  e.min_weight = o.min_weight;
  e.max_dist = o.max_dist_vox;
  m->esdf_opts = o;
  m->esdf_gen = 0;
  return TSDF_OK;
}

tsdf_status esdf_read_counts(tsdf_map* m, cudaStream_t s) {
  if (cudaMemcpyAsync(m->esdf_host, m->esdf.cnt, sizeof(uint32_t) * 8, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

}  // namespace

tsdf_status map_esdf_update(tsdf_map* map, const tsdf_esdf_opts* opts, void* cuda_stream) {
  if (!map || !esdf_layer_ok(map)) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  tsdf_esdf_opts o{map->v, 1e-4f, 64};
  if (opts) o = *opts;
  if (!(o.site_eps >= 0.0f) || !std::isfinite(o.site_eps) || !std::isfinite(o.min_weight) ||
      o.max_dist_vox < 1 || o.max_dist_vox > 255)
    return TSDF_ERR_ARG;
  if (map->esdf_on && (o.site_eps != map->esdf_opts.site_eps ||
                       o.min_weight != map->esdf_opts.min_weight ||
                       o.max_dist_vox != map->esdf_opts.max_dist_vox))
    return TSDF_ERR_ARG;  // parameters are fixed by the first update
  if (!map->esdf_on) {
    tsdf_status st = esdf_alloc(map, o);
    if (st != TSDF_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  EsdfDev& e = map->esdf;
  // mark sites and clear invalid parents: update set 0 gets generation g
  const uint32_t g = ++map->esdf_gen;
  if (cudaMemsetAsync(e.cnt, 0, sizeof(uint32_t) * 8, s) != cudaSuccess ||
      cudaMemsetAsync(e.bits, 0, sizeof(uint32_t) * 2 * gbt::kEsdfBitWords, s) != cudaSuccess ||
      gbt::launch_esdf_mark(map->dev, e, g, s) != cudaSuccess ||
      gbt::launch_esdf_clear(map->dev, e, g, s) != cudaSuccess)
    return cuda_fail();
  // lower until no block changes: four iterations per read-back of the set
  // size (iterations on an empty set return at once)
  constexpr int kItersPerCheck = 4;
  int cur = 0;
  for (;;) {
    for (int k = 0; k < kItersPerCheck; ++k) {
      const uint32_t gen_t = ++map->esdf_gen, gen_next = ++map->esdf_gen;
      if (gbt::launch_esdf_iteration(map->dev, e, cur, gen_t, gen_next, s) != cudaSuccess)
        return cuda_fail();
      cur = 1 - cur;
    }
    tsdf_status st = esdf_read_counts(map, s);
    if (st != TSDF_OK) return st;
    if (map->esdf_host[cur] == 0) break;
  }
  return TSDF_OK;
}

tsdf_status map_esdf_stats(const tsdf_map* map, int64_t out[4]) {
  if (!map || !out) return TSDF_ERR_ARG;
  unsigned long long st[4] = {0, 0, 0, 0};
  if (map->esdf_on && (cudaDeviceSynchronize() != cudaSuccess ||
                       cudaMemcpy(st, map->esdf.stats, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess))
    return cuda_fail();
  out[0] = (int64_t)st[1];
  out[1] = (int64_t)st[2];
  out[2] = (int64_t)st[3];
  out[3] = (int64_t)st[0];
  return TSDF_OK;
}

tsdf_status map_esdf_export(const tsdf_map* map, int32_t* keys_host, uint32_t* states_host, int64_t n) {
  if (!map || !keys_host || !map->esdf_on) return TSDF_ERR_ARG;
  int64_t nb = 0;
  tsdf_status st = map_num_blocks(map, &nb);
  if (st != TSDF_OK) return st;
  if (n != nb) return TSDF_ERR_ARG;
  if (nb == 0) return TSDF_OK;
  std::vector<unsigned long long> bk(nb);
  std::vector<uint32_t> all;
  if (cudaMemcpy(bk.data(), map->dev.block_keys, sizeof(unsigned long long) * nb,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail();
  if (states_host) {
    all.resize((size_t)nb * 512);
    if (cudaMemcpy(all.data(), map->esdf.st, sizeof(uint32_t) * all.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return cuda_fail();
  }
  std::vector<int64_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  auto coords = [&](int64_t i, int axis) { return gbt::key_coord(bk[i], axis); };
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    for (int ax = 0; ax < 3; ++ax)
      if (coords(a, ax) != coords(b, ax)) return coords(a, ax) < coords(b, ax);
    return false;
  });
  for (int64_t r = 0; r < nb; ++r) {
    const int64_t i = order[r];
    for (int ax = 0; ax < 3; ++ax) keys_host[3 * r + ax] = coords(i, ax);
    if (states_host) std::memcpy(states_host + 512 * r, all.data() + 512 * i, sizeof(uint32_t) * 512);
  }
  return TSDF_OK;
}

tsdf_status map_esdf_query(const tsdf_map* map, const float* pts_dev, int64_t n, float* dist_dev,
                           void* cuda_stream) {
  if (!map || !map->esdf_on || n < 0 || (n > 0 && (!pts_dev || !dist_dev))) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  if (gbt::launch_esdf_query(map->dev, map->esdf, pts_dev, n, dist_dev, (cudaStream_t)cuda_stream) !=
      cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

tsdf_status map_import(tsdf_map* map, const int32_t* keys_host, const float* dist_host,
                       const float* weight_host, int64_t n) {
  if (!map || n < 0 || (n > 0 && (!keys_host || !dist_host))) return TSDF_ERR_ARG;
  if (map->storage == gbt::kStorageColor) return TSDF_ERR_ARG;
  if (n > 0 && map->storage != gbt::kStorageOcc && !weight_host) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  if (n == 0) return TSDF_OK;
  std::vector<std::array<int32_t, 3>> ks((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      const int32_t c = keys_host[3 * i + a];
      if (c <= -gbt::kKeyBias || c >= gbt::kKeyBias) return TSDF_ERR_ARG;
      ks[i][a] = c;
    }
  }
  std::sort(ks.begin(), ks.end());
  if (std::adjacent_find(ks.begin(), ks.end()) != ks.end()) return TSDF_ERR_ARG;  // duplicate keys
  int32_t* dk = nullptr;
  float *dD = nullptr, *dW = nullptr;
  const size_t vox = (size_t)n * 512;
  std::vector<float> zeros;
  if (!weight_host) zeros.assign(vox, 0.0f);
  bool ok = cudaMalloc(&dk, sizeof(int32_t) * 3 * n) == cudaSuccess &&
            cudaMalloc(&dD, sizeof(float) * vox) == cudaSuccess &&
            cudaMalloc(&dW, sizeof(float) * vox) == cudaSuccess &&
            cudaMemcpy(dk, keys_host, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dD, dist_host, sizeof(float) * vox, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dW, weight_host ? weight_host : zeros.data(), sizeof(float) * vox,
                       cudaMemcpyHostToDevice) == cudaSuccess &&
            gbt::launch_import(map->dev, dk, dD, dW, n, 0) == cudaSuccess &&
            cudaDeviceSynchronize() == cudaSuccess;
  cudaFree(dk);
  cudaFree(dD);
  cudaFree(dW);
  if (!ok) return cuda_fail();
  return TSDF_OK;
}

// ------------------------------------------------------------------ mesh

namespace {

// Marching-cubes case table.  Each face's corners are listed counter-
// clockwise as seen from outside the cube; walking round a face, a segment
// runs from the edge where the walk enters a run of inside corners to the
// edge where it leaves the run (so a face with two diagonal inside corners
// gets one segment around each).  The segments of the six faces chain into
// loops; a loop starts at its smallest edge number and is cut into the fan
// (e0, ei, ei+1).  Corner c = x + 2 y + 4 z; edge number 4 * axis + u + 2 w,
// u and w the edge's coordinates on the other two axes in increasing order.
gbt::MeshTable make_mesh_table() {
  static const int kFaces[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                   {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
  auto edge_between = [](int a, int b) {
    const int axis = (a ^ b) == 1 ? 0 : ((a ^ b) == 2 ? 1 : 2);
    const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    return 4 * axis + ((a >> o1) & 1) + 2 * ((a >> o2) & 1);
  };
  gbt::MeshTable t;
  std::memset(&t, 0, sizeof(t));
  for (int ci = 0; ci < 256; ++ci) {
    int next[12];
    std::fill(next, next + 12, -1);
    for (const auto& f : kFaces) {
      for (int j = 0; j < 4; ++j) {
        const bool out_j = !((ci >> f[j]) & 1), in_j1 = (ci >> f[(j + 1) & 3]) & 1;
        if (!(out_j && in_j1)) continue;
        int k = (j + 1) & 3;  // last inside corner of the run
        while ((ci >> f[(k + 1) & 3]) & 1) k = (k + 1) & 3;
        next[edge_between(f[j], f[(j + 1) & 3])] = edge_between(f[k], f[(k + 1) & 3]);
      }
    }
    bool used[12] = {false};
    int n = 0;
    for (int s0 = 0; s0 < 12; ++s0) {
      if (next[s0] < 0 || used[s0]) continue;
      int loop[12], len = 0;
      for (int e = s0; !used[e]; e = next[e]) {
        used[e] = true;
        loop[len++] = e;
      }
      for (int i = 1; i + 1 < len && n < 5; ++i, ++n) {
        t.edges[ci][3 * n] = (int8_t)loop[0];
        t.edges[ci][3 * n + 1] = (int8_t)loop[i];
        t.edges[ci][3 * n + 2] = (int8_t)loop[i + 1];
      }
    }
    t.count[ci] = (uint8_t)n;
  }
  return t;
}

const gbt::MeshTable& mesh_table() {
  static const gbt::MeshTable t = make_mesh_table();
  return t;
}

}  // namespace

tsdf_status map_mesh(tsdf_map* map, float min_weight, int32_t changed_only, float* tri_pos_dev,
                     int32_t* tri_keys_dev, int32_t* tri_cube_dev, int64_t cap, int64_t* n_tris,
                     void* cuda_stream) {
  if (!map || !n_tris || cap < 0 || (cap > 0 && !tri_pos_dev) || !std::isfinite(min_weight)) return TSDF_ERR_ARG;
  if (map->storage != TSDF_STORAGE_FP32 && map->storage != TSDF_STORAGE_FP16 &&
      map->storage != TSDF_STORAGE_FIXED16)
    return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  gbt::MeshDev& md = map->mesh;
  if (!map->mesh_on) {
    std::memset(&md, 0, sizeof(md));
    map->mesh_on = true;  // free_map releases whatever was allocated
    if (cudaMalloc(&md.list, sizeof(uint32_t) * map->max_blocks) != cudaSuccess ||
        cudaMalloc(&md.stamp, sizeof(uint32_t) * map->max_blocks) != cudaSuccess ||
        cudaMalloc(&md.cnt, sizeof(unsigned long long) * 2) != cudaSuccess ||
        cudaMemset(md.stamp, 0, sizeof(uint32_t) * map->max_blocks) != cudaSuccess)
      return cuda_fail();
    map->mesh_gen = 0;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long cnt[2] = {0, 0};
  if (cudaMemsetAsync(md.cnt, 0, sizeof(cnt), s) != cudaSuccess ||
      gbt::launch_mesh(map->dev, md, mesh_table(), changed_only ? 1 : 0, ++map->mesh_gen, min_weight,
                       tri_pos_dev, tri_keys_dev, tri_cube_dev, cap, s) != cudaSuccess ||
      cudaMemcpyAsync(cnt, md.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail();
  *n_tris = (int64_t)cnt[1];
  return cnt[1] > (unsigned long long)cap ? TSDF_ERR_CAPACITY : TSDF_OK;
}

tsdf_status map_wait_test(tsdf_map* map, int32_t extra_ctas) {
  if (!map || extra_ctas < 0) return TSDF_ERR_ARG;
  map->wait_extra = extra_ctas;
  return TSDF_OK;
}

tsdf_status map_reset(tsdf_map* map, void* cuda_stream) {
  if (!map) return TSDF_ERR_ARG;
  if (!on_device(map)) return TSDF_ERR_STATE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (gbt::launch_reset(map->dev, map->cap, s) != cudaSuccess ||
      cudaMemsetAsync(map->mask1, 0, sizeof(uint32_t) * map->cap, s) != cudaSuccess ||
      cudaMemsetAsync(map->ctl1, 0, sizeof(unsigned int) * 4, s) != cudaSuccess ||
      cudaMemsetAsync(map->dev.dirty, 0, (size_t)map->max_blocks, s) != cudaSuccess)
    return cuda_fail();
  if (map->esdf_on &&
      (cudaMemsetAsync(map->esdf.st, 0, sizeof(uint32_t) * 512 * map->max_blocks, s) != cudaSuccess ||
       cudaMemsetAsync(map->esdf.stats, 0, sizeof(unsigned long long) * 4, s) != cudaSuccess))
    return cuda_fail();
  map->status_seen = 0;
  map->frames = 0;
  return TSDF_OK;
}

tsdf_status map_destroy(tsdf_map* map) {
  if (!map) return TSDF_ERR_ARG;
  cudaDeviceSynchronize();
  free_map(map);
  return TSDF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// integrate_depth_static: the allocation-free entry point.
//
// Some callers cannot allocate GPU memory themselves or through this library
// (a process whose device allocator is owned by another framework, real-time
// loops that forbid allocation after start-up).  For them the per-call work
// list that the integration needs lives in g_static_scratch, a fixed-size
// array in device memory that the module reserves on every GPU that loads it
// and keeps until the process exits.  The caller owns all map storage and
// the input image.

// The caller sizes and decodes its buffers from the header's constants; they
// must be the kernels' own.
static_assert(TSDF_NUM_COUNTERS == gbt::kNumCounters, "counter words written by the kernels");
static_assert(TSDF_STORAGE_FP32 == gbt::kStorageF32 && TSDF_STORAGE_FP16 == gbt::kStorageF16 &&
                  TSDF_STORAGE_FIXED16 == gbt::kStorageX16,
              "ABI storage codes are the kernels' own");
static_assert(TSDF_KEY_BIAS == gbt::kKeyBias, "block key bias");
static_assert(gbt::pack_key(1, 0, 0) - gbt::pack_key(0, 0, 0) == 1ull &&
                  gbt::pack_key(0, 1, 0) - gbt::pack_key(0, 0, 0) == (1ull << TSDF_KEY_BITS) &&
                  gbt::pack_key(0, 0, 1) - gbt::pack_key(0, 0, 0) == (1ull << (2 * TSDF_KEY_BITS)) &&
                  gbt::pack_key(0, 0, 0) == ((unsigned long long)TSDF_KEY_BIAS *
                                             (1ull + (1ull << TSDF_KEY_BITS) + (1ull << (2 * TSDF_KEY_BITS)))),
              "block key packing");

namespace {

constexpr int64_t kStaticMaxBlocks = TSDF_STATIC_MAX_BLOCKS;
// [0, kStaticMaxBlocks): work list of hash slots; then 4 control words
// (list length, finished integration CTAs, entries handed out, spare).
static __device__ __align__(256) uint32_t g_static_scratch[kStaticMaxBlocks + 4];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
uint32_t* g_static_ptr[kStaticMaxDevices] = {};  // device address of g_static_scratch per device

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
tsdf_status static_scratch(uint32_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return cuda_fail();
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return cuda_fail();
    g_static_ptr[dev] = static_cast<uint32_t*>(ptr);
  }
  *out = g_static_ptr[dev];
  return TSDF_OK;
}

}  // namespace

extern "C" {

tsdf_status integrate_depth_static(const tsdf_map_buffers* buf, float voxel_size,
                                   int32_t truncation_voxels, float max_weight,
                                   const float* depth_dev, const tsdf_pinhole* intr,
                                   const double T_world_cam[16], void* cuda_stream) {
  if (!buf || !buf->keys || !buf->vals || !buf->mask || !buf->pool || !buf->block_keys ||
      !buf->counters || !depth_dev || !intr || !T_world_cam)
    return TSDF_ERR_ARG;
  if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size) || truncation_voxels <= 0 ||
      !(max_weight > 0.0f) || !std::isfinite(max_weight))
    return TSDF_ERR_ARG;
  if (buf->max_blocks <= 0) return TSDF_ERR_ARG;
  if (buf->max_blocks > kStaticMaxBlocks) return TSDF_ERR_CAPACITY;  // beyond the scratch size
  const int64_t cap = buf->hash_capacity;
  if (cap < 2 * buf->max_blocks || cap > (1ll << 30) || (cap & (cap - 1)) != 0) return TSDF_ERR_ARG;
  uint32_t* scratch = nullptr;
  tsdf_status st = static_scratch(&scratch);
  if (st != TSDF_OK) return st;

  BatchParams<1, 1> p;
  std::memset(&p, 0, sizeof(p));
  p.n_frames = 1;
  p.n_maps = 1;
  MapDev& d = p.maps[0];
  d.keys = buf->keys;
  d.vals = buf->vals;
  d.mask = buf->mask;
  d.pool = buf->pool;
  d.block_keys = buf->block_keys;
  d.counters = buf->counters;
  d.list = scratch;
  d.ctl = scratch + kStaticMaxBlocks;
  d.list_cap = (uint32_t)buf->max_blocks;
  d.cap_mask = (uint32_t)(cap - 1);
  d.max_blocks = (int32_t)buf->max_blocks;
  d.storage = TSDF_STORAGE_FP32;
  d.lidar_nearest = 0;
  d.v = voxel_size;
  d.tau = (float)((double)truncation_voxels * (double)voxel_size);
  d.inv_tau = 1.0f / d.tau;
  d.wmax = max_weight;
  d.guard = d.tau;

  FrameDev& F = p.fr[0];
  if (!rigid(T_world_cam) || !valid_pinhole(intr)) return TSDF_ERR_ARG;
  F.kind = TSDF_SENSOR_PINHOLE;
  F.map = 0;
  F.depth = depth_dev;
  F.width = intr->width;
  F.height = intr->height;
  F.fu = intr->fu;
  F.fv = intr->fv;
  F.cu = intr->cu;
  F.cv = intr->cv;
  F.blk_begin = 0;
  F.bit = 0;
  if (!prepare_pose(8.0 * (double)voxel_size, T_world_cam, F)) return TSDF_ERR_ARG;
  p.fast_rcp = fast_rcp_ok(F, (double)voxel_size, INT_MAX) ? 1 : 0;
  F.short_walks = short_walks_ok(F, truncation_voxels) ? 1 : 0;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cuda_fail();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the control words must start at zero; a previous call leaves them so,
  // but a call that never ran to completion might not have
  if (cudaMemsetAsync(d.ctl, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return cuda_fail();
  const int th = pick_tile_h((int64_t)F.width * F.height);
  if (gbt::launch_band_alloc(p, alloc_ctas(F, th), th, s) != cudaSuccess) return cuda_fail();
  if (gbt::launch_integrate(p, std::max(1, sms) * gbt::integrate_ctas_per_sm(TSDF_STORAGE_FP32), s) !=
      cudaSuccess)
    return cuda_fail();
  return TSDF_OK;
}

}  // extern "C"
