// CUDA kernels of the GB300 TSDF library (sm_103a).
//
//  band_alloc_kernel  Sec. IV-B first step: every valid pixel's ray segment
//                     inside the truncation band is walked through the block
//                     grid (Amanatides & Woo traversal); lanes of a warp that
//                     reach the same block are merged with match.any, the
//                     leader inserts it into the open-addressing hash
//                     (atomicCAS on the packed key), assigns a pool block if
//                     new, and sets its frame bit; the first frame bit on a
//                     block appends it to the batch work list.
//  integrate_kernel   Sec. IV-B second step (Eq. 1-3 and the TSDF update
//                     functor): one CTA per work-list block, 4 voxels per
//                     thread held in registers across every frame of the
//                     batch that met the block, one coalesced 16-byte read
//                     and write per thread and frame batch.
//  query_kernel       point -> voxel lookup through the hash.
//
// Discrete decisions use explicit round-to-nearest intrinsics in a fixed
// order (no contraction) so that they are reproducible on a CPU.
#include <cfloat>

#include "tsdf_internal.cuh"

namespace gbt {
namespace {

constexpr float kPiF = (float)3.14159265358979323846;
constexpr float kHalfPiF = (float)(3.14159265358979323846 / 2);

// ------------------------------------------------------------------ hash

__device__ __forceinline__ int hash_insert(const MapDev& m, unsigned long long key, bool& inserted) {
  uint32_t slot = hash_key(key) & m.cap_mask;
  inserted = false;
  for (uint32_t probe = 0; probe <= m.cap_mask; ++probe) {
    const unsigned long long k = __ldcg(m.keys + slot);
    if (k == key) return (int)slot;
    if (k == kEmptyKey) {
      const unsigned long long old = atomicCAS(m.keys + slot, kEmptyKey, key);
      if (old == kEmptyKey) {
        inserted = true;
        return (int)slot;
      }
      if (old == key) return (int)slot;
    }
    slot = (slot + 1) & m.cap_mask;
  }
  return -1;
}

__device__ __forceinline__ int hash_find(const MapDev& m, unsigned long long key) {
  uint32_t slot = hash_key(key) & m.cap_mask;
  for (uint32_t probe = 0; probe <= m.cap_mask; ++probe) {
    const unsigned long long k = m.keys[slot];
    if (k == key) return (int)slot;
    if (k == kEmptyKey) return -1;
    slot = (slot + 1) & m.cap_mask;
  }
  return -1;
}

// ------------------------------------------------- block-grid traversal

// Walk of a segment o + s dir, s in [s0, s1] (block units, anchor-relative)
// through the block grid: crossing parameters are recomputed from the origin
// at every step, ties between axes go to x, then y, then z; at most
// kMaxCells cells.
struct Walk {
  int cx, cy, cz;
  int sx, sy, sz;
  float ix, iy, iz;
  float tx, ty, tz;
  float s1;
  int n;

  __device__ __forceinline__ static float cross(int c, int step, float o, float inv) {
    if (step == 0) return __int_as_float(0x7f800000);  // +inf
    const float bnd = (float)(step > 0 ? c + 1 : c);
    return __fmul_rn(__fsub_rn(bnd, o), inv);
  }
  __device__ __forceinline__ static int sgn(float d) { return d > 0.0f ? 1 : (d < 0.0f ? -1 : 0); }

  // false if the segment starts outside the 21-bit key range
  __device__ __forceinline__ bool start(const float* o, float dx, float dy, float dz, float s0,
                                        float s1_) {
    const float px = __fmaf_rn(s0, dx, o[0]), py = __fmaf_rn(s0, dy, o[1]), pz = __fmaf_rn(s0, dz, o[2]);
    if (!(fabsf(px) < 262144.0f && fabsf(py) < 262144.0f && fabsf(pz) < 262144.0f)) return false;
    cx = (int)floorf(px);
    cy = (int)floorf(py);
    cz = (int)floorf(pz);
    sx = sgn(dx);
    sy = sgn(dy);
    sz = sgn(dz);
    ix = sx ? __frcp_rn(dx) : 0.0f;
    iy = sy ? __frcp_rn(dy) : 0.0f;
    iz = sz ? __frcp_rn(dz) : 0.0f;
    tx = cross(cx, sx, o[0], ix);
    ty = cross(cy, sy, o[1], iy);
    tz = cross(cz, sz, o[2], iz);
    s1 = s1_;
    n = 1;
    return true;
  }
  // advance to the next cell; false when the segment ends
  __device__ __forceinline__ bool next(const float* o) {
    int k = 0;
    float t = tx;
    if (ty < t) { k = 1; t = ty; }
    if (tz < t) { k = 2; t = tz; }
    if (!(t <= s1) || n == kMaxCells) return false;
    if (k == 0) { cx += sx; tx = cross(cx, sx, o[0], ix); }
    else if (k == 1) { cy += sy; ty = cross(cy, sy, o[1], iy); }
    else { cz += sz; tz = cross(cz, sz, o[2], iz); }
    ++n;
    return true;
  }
};

__device__ __forceinline__ void claim_block(const MapDev& m, unsigned long long key, int bit) {
  bool ins;
  const int slot = hash_insert(m, key, ins);
  if (slot < 0) {
    atomicOr(m.counters + kCntStatus, (unsigned long long)kStHashFull);
    return;
  }
  if (ins) {
    const unsigned long long p = atomicAdd(m.counters + kCntBlocks, 1ull);
    if (p < (unsigned long long)m.max_blocks) {
      m.vals[slot] = -(int)p - 2;
      m.block_keys[p] = key;
    } else {
      m.vals[slot] = -1;
      atomicOr(m.counters + kCntStatus, (unsigned long long)kStPoolFull);
    }
  }
  const uint32_t b = 1u << bit;
  if (__ldcg(m.mask + slot) & b) return;
  if (atomicOr(m.mask + slot, b) == 0u) {
    const uint32_t idx = atomicAdd(m.ctl, 1u);
    if (idx < m.list_cap) m.list[idx] = (uint32_t)slot;
    else atomicOr(m.counters + kCntStatus, (unsigned long long)kStListFull);
  }
}

template <int NF, int NM>
__global__ void __launch_bounds__(kAllocThreads)
    band_alloc_kernel(const __grid_constant__ BatchParams<NF, NM> p) {
  int f = 0;
#pragma unroll 1
  for (int k = 1; k < p.n_frames; ++k)
    if ((int)blockIdx.x >= p.fr[k].blk_begin) f = k;
  const FrameDev& F = p.fr[f];
  const MapDev& m = p.maps[F.map];
  const int pix = ((int)blockIdx.x - F.blk_begin) * kAllocThreads + (int)threadIdx.x;
  const int npix = F.width * F.height;

  Walk wk;
  bool live = false;
  if (pix < npix) {
    const float d = __ldg(F.depth + pix);
    const int i = pix % F.width, j = pix / F.width;
    float dx, dy, dz;
    bool valid;
    if (F.kind == kSensorPinhole) {
      valid = d > 0.0f && d <= FLT_MAX;
      const float rx = __fdiv_rn(__fsub_rn((float)i, F.cu), F.fu);
      const float ry = __fdiv_rn(__fsub_rn((float)j, F.cv), F.fv);
      dx = __fmaf_rn(F.M[0], rx, __fmaf_rn(F.M[1], ry, F.M[2]));
      dy = __fmaf_rn(F.M[3], rx, __fmaf_rn(F.M[4], ry, F.M[5]));
      dz = __fmaf_rn(F.M[6], rx, __fmaf_rn(F.M[7], ry, F.M[8]));
    } else {
      valid = d >= F.min_range && d <= F.max_range;
      const float2 az = __ldg(reinterpret_cast<const float2*>(F.tab) + i);
      const float2 el = __ldg(reinterpret_cast<const float2*>(F.tab) + F.width + j);
      const float bx = __fmul_rn(el.y, az.x), by = __fmul_rn(el.y, az.y), bz = el.x;
      dx = __fmaf_rn(F.M[0], bx, __fmaf_rn(F.M[1], by, __fmul_rn(F.M[2], bz)));
      dy = __fmaf_rn(F.M[3], bx, __fmaf_rn(F.M[4], by, __fmul_rn(F.M[5], bz)));
      dz = __fmaf_rn(F.M[6], bx, __fmaf_rn(F.M[7], by, __fmul_rn(F.M[8], bz)));
    }
    if (valid) {
      const float s0 = fmaxf(__fsub_rn(d, m.tau), 0.0f), s1 = __fadd_rn(d, m.tau);
      live = wk.start(F.o, dx, dy, dz, s0, s1);
    }
  }
  const unsigned lane = threadIdx.x & 31u;
  while (true) {
    const unsigned act = __ballot_sync(0xffffffffu, live);
    if (act == 0u) break;
    if (live) {
      const unsigned long long key = pack_key(F.a[0] + wk.cx, F.a[1] + wk.cy, F.a[2] + wk.cz);
      const unsigned peers = __match_any_sync(act, key);
      if (lane == (unsigned)(__ffs(peers) - 1)) claim_block(m, key, F.bit);
      live = wk.next(F.o);
    }
  }
}

// ------------------------------------------------ per-voxel projection

// FP32 atan2 for decisions: octant reduction, the half-angle identity
// atan t = 2 atan(t / (1 + sqrt(1 + t^2))) applied twice (|t| <= tan(pi/16)),
// then the Maclaurin series of atan through t^13.
__device__ __forceinline__ float atan2_dec(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  if (mx == 0.0f) return 0.0f;
  const float t = __fdiv_rn(mn, mx);
  const float t1 = __fdiv_rn(t, __fadd_rn(1.0f, __fsqrt_rn(__fmaf_rn(t, t, 1.0f))));
  const float t2 = __fdiv_rn(t1, __fadd_rn(1.0f, __fsqrt_rn(__fmaf_rn(t1, t1, 1.0f))));
  const float z = __fmul_rn(t2, t2);
  float q = 1.0f / 13.0f;
  q = __fmaf_rn(q, z, -(1.0f / 11.0f));
  q = __fmaf_rn(q, z, 1.0f / 9.0f);
  q = __fmaf_rn(q, z, -(1.0f / 7.0f));
  q = __fmaf_rn(q, z, 1.0f / 5.0f);
  q = __fmaf_rn(q, z, -(1.0f / 3.0f));
  q = __fmaf_rn(q, z, 1.0f);
  float a = __fmul_rn(4.0f, __fmul_rn(t2, q));
  if (ay > ax) a = __fsub_rn(kHalfPiF, a);
  if (x < 0.0f) a = __fsub_rn(kPiF, a);
  if (y < 0.0f) a = -a;
  return a;
}

__device__ __forceinline__ bool lidar_valid(const FrameDev& F, float d) {
  return d >= F.min_range && d <= F.max_range;
}

// Sample the image at the projection of sensor-frame point (px, py, pz).
// Returns false if the voxel is not updated; else the depth sample d and the
// voxel depth d_v (z for a camera, range for a LiDAR).  Eq. 1-3.
__device__ __forceinline__ bool sample(const FrameDev& F, const MapDev& m, float px, float py,
                                       float pz, float& d, float& dv) {
  if (F.kind == kSensorPinhole) {
    if (!(pz > 0.0f)) return false;
    const float iz = __frcp_rn(pz);
    const float u = __fadd_rn(__fmaf_rn(__fmul_rn(px, iz), F.fu, F.cu), 0.5f);
    const float v = __fadd_rn(__fmaf_rn(__fmul_rn(py, iz), F.fv, F.cv), 0.5f);
    if (!(u >= 0.0f && u < (float)F.width && v >= 0.0f && v < (float)F.height)) return false;
    d = __ldg(F.depth + (int)v * F.width + (int)u);
    if (!(d > 0.0f && d <= FLT_MAX)) return false;
    dv = pz;
    return true;
  }
  const float r = __fsqrt_rn(__fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz))));
  if (!(r > 0.0f)) return false;
  const float rho = __fsqrt_rn(__fmaf_rn(px, px, __fmul_rn(py, py)));
  const float th = atan2_dec(py, px);
  const float ph = atan2_dec(rho, pz);
  const float u = __fmul_rn(__fsub_rn(th, F.theta_start), F.alpha);
  const float v = __fmul_rn(__fsub_rn(ph, F.phi_start), F.beta);
  const int naz = F.width, nel = F.height;
  if (m.lidar_nearest) {
    const float ku = floorf(u), jv = floorf(v);
    if (!(jv >= 0.0f && jv <= (float)(nel - 1))) return false;
    if (!(ku >= -1.0f && ku <= (float)naz)) return false;
    const int kk = (((int)ku % naz) + naz) % naz, jj = (int)jv;
    d = __ldg(F.depth + jj * naz + kk);
    if (!lidar_valid(F, d)) return false;
  } else {
    const float uu = __fsub_rn(u, 0.5f), vv = __fsub_rn(v, 0.5f);
    const float k0f = floorf(uu), j0f = floorf(vv);
    if (!(j0f >= 0.0f && j0f <= (float)(nel - 2))) return false;
    if (!(k0f >= -1.0f && k0f <= (float)naz)) return false;
    const float fx = __fsub_rn(uu, k0f), fy = __fsub_rn(vv, j0f);
    const int k0 = (((int)k0f % naz) + naz) % naz, k1 = (k0 + 1) % naz, j0 = (int)j0f;
    const float* row0 = F.depth + j0 * naz;
    const float* row1 = row0 + naz;
    const float d00 = __ldg(row0 + k0), d10 = __ldg(row0 + k1);
    const float d01 = __ldg(row1 + k0), d11 = __ldg(row1 + k1);
    if (!(lidar_valid(F, d00) && lidar_valid(F, d10) && lidar_valid(F, d01) && lidar_valid(F, d11)))
      return false;
    const float hi = fmaxf(fmaxf(d00, d10), fmaxf(d01, d11));
    const float lo = fminf(fminf(d00, d10), fminf(d01, d11));
    if (__fsub_rn(hi, lo) > m.guard) return false;
    const float top = __fmaf_rn(fx, __fsub_rn(d10, d00), d00);
    const float bot = __fmaf_rn(fx, __fsub_rn(d11, d01), d01);
    d = __fmaf_rn(fy, __fsub_rn(bot, top), top);
  }
  dv = r;
  return true;
}

// TSDF update functor (Sec. IV-B): weighted running average with weight 1,
// the average taken with the unclamped weight sum, then weights capped.
__device__ __forceinline__ void fuse(float& D, float& W, float s, float wmax) {
  const float wn = W + 1.0f;
  D = D + __fdividef(s - D, wn);
  W = fminf(wn, wmax);
}

template <int STORAGE>
struct Voxels4;

template <>
struct Voxels4<kStorageF32> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W) {
    const float4* src = reinterpret_cast<const float4*>(m.pool) + (size_t)pool * 256 + 2 * t;
    const float4 a = src[0], b = src[1];
    D[0] = a.x; W[0] = a.y; D[1] = a.z; W[1] = a.w;
    D[2] = b.x; W[2] = b.y; D[3] = b.z; W[3] = b.w;
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W) {
    float4* dst = reinterpret_cast<float4*>(m.pool) + (size_t)pool * 256 + 2 * t;
    dst[0] = make_float4(D[0], W[0], D[1], W[1]);
    dst[1] = make_float4(D[2], W[2], D[3], W[3]);
  }
};

template <>
struct Voxels4<kStorageF16> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W) {
    const uint4 raw = reinterpret_cast<const uint4*>(m.pool)[(size_t)pool * 128 + t];
    const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2 h = *reinterpret_cast<const __half2*>(&w4[i]);
      D[i] = __low2float(h) * m.tau;
      W[i] = __high2float(h);
    }
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W) {
    uint32_t w4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2 h = __floats2half2_rn(D[i] * m.inv_tau, W[i]);
      w4[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    reinterpret_cast<uint4*>(m.pool)[(size_t)pool * 128 + t] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
};

template <int NF, int NM, int STORAGE>
__global__ void __launch_bounds__(kIntegrateThreads)
    integrate_kernel(const __grid_constant__ BatchParams<NF, NM> p) {
  __shared__ uint32_t s_begin[NM + 1];
  __shared__ uint32_t s_map, s_slot, s_mask;
  __shared__ int32_t s_val;
  __shared__ unsigned long long s_key;
  __shared__ unsigned long long s_upd[kIntegrateThreads / 32];
  const int t = threadIdx.x;
  if (t == 0) {
    // the batch's work = the concatenation of every map's list
    uint32_t acc = 0;
    for (int k = 0; k < p.n_maps; ++k) {
      s_begin[k] = acc;
      acc += min(__ldcg(p.maps[k].ctl), p.maps[k].list_cap);
    }
    s_begin[p.n_maps] = acc;
  }
  __syncthreads();
  const uint32_t n = s_begin[p.n_maps];
  // this thread's voxels: x = lx0 .. lx0 + 3 at (ly, lz)
  const int lx0 = (t & 1) * 4, ly = (t >> 1) & 7, lz = t >> 4;

  for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
    if (t == 0) {
      int mi = 0;
      while (mi + 1 < p.n_maps && e >= s_begin[mi + 1]) ++mi;
      const MapDev& m0 = p.maps[mi];
      const uint32_t slot = m0.list[e - s_begin[mi]];
      s_map = mi;
      s_slot = slot;
      s_val = m0.vals[slot];
      s_mask = m0.mask[slot];
      s_key = m0.keys[slot];
    }
    __syncthreads();
    const MapDev& m = p.maps[s_map];
    const int val = s_val;
    const bool fresh = val <= -2;
    const int pool = fresh ? -val - 2 : val;
    unsigned long long my_upd = 0;
    if (val != -1) {
      float D[4], W[4];
      if (fresh) {
#pragma unroll
        for (int i = 0; i < 4; ++i) { D[i] = 0.0f; W[i] = 0.0f; }
      } else {
        Voxels4<STORAGE>::load(m, pool, t, D, W);
      }
      const int bx = key_coord(s_key, 0), by = key_coord(s_key, 1), bz = key_coord(s_key, 2);
      uint32_t bits = s_mask;
      while (bits) {
        // bit k of the mask is frame k of the batch; frames apply in batch order
        const int f = __ffs(bits) - 1;
        bits &= bits - 1u;
        const FrameDev& F = p.fr[f];
        const int rx = (bx - F.a[0]) * 8 + lx0;
        const int ry = (by - F.a[1]) * 8 + ly;
        const int rz = (bz - F.a[2]) * 8 + lz;
        const float qy = __fmul_rn(__fadd_rn((float)ry, 0.5f), m.v);
        const float qz = __fmul_rn(__fadd_rn((float)rz, 0.5f), m.v);
        // innermost terms of p_i = fma(R_i0, qx, fma(R_i1, qy, fma(R_i2, qz, t_i)))
        const float cx = __fmaf_rn(F.Rcl[1], qy, __fmaf_rn(F.Rcl[2], qz, F.tloc[0]));
        const float cy = __fmaf_rn(F.Rcl[4], qy, __fmaf_rn(F.Rcl[5], qz, F.tloc[1]));
        const float cz = __fmaf_rn(F.Rcl[7], qy, __fmaf_rn(F.Rcl[8], qz, F.tloc[2]));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float qx = __fmul_rn(__fadd_rn((float)(rx + i), 0.5f), m.v);
          const float px = __fmaf_rn(F.Rcl[0], qx, cx);
          const float py = __fmaf_rn(F.Rcl[3], qx, cy);
          const float pz = __fmaf_rn(F.Rcl[6], qx, cz);
          float d, dv;
          if (!sample(F, m, px, py, pz, d, dv)) continue;
          const float dp = __fsub_rn(d, dv);
          if (dp < -m.tau) continue;
          fuse(D[i], W[i], fminf(dp, m.tau), m.wmax);
          ++my_upd;
        }
      }
      Voxels4<STORAGE>::store(m, pool, t, D, W);
    }
    // per-map update count: warp sums, one atomic per CTA and block
    for (int o = 16; o > 0; o >>= 1) my_upd += __shfl_down_sync(0xffffffffu, my_upd, o);
    if ((t & 31) == 0) s_upd[t >> 5] = my_upd;
    __syncthreads();
    if (t == 0) {
      unsigned long long tot = 0;
      for (int k = 0; k < kIntegrateThreads / 32; ++k) tot += s_upd[k];
      if (tot) atomicAdd(m.counters + kCntUpdates, tot);
      m.mask[s_slot] = 0u;
      if (fresh) m.vals[s_slot] = pool;
    }
  }
  // the last CTA to finish resets every map's work list for the next batch
  if (t == 0) {
    __threadfence();
    const unsigned done = atomicAdd(p.maps[0].ctl + 1, 1u);
    if (done == gridDim.x - 1) {
      for (int k = 0; k < p.n_maps; ++k) p.maps[k].ctl[0] = 0u;
      p.maps[0].ctl[1] = 0u;
    }
  }
}

template <int STORAGE>
__global__ void query_kernel(const MapDev m, const float* __restrict__ pts, int64_t n,
                             float* __restrict__ dist, float* __restrict__ weight) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float outD = 0.0f, outW = 0.0f;
  const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
  const float gx = floorf(__fdiv_rn(x, m.v)), gy = floorf(__fdiv_rn(y, m.v)), gz = floorf(__fdiv_rn(z, m.v));
  const float lim = 8.0f * 1048576.0f;
  if (fabsf(gx) < lim && fabsf(gy) < lim && fabsf(gz) < lim) {
    const int ix = (int)gx, iy = (int)gy, iz = (int)gz;
    const int slot = hash_find(m, pack_key(ix >> 3, iy >> 3, iz >> 3));
    if (slot >= 0) {
      const int val = m.vals[slot];
      if (val >= 0) {
        const int l = (ix & 7) + 8 * (iy & 7) + 64 * (iz & 7);
        if (STORAGE == kStorageF32) {
          const float2 v = reinterpret_cast<const float2*>(m.pool)[(size_t)val * 512 + l];
          outD = v.x;
          outW = v.y;
        } else {
          const __half2 h = reinterpret_cast<const __half2*>(m.pool)[(size_t)val * 512 + l];
          outD = __low2float(h) * m.tau;
          outW = __high2float(h);
        }
      }
    }
  }
  dist[i] = outD;
  weight[i] = outW;
}

__global__ void reset_kernel(const MapDev m, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    m.keys[i] = kEmptyKey;
    m.vals[i] = -1;
    m.mask[i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < kNumCounters) m.counters[threadIdx.x] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x < 2) m.ctl[threadIdx.x] = 0u;
}

}  // namespace

template <int NF, int NM>
cudaError_t launch_band_alloc(const BatchParams<NF, NM>& p, int n_ctas, cudaStream_t s) {
  if (n_ctas <= 0) return cudaSuccess;
  band_alloc_kernel<NF, NM><<<n_ctas, kAllocThreads, 0, s>>>(p);
  return cudaGetLastError();
}

template <int NF, int NM>
cudaError_t launch_integrate(const BatchParams<NF, NM>& p, int n_ctas, cudaStream_t s) {
  // all maps of a batch share one storage type (checked by the host API)
  if (p.maps[0].storage == kStorageF16)
    integrate_kernel<NF, NM, kStorageF16><<<n_ctas, kIntegrateThreads, 0, s>>>(p);
  else
    integrate_kernel<NF, NM, kStorageF32><<<n_ctas, kIntegrateThreads, 0, s>>>(p);
  return cudaGetLastError();
}

template cudaError_t launch_band_alloc<1, 1>(const BatchParams<1, 1>&, int, cudaStream_t);
template cudaError_t launch_band_alloc<kMaxFrames, kMaxMaps>(const BatchParams<kMaxFrames, kMaxMaps>&,
                                                             int, cudaStream_t);
template cudaError_t launch_integrate<1, 1>(const BatchParams<1, 1>&, int, cudaStream_t);
template cudaError_t launch_integrate<kMaxFrames, kMaxMaps>(const BatchParams<kMaxFrames, kMaxMaps>&,
                                                            int, cudaStream_t);

cudaError_t launch_query(const MapDev& m, const float* pts, int64_t n, float* dist, float* weight,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (m.storage == kStorageF16)
    query_kernel<kStorageF16><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  else
    query_kernel<kStorageF32><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  return cudaGetLastError();
}

cudaError_t launch_reset(const MapDev& m, uint32_t cap, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  reset_kernel<<<sms * 4, 256, 0, s>>>(m, cap);
  return cudaGetLastError();
}

int integrate_ctas_per_sm(int storage) {
  int n = 0;
  cudaError_t e;
  if (storage == kStorageF16)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, integrate_kernel<kMaxFrames, kMaxMaps, kStorageF16>, kIntegrateThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, integrate_kernel<kMaxFrames, kMaxMaps, kStorageF32>, kIntegrateThreads, 0);
  if (e != cudaSuccess || n <= 0) n = 4;
  return n;
}

}  // namespace gbt
