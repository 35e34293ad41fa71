// CUDA kernels of the GB300 TSDF library (sm_103a).
//
//  band_alloc_kernel  Sec. IV-B first step: one CTA per pixel tile; every
//                     valid pixel's ray segment inside the truncation band is
//                     walked through the block grid (Amanatides & Woo
//                     traversal) and its blocks recorded in a CTA-local set
//                     in shared memory; the tile's distinct blocks are then
//                     claimed in the open-addressing hash (atomicCAS on the
//                     packed key), given a pool block if new, and get the
//                     frame's bit; the first bit on a block appends it to
//                     the batch work list.
//  integrate_kernel   Sec. IV-B second step (Eq. 1-3 and the update
//                     functors: TSDF, occupancy, colour): persistent CTAs
//                     take work-list blocks, 4 voxels per thread held in
//                     registers across every frame of the batch that met the
//                     block, one coalesced read and write per block and
//                     batch.
//  query_kernel,      point -> voxel lookup through the hash.
//  query_color_kernel
//  decay_kernel       occupancy decay over every allocated block (Sec. V-E).
//
// Discrete decisions use explicit round-to-nearest intrinsics in a fixed
// order (no contraction) so that they are reproducible on a CPU.
#include <algorithm>
#include <cfloat>

#include "tsdf_internal.cuh"

namespace gbt {
namespace {

// Programmatic dependent launch: a kernel launched with BatchParams::overlap
// may be scheduled while the stream's previous kernel is still running; it
// waits here, before its first memory access, until that kernel has
// completed and its writes are visible.  Such a kernel lets the next one be
// scheduled once its CTAs have done their main work.  Ordinary launches skip
// both instructions.
__device__ __forceinline__ void wait_prev_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr float kPiF = (float)3.14159265358979323846;
constexpr float kHalfPiF = (float)(3.14159265358979323846 / 2);

// IEEE round-to-nearest reciprocal of a decision input.  FAST: the hardware
// approximation (within 1 ulp) refined by one Newton step with fused
// multiply-adds, e = 1 - x y, y' = y + y e (Markstein's method), which equals
// __frcp_rn(x) bit for bit for |x| in [2^-126, 2^126] (checked over all
// 4,227,858,434 such inputs).  The host selects FAST kernels only for
// batches whose inverted values all lie in that range or are zero (zero is
// never inverted), see fast_rcp_ok in the host code.
template <bool FAST>
__device__ __forceinline__ float rcp_dec(float x) {
  if (!FAST) return __frcp_rn(x);
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  const float e = __fmaf_rn(-x, y, 1.0f);
  return __fmaf_rn(y, e, y);
}

// rcp_dec of a pair: the two refinement steps on the paired FP32
// operations (per component the same round-to-nearest result).
template <bool FAST>
__device__ __forceinline__ float2 rcp_dec2(float a, float b) {
  if (!FAST) return make_float2(__frcp_rn(a), __frcp_rn(b));
  float2 y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(a));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(b));
  const float2 e = __ffma2_rn(make_float2(-a, -b), y, make_float2(1.0f, 1.0f));
  return __ffma2_rn(y, e, y);
}

// ------------------------------------------------------------------ hash

__device__ __forceinline__ int hash_insert(const MapDev& m, unsigned long long key, bool& inserted) {
  uint32_t slot = hash_key(key) & m.cap_mask;
  inserted = false;
  // one atomic per probed slot: it inserts into an empty slot and reports
  // the slot's key otherwise (a single L2 round trip when the key is found)
  for (uint32_t probe = 0; probe <= m.cap_mask; ++probe) {
    const unsigned long long old = atomicCAS(m.keys + slot, kEmptyKey, key);
    if (old == kEmptyKey) {
      inserted = true;
      return (int)slot;
    }
    if (old == key) return (int)slot;
    slot = (slot + 1) & m.cap_mask;
  }
  return -1;
}

// ------------------------------------------------- block-grid traversal

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
  if (atomicOr(m.mask + slot, 1u << bit) == 0u) {
    const uint32_t idx = atomicAdd(m.ctl, 1u);
    if (idx < m.list_cap) m.list[idx] = (uint32_t)slot;
    else atomicOr(m.counters + kCntStatus, (unsigned long long)kStListFull);
  }
}

// Walk in anchor-relative cell coordinates with a 32-bit key
// (cx + 512) | (cy + 512) << 10 | (cz + 512) << 20; used when the segment
// starts within kRelStart cells of the anchor, so that every cell of the walk
// (at most kMaxCells steps) stays inside the 10-bit fields.  The decisions
// are the prescribed FP32 sequence of the traversal, cell for cell.
constexpr int kRelBias = 512;
constexpr float kRelStart = 470.0f;
constexpr uint32_t kEmptyRel = 0xFFFFFFFFu;

// The sensor origin o is not stored: it is frame-wide (uniform across the
// CTA) and passed to every step, which keeps the per-lane state small (the
// allocator is compiled for 32 registers a thread: 8 CTAs of 256 threads per
// SM; measured faster than 40 registers without spills at 6 CTAs).
struct Walk32 {
  uint32_t key;
  uint32_t kx, ky, kz;  // key change of one step along each axis (+unit, -unit, 0)
  float bx, by, bz;     // next boundary per axis (+inf for an axis the ray does not cross)
  float ix, iy, iz;      // reciprocal direction per axis
  float s1;
  int n;

  // t of an axis is always (b - o) * inv; an axis with zero direction has
  // b = +inf and inv = 1, so its t is +inf.
  template <bool FAST>
  __device__ __forceinline__ void axis(float d, float fl, uint32_t unit, uint32_t& k, float& inv, float& b) {
    const bool pos = d > 0.0f, neg = d < 0.0f;
    k = pos ? unit : (neg ? 0u - unit : 0u);
    inv = (pos || neg) ? rcp_dec<FAST>(d) : 1.0f;
    b = pos ? fl + 1.0f : (neg ? fl : __int_as_float(0x7f800000));
  }
  template <bool FAST>
  __device__ __forceinline__ void start(float px, float py, float pz, float dx, float dy, float dz,
                                        float s1_, int bx0, int by0, int bz0, uint32_t flag) {
    const float flx = floorf(px), fly = floorf(py), flz = floorf(pz);
    key = ((uint32_t)((int)flx - bx0 + kRelBias) | ((uint32_t)((int)fly - by0 + kRelBias) << 10) |
           ((uint32_t)((int)flz - bz0 + kRelBias) << 20)) | flag;
    axis<FAST>(dx, flx, 1u, kx, ix, bx);
    axis<FAST>(dy, fly, 1u << 10, ky, iy, by);
    axis<FAST>(dz, flz, 1u << 20, kz, iz, bz);
    s1 = s1_;
    n = 1;
  }
  // The crossing parameters are recomputed from the boundaries at every
  // step, not carried: they are dead while the cell's key is recorded (at 32
  // registers a thread, carrying them spilled 88 bytes; 94.6 against 97.7 us
  // per 32-frame launch).  CAP: stop after kMaxCells cells; without it the
  // host has proved that every segment of the batch ends sooner (the cell
  // count then needs no register and no test).
  template <bool CAP>
  __device__ __forceinline__ bool next(float ox, float oy, float oz) {
    const float tx = __fmul_rn(__fsub_rn(bx, ox), ix);
    const float ty = __fmul_rn(__fsub_rn(by, oy), iy);
    const float tz = __fmul_rn(__fsub_rn(bz, oz), iz);
    const bool sy_ = ty < tx;
    const float t01 = fminf(tx, ty);
    const bool sz_ = tz < t01;
    const float t = fminf(t01, tz);
    if (!(t <= s1) || (CAP && n == kMaxCells)) return false;
    const bool sx_ = !sz_ && !sy_, syy = !sz_ && sy_;
    const uint32_t dk = sz_ ? kz : (sy_ ? ky : kx);
    key += dk;
    // the boundary moves by +1 or -1 along the stepped axis: the sign of its
    // key change (never 0: an axis the ray does not cross has t = +inf)
    const float f = __uint_as_float((dk & 0x80000000u) | 0x3f800000u);
    // predicated additions (an unconditional add of 0 costs a select more)
    if (sx_) bx = __fadd_rn(bx, f);
    if (syy) by = __fadd_rn(by, f);
    if (sz_) bz = __fadd_rn(bz, f);
    if (CAP) ++n;
    return true;
  }
};

__device__ __forceinline__ unsigned long long rel_to_key(uint32_t r, const int* a, int bx0 = 0,
                                                         int by0 = 0, int bz0 = 0) {
  return pack_key(a[0] + bx0 + (int)(r & 1023u) - kRelBias,
                  a[1] + by0 + (int)((r >> 10) & 1023u) - kRelBias,
                  a[2] + bz0 + (int)((r >> 20) & 1023u) - kRelBias);
}
constexpr uint32_t kFarFlag = 1u << 30;  // key counted from the segment's own start cell

// CTA-local set of relative block keys (open addressing in shared memory):
// `set` holds kSetSize slots, `keys` receives each key when it first enters
// the set (appended at *nkeys), so the tile's distinct blocks need no scan of
// the slots afterwards.  Returns false when the key could not be placed
// within kSetProbes slots, or is a far segment's key (bit 30: counted from
// the segment's own start cell, never in the set; it cannot match a slot,
// which holds a near key or kEmptyRel, so it always reaches the slow path);
// the caller then claims it globally itself.  The probing loop is inlined:
// at the allocator's 32 registers a call's saves and restores cost more
// than the larger code (measured 5 % slower as a call).
__device__ __forceinline__ bool set_insert_slow(uint32_t* set, uint32_t* keys, uint32_t* nkeys,
                                                uint32_t key, uint32_t h);

__device__ __forceinline__ bool set_insert(uint32_t* set, uint32_t* keys, uint32_t* nkeys, uint32_t key) {
  const uint32_t h = (key * 0x9E3779B1u) >> (32 - kSetBits);
  // common case: the key is already at its home slot
  if (((volatile uint32_t*)set)[h] == key) return true;
  return set_insert_slow(set, keys, nkeys, key, h);
}

__device__ __forceinline__ bool set_insert_slow(uint32_t* set, uint32_t* keys, uint32_t* nkeys,
                                                uint32_t key, uint32_t h) {
  if (key & kFarFlag) return false;
  volatile uint32_t* vs = set;
#pragma unroll 1
  for (int probe = 0; probe < kSetProbes; ++probe) {
    const uint32_t cur = vs[h];
    if (cur == key) return true;
    if (cur == kEmptyRel) {
      const uint32_t old = atomicCAS(set + h, kEmptyRel, key);
      if (old == kEmptyRel) {
        keys[atomicAdd(nkeys, 1u)] = key;  // at most kSetSize distinct keys
        return true;
      }
      if (old == key) return true;
    }
    h = (h + 1) & (kSetSize - 1);
  }
  return false;
}

// Band segment of pixel (i, j) (Sec. IV-B ray through the block grid): ray
// direction in anchor-relative block units per unit of depth (camera) or
// range (LiDAR) and the band [max(d - tau, 0), d + tau].  False if the pixel
// is outside the image or its depth is invalid.  A pinhole pixel outside the
// image was given depth 0, which is invalid; its ray is computed and unused.
// Pinhole rays: d = (fma(M0, rx, c0), fma(M3, rx, c1), fma(M6, rx, c2)) with
// the row's c = fma(M[3k+1], ry, M[3k+2]) staged once per tile row.
template <bool PINHOLE_ONLY>
__device__ __forceinline__ bool pixel_segment(const FrameDev& F, const MapDev& m,
                                              const float* s_ray, int i, int j, int lane, int ty,
                                              float d, float& dx, float& dy, float& dz, float& s0,
                                              float& s1) {
  bool valid;
  if (PINHOLE_ONLY || F.kind == kSensorPinhole) {
    valid = d > 0.0f && d <= FLT_MAX;
    const float rx = s_ray[lane];
    const float4 c = reinterpret_cast<const float4*>(s_ray + kTileW)[ty];
    dx = __fmaf_rn(F.M[0], rx, c.x);
    dy = __fmaf_rn(F.M[3], rx, c.y);
    dz = __fmaf_rn(F.M[6], rx, c.z);
  } else {
    if (i >= F.width || j >= F.height) return false;
    valid = d >= F.min_range && d <= F.max_range;
    const float2 az = __ldg(reinterpret_cast<const float2*>(F.tab) + i);
    const float2 el = __ldg(reinterpret_cast<const float2*>(F.tab) + F.width + j);
    const float bx = __fmul_rn(el.y, az.x), by = __fmul_rn(el.y, az.y), bz = el.x;
    dx = __fmaf_rn(F.M[0], bx, __fmaf_rn(F.M[1], by, __fmul_rn(F.M[2], bz)));
    dy = __fmaf_rn(F.M[3], bx, __fmaf_rn(F.M[4], by, __fmul_rn(F.M[5], bz)));
    dz = __fmaf_rn(F.M[6], bx, __fmaf_rn(F.M[7], by, __fmul_rn(F.M[8], bz)));
  }
  s0 = fmaxf(__fsub_rn(d, m.tau), 0.0f);
  s1 = __fadd_rn(d, m.tau);
  return valid;
}

// Shared memory of one allocation tile.
template <int TH>
struct AllocSmem {
  uint32_t set[kSetSize];   // CTA-local set of relative block keys
  uint32_t keys[kSetSize];  // the set's keys, in order of first insertion
  uint32_t nkeys;
  // pinhole: rx = (i - cu) / fu per column, then per row the three
  // fma(M[3k+1], ry, M[3k+2]) with ry = (j - cv) / fv (and one pad word)
  __align__(16) float ray[kTileW + 4 * TH];
};

// Allocation tile `cta` of the batch (tiles are numbered frame by frame,
// FrameDev::blk_begin being a frame's first), run by all kAllocThreads
// threads of a CTA.  With p.overlap the stream's next kernel may be
// scheduled once the walks are done.
template <int NF, int NM, int TH, bool PINHOLE_ONLY, bool STATS, bool FAST, bool CAP>
__device__ __forceinline__ void alloc_tile(const BatchParams<NF, NM>& p, int cta, AllocSmem<TH>& sm) {
  constexpr int kRows = TH * kTileW / kAllocThreads;  // pixel rows per thread
  uint32_t segs = 0, cells = 0;                        // walk statistics
  uint32_t* s_set = sm.set;
  uint32_t* s_keys = sm.keys;
  float* s_ray = sm.ray;
  __syncthreads();  // a previous tile of this CTA is done with the shared arrays
  for (int i = threadIdx.x; i < kSetSize; i += kAllocThreads) s_set[i] = kEmptyRel;
  if (threadIdx.x == 0) sm.nkeys = 0;
  // frame of this tile: the last frame whose first tile is <= cta
  int f = 0;
  for (int lo = 1, hi = p.n_frames - 1; lo <= hi;) {
    const int mid = (lo + hi) >> 1;
    if (cta >= p.fr[mid].blk_begin) {
      f = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  const FrameDev& F = p.fr[f];
  // with one map its fields are constant operands, not indexed loads
  const MapDev& m = NM == 1 ? p.maps[0] : p.maps[F.map];
  const int tiles_x = (F.width + kTileW - 1) / kTileW;
  const int tile = cta - F.blk_begin;
  const int x0 = (tile % tiles_x) * kTileW, y0 = (tile / tiles_x) * TH;
  const int lane = threadIdx.x % kTileW, wy = threadIdx.x / kTileW;
  // all of this thread's depths are requested before any is used
  float dep[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int i = x0 + lane, j = y0 + wy + q * (kAllocThreads / kTileW);
    dep[q] = (i < F.width && j < F.height) ? __ldg(F.depth + (size_t)j * F.width + i) : 0.0f;
  }
  if (PINHOLE_ONLY || F.kind == kSensorPinhole) {
    if (threadIdx.x < kTileW)
      s_ray[threadIdx.x] = __fdiv_rn(__fsub_rn((float)(x0 + (int)threadIdx.x), F.cu), F.fu);
    else if (threadIdx.x < kTileW + TH) {
      const float ry = __fdiv_rn(__fsub_rn((float)(y0 + (int)threadIdx.x - kTileW), F.cv), F.fv);
      reinterpret_cast<float4*>(s_ray + kTileW)[threadIdx.x - kTileW] =
          make_float4(__fmaf_rn(F.M[1], ry, F.M[2]), __fmaf_rn(F.M[4], ry, F.M[5]),
                      __fmaf_rn(F.M[7], ry, F.M[8]), 0.0f);
    }
  }
  __syncthreads();

#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int ty = wy + q * (kAllocThreads / kTileW);
    bool live = false;
    Walk32 wk;
    wk.key = kEmptyRel;
    int b0x = 0, b0y = 0, b0z = 0;  // key origin of a far segment
    float dx, dy, dz, s0, s1;
    if (pixel_segment<PINHOLE_ONLY>(F, m, s_ray, x0 + lane, y0 + ty, lane, ty, dep[q], dx, dy, dz, s0, s1)) {
      const float px = __fmaf_rn(s0, dx, F.o[0]), py = __fmaf_rn(s0, dy, F.o[1]),
                  pz = __fmaf_rn(s0, dz, F.o[2]);
      if (fabsf(px) < kRelStart && fabsf(py) < kRelStart && fabsf(pz) < kRelStart) {
        wk.start<FAST>(px, py, pz, dx, dy, dz, s1, 0, 0, 0, 0u);
        live = true;
      } else if (fabsf(px) < 262144.0f && fabsf(py) < 262144.0f && fabsf(pz) < 262144.0f) {
        // far from the sensor's block (long range or small voxels): count
        // cells from the start cell and claim them globally one by one
        b0x = (int)floorf(px);
        b0y = (int)floorf(py);
        b0z = (int)floorf(pz);
        wk.start<FAST>(px, py, pz, dx, dy, dz, s1, b0x, b0y, b0z, kFarFlag);
        live = true;
      }
    }
    segs += live ? 1u : 0u;
    while (__any_sync(0xffffffffu, live)) {
      if (live) {
        ++cells;
        if (!set_insert(s_set, s_keys, &sm.nkeys, wk.key)) {
          if (wk.key & kFarFlag)
            claim_block(m, rel_to_key(wk.key & ~kFarFlag, F.a, b0x, b0y, b0z), F.bit);
          else
            claim_block(m, rel_to_key(wk.key, F.a), F.bit);
        }
        live = wk.template next<CAP>(F.o[0], F.o[1], F.o[2]);
      }
    }
  }
  if (p.overlap) allow_next_grid();
  __syncthreads();
  // the tile's distinct blocks, claimed one per thread
  const uint32_t nk = sm.nkeys;
  for (uint32_t i = threadIdx.x; i < nk; i += kAllocThreads) claim_block(m, rel_to_key(s_keys[i], F.a), F.bit);
  if (STATS) {
    for (int o = 16; o > 0; o >>= 1) {
      segs += __shfl_down_sync(0xffffffffu, segs, o);
      cells += __shfl_down_sync(0xffffffffu, cells, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(m.counters + kCntSegments, (unsigned long long)segs);
      atomicAdd(m.counters + kCntCells, (unsigned long long)cells);
    }
  }
}

// One CTA per kTileW x TH pixel tile of one frame.  Each warp walks the
// band segments of one pixel row at a time and records the blocks met in a
// CTA-local set; then the tile's distinct blocks are claimed in the global
// hash.  Segments that start far from the sensor's block count cells from
// their own start cell and claim their blocks directly.  PINHOLE_ONLY: every
// frame of the batch is a pinhole camera (the LiDAR code is left out);
// STATS: count band segments and walked cells (a diagnostic, 5 % slower);
// FAST: reciprocals by rcp_dec<true> (the host checked their range); CAP:
// walks stop after kMaxCells cells (without it the host proved them shorter).
template <int NF, int NM, int TH, bool PINHOLE_ONLY, bool STATS, bool FAST, bool CAP>
__global__ void __launch_bounds__(kAllocThreads, 7)
    band_alloc_kernel(const __grid_constant__ BatchParams<NF, NM> p) {
  if (p.overlap) wait_prev_grid();
  __shared__ AllocSmem<TH> sm;
  alloc_tile<NF, NM, TH, PINHOLE_ONLY, STATS, FAST, CAP>(p, (int)blockIdx.x, sm);
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

// Azimuth column k in [-1, naz] wrapped into [0, naz).
__device__ __forceinline__ int wrap_az(int k, int naz) {
  return k < 0 ? k + naz : (k >= naz ? k - naz : k);
}

__device__ __forceinline__ bool lidar_valid(const FrameDev& F, float d) {
  return d >= F.min_range && d <= F.max_range;
}

// TSDF update functor (Sec. IV-B): weighted running average, the average
// taken with the unclamped weight sum, then weights capped; a zero weight on
// an unobserved voxel changes nothing.
__device__ __forceinline__ void fuse(float& D, float& W, float s, float w, float wmax) {
  const float wn = W + w;
  if (!(wn > 0.0f)) return;
  D = D + __fdividef(w * (s - D), wn);
  W = fminf(wn, wmax);
}

// Weight f_w(d_p) (Sec. IV-B: constant or from the sensor's error model):
// 1, times 1 / d_v^2 for inverse-square weighting, times a linear drop-off
// from 1 at d_p = -dropoff to 0 at d_p = -tau behind the surface.
__device__ __forceinline__ float weight(const MapDev& m, float dv, float dp) {
  float w = 1.0f;
  if (m.weighting & 1) w = __fdividef(1.0f, dv * dv);
  if ((m.weighting & 2) && dp < -m.dropoff) w *= __fdividef(m.tau + dp, m.tau - m.dropoff);
  return w;
}

// Update functor of a voxel that passed the projection test, d_p >= -tau:
// the TSDF average, or for an occupancy layer (Sec. IV-B, second functor)
// the running addition of l_free in front of the surface (d_p > 0) and
// l_occ otherwise.
// WEIGHTED: the map uses a non-constant weighting function (the constant
// weight 1 keeps the update short: fewer instructions in the unrolled loops).
template <int STORAGE, bool WEIGHTED>
__device__ __forceinline__ void apply(const MapDev& m, float& D, float& W, float dv, float dp) {
  if (STORAGE == kStorageOcc) {
    D += dp > 0.0f ? m.l_free : m.l_occ;
  } else if (WEIGHTED) {
    fuse(D, W, fminf(dp, m.tau), weight(m, dv, dp), m.wmax);
  } else {
    const float wn = W + 1.0f;
    D = D + __fdividef(fminf(dp, m.tau) - D, wn);
    W = fminf(wn, m.wmax);
  }
}

// Colour functor: the running average of the pixel's r, g, b with weight 1
// per frame (the TSDF average applied per channel), weights capped.
__device__ __forceinline__ void apply_color(const MapDev& m, float& R, float& G, float& B, float& W,
                                            uint32_t c) {
  const float wn = W + 1.0f;
  const float iw = __frcp_rn(wn);
  R = __fmaf_rn(__fsub_rn((float)(c & 255u), R), iw, R);
  G = __fmaf_rn(__fsub_rn((float)((c >> 8) & 255u), G), iw, G);
  B = __fmaf_rn(__fsub_rn((float)((c >> 16) & 255u), B), iw, B);
  W = fminf(wn, m.wmax);
}

// A thread's four voxels in registers: D and W (TSDF distance and weight,
// occupancy log-odds, or colour red and weight) and, for colour only, G and B.
template <int STORAGE>
struct Voxels4;

template <>
struct Voxels4<kStorageF32> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W,
                                              float* G, float* B) {
    const float4* src = reinterpret_cast<const float4*>(m.pool) + (size_t)pool * 256 + 2 * t;
    const float4 a = src[0], b = src[1];
    D[0] = a.x; W[0] = a.y; D[1] = a.z; W[1] = a.w;
    D[2] = b.x; W[2] = b.y; D[3] = b.z; W[3] = b.w;
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W, const float* G, const float* B) {
    float4* dst = reinterpret_cast<float4*>(m.pool) + (size_t)pool * 256 + 2 * t;
    dst[0] = make_float4(D[0], W[0], D[1], W[1]);
    dst[1] = make_float4(D[2], W[2], D[3], W[3]);
  }
};

template <>
struct Voxels4<kStorageOcc> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W,
                                              float* G, float* B) {
    const float4 a = reinterpret_cast<const float4*>(m.pool)[(size_t)pool * 128 + t];
    D[0] = a.x; D[1] = a.y; D[2] = a.z; D[3] = a.w;
    W[0] = W[1] = W[2] = W[3] = 0.0f;
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W, const float* G, const float* B) {
    reinterpret_cast<float4*>(m.pool)[(size_t)pool * 128 + t] = make_float4(D[0], D[1], D[2], D[3]);
  }
};

template <>
struct Voxels4<kStorageF16> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W,
                                              float* G, float* B) {
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
                                               const float* W, const float* G, const float* B) {
    uint32_t w4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2 h = __floats2half2_rn(D[i] * m.inv_tau, W[i]);
      w4[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    reinterpret_cast<uint4*>(m.pool)[(size_t)pool * 128 + t] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
};

template <>
struct Voxels4<kStorageX16> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W,
                                              float* G, float* B) {
    const uint4 raw = reinterpret_cast<const uint4*>(m.pool)[(size_t)pool * 128 + t];
    const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      D[i] = x16_dist(w4[i], m.x16_unit);
      W[i] = x16_weight(w4[i]);
    }
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W, const float* G, const float* B) {
    reinterpret_cast<uint4*>(m.pool)[(size_t)pool * 128 + t] =
        make_uint4(x16_pack(D[0], W[0], m.x16_scale), x16_pack(D[1], W[1], m.x16_scale),
                   x16_pack(D[2], W[2], m.x16_scale), x16_pack(D[3], W[3], m.x16_scale));
  }
};

template <>
struct Voxels4<kStorageColor> {
  __device__ __forceinline__ static void load(const MapDev& m, int pool, int t, float* D, float* W,
                                              float* G, float* B) {
    const float4* src = reinterpret_cast<const float4*>(m.pool) + (size_t)pool * 512 + 4 * t;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 a = src[i];
      D[i] = a.x; G[i] = a.y; B[i] = a.z; W[i] = a.w;
    }
  }
  __device__ __forceinline__ static void store(const MapDev& m, int pool, int t, const float* D,
                                               const float* W, const float* G, const float* B) {
    float4* dst = reinterpret_cast<float4*>(m.pool) + (size_t)pool * 512 + 4 * t;
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = make_float4(D[i], G[i], B[i], W[i]);
  }
};

// A thread's four voxels: block (bx, by, bz), local x = lx0 .. lx0 + 3 at
// local (ly, lz).
struct VoxelRow {
  int bx, by, bz, lx0, ly, lz;
};

// Voxel centres of a row in frame F's sensor frame (Eq. 1), in the FP32
// decision sequence p_i = fma(R_i0, qx, fma(R_i1, qy, fma(R_i2, qz, t_i))).
__device__ __forceinline__ void row_points(const FrameDev& F, float v, const VoxelRow& r,
                                           float* px, float* py, float* pz) {
  const int rx = (r.bx - F.a[0]) * 8 + r.lx0;
  const int ry = (r.by - F.a[1]) * 8 + r.ly;
  const int rz = (r.bz - F.a[2]) * 8 + r.lz;
  const float qy = __fmul_rn(__fadd_rn((float)ry, 0.5f), v);
  const float qz = __fmul_rn(__fadd_rn((float)rz, 0.5f), v);
  const float cx = __fmaf_rn(F.Rcl[1], qy, __fmaf_rn(F.Rcl[2], qz, F.tloc[0]));
  const float cy = __fmaf_rn(F.Rcl[4], qy, __fmaf_rn(F.Rcl[5], qz, F.tloc[1]));
  const float cz = __fmaf_rn(F.Rcl[7], qy, __fmaf_rn(F.Rcl[8], qz, F.tloc[2]));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float qx = __fmul_rn(__fadd_rn((float)(rx + i), 0.5f), v);
    px[i] = __fmaf_rn(F.Rcl[0], qx, cx);
    py[i] = __fmaf_rn(F.Rcl[3], qx, cy);
    pz[i] = __fmaf_rn(F.Rcl[6], qx, cz);
  }
}

// A pinhole frame's projection constants, staged in shared memory once per
// CTA: six 16-byte loads per frame in the voxel loop instead of one
// constant-bank load per field (the frame index is not known at compile
// time, so the fields cannot be instruction operands).
struct __align__(16) FrameProj {
  float4 r0, r1, r2;  // rows of R_CL, with t_loc in w
  float4 cam;         // fu, fv, cu, cv
  int4 anchor;        // a, width
  float4 size;        // width, height (as floats), height (integer bits), unused
};

__device__ __forceinline__ void stage_frame(const FrameDev& F, FrameProj& S) {
  S.r0 = make_float4(F.Rcl[0], F.Rcl[1], F.Rcl[2], F.tloc[0]);
  S.r1 = make_float4(F.Rcl[3], F.Rcl[4], F.Rcl[5], F.tloc[1]);
  S.r2 = make_float4(F.Rcl[6], F.Rcl[7], F.Rcl[8], F.tloc[2]);
  S.cam = make_float4(F.fu, F.fv, F.cu, F.cv);
  S.anchor = make_int4(F.a[0], F.a[1], F.a[2], F.width);
  S.size = make_float4((float)F.width, (float)F.height, __int_as_float(F.height), 0.0f);
}

// row_points with staged constants (same arithmetic).
__device__ __forceinline__ void row_points_staged(const float4& r0, const float4& r1, const float4& r2,
                                                  const int4& an, float v, const VoxelRow& r,
                                                  float* px, float* py, float* pz) {
  const int rx = (r.bx - an.x) * 8 + r.lx0;
  const int ry = (r.by - an.y) * 8 + r.ly;
  const int rz = (r.bz - an.z) * 8 + r.lz;
  const float qy = __fmul_rn(__fadd_rn((float)ry, 0.5f), v);
  const float qz = __fmul_rn(__fadd_rn((float)rz, 0.5f), v);
  const float cx = __fmaf_rn(r0.y, qy, __fmaf_rn(r0.z, qz, r0.w));
  const float cy = __fmaf_rn(r1.y, qy, __fmaf_rn(r1.z, qz, r1.w));
  const float cz = __fmaf_rn(r2.y, qy, __fmaf_rn(r2.z, qz, r2.w));
  const float fx = (float)rx;  // rx + i is exact in FP32 (|rx| < 2^24)
  // voxel pairs on the paired FP32 operations (per component the same
  // round-to-nearest result as the scalar ones)
  const float2 half = make_float2(0.5f, 0.5f), vv = make_float2(v, v);
  const float2 c0 = make_float2(cx, cx), c1 = make_float2(cy, cy), c2 = make_float2(cz, cz);
  const float2 a0 = make_float2(r0.x, r0.x), a1 = make_float2(r1.x, r1.x), a2 = make_float2(r2.x, r2.x);
#pragma unroll
  for (int i = 0; i < 4; i += 2) {
    const float2 qx = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(fx, fx), make_float2((float)i, (float)(i + 1))),
                                            half), vv);
    const float2 x = __ffma2_rn(a0, qx, c0), y = __ffma2_rn(a1, qx, c1), z = __ffma2_rn(a2, qx, c2);
    px[i] = x.x; px[i + 1] = x.y;
    py[i] = y.x; py[i + 1] = y.y;
    pz[i] = z.x; pz[i + 1] = z.y;
  }
}

// PAIRED_RCP: the projection reciprocals refined on the paired operations
// (pinhole-only kernels; in the kernels with the LiDAR path it raised the
// register count from 72 to 79, one resident CTA per SM fewer).
// NQ consecutive pinhole frames of the batch: phase 1 projects every voxel
// into every frame (Eq. 2, nearest pixel) and issues all depth loads (and
// colour loads for a colour layer), phase 2 applies the updates in frame
// order.  An out-of-image projection reads no pixel and yields d = 0, which
// is invalid like a missing depth.  A colour layer updates only voxels within
// tau of the surface on both sides.
template <int NQ, int STORAGE, bool WEIGHTED, bool FAST, bool PAIRED_RCP, class P>
__device__ __forceinline__ void fuse_pinhole(const P& p, const FrameProj* s_fp, const int (&fq)[4],
                                             const MapDev& m, const VoxelRow& r, float* D, float* W,
                                             float* G, float* B, unsigned long long& upd) {
  float d[NQ][4], z[NQ][4];
  uint32_t c[NQ][4];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const FrameProj& S = s_fp[fq[q]];
    const float4 r0 = S.r0, r1 = S.r1, r2 = S.r2, cam = S.cam, size = S.size;
    const int4 an = S.anchor;
    const float* depth = p.fr[fq[q]].depth;
    float px[4], py[4];
    row_points_staged(r0, r1, r2, an, m.v, r, px, py, z[q]);
    // pixel coordinates of voxel pairs on the paired FP32 operations
    float uu[4], vv[4];
    const float2 fu2 = make_float2(cam.x, cam.x), cu2 = make_float2(cam.z, cam.z);
    const float2 fv2 = make_float2(cam.y, cam.y), cv2 = make_float2(cam.w, cam.w);
    const float2 half = make_float2(0.5f, 0.5f);
#pragma unroll
    for (int i = 0; i < 4; i += 2) {
      const float2 iz = PAIRED_RCP ? rcp_dec2<FAST>(z[q][i], z[q][i + 1])
                                   : make_float2(rcp_dec<FAST>(z[q][i]), rcp_dec<FAST>(z[q][i + 1]));
      const float2 u = __fadd2_rn(__ffma2_rn(__fmul2_rn(make_float2(px[i], px[i + 1]), iz), fu2, cu2), half);
      const float2 v = __fadd2_rn(__ffma2_rn(__fmul2_rn(make_float2(py[i], py[i + 1]), iz), fv2, cv2), half);
      uu[i] = u.x; uu[i + 1] = u.y;
      vv[i] = v.x; vv[i + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float u = uu[i], v = vv[i];
      bool in;
      int pix;
      if (FAST) {
        // pixel = floor(u), valid iff 0 <= u < W: one unsigned comparison of
        // the floored value per axis (u is finite here: z > 0 implies
        // z >= 2^-126 in FAST batches, so 1 / z is finite)
        const int iu = __float2int_rd(u), iv = __float2int_rd(v);
        in = z[q][i] > 0.0f && (unsigned)iu < (unsigned)an.w && (unsigned)iv < (unsigned)__float_as_int(size.z);
        pix = iv * an.w + iu;
      } else {
        in = z[q][i] > 0.0f && u >= 0.0f && u < size.x && v >= 0.0f && v < size.y;
        pix = (int)v * an.w + (int)u;
      }
      if (STORAGE == kStorageColor) {
        d[q][i] = in ? __ldg(depth + pix) : 0.0f;
        c[q][i] = in ? __ldg(p.fr[fq[q]].rgba + pix) : 0u;
      } else {
        d[q][i] = in ? __ldg(depth + pix) : 0.0f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float dp = __fsub_rn(d[q][i], z[q][i]);
      // a valid depth, 0 < d <= FLT_MAX: one unsigned comparison of its bits
      if ((__float_as_uint(d[q][i]) - 1u) < 0x7F7FFFFFu && !(dp < -m.tau)) {
        if (STORAGE == kStorageColor) {
          if (dp > m.tau) continue;
          apply_color(m, D[i], G[i], B[i], W[i], c[q][i]);
        } else {
          apply<STORAGE, WEIGHTED>(m, D[i], W[i], z[q][i], dp);
        }
        ++upd;
      }
    }
}

// A LiDAR frame (Eq. 1 and 3): phase 1 finds every voxel's beam cell and
// issues its range loads (the four around it, or the nearest one), phase 2
// applies the guarded bilinear sample and the updates.  A voxel at the
// sensor origin, outside the elevation rows or with an invalid sample is not
// updated; azimuth wraps.  Colour layers take pinhole frames only.
template <int STORAGE, bool WEIGHTED>
__device__ __forceinline__ void fuse_lidar(const FrameDev& F, const MapDev& m, const VoxelRow& r,
                                           float* D, float* W, unsigned long long& upd) {
  if (STORAGE == kStorageColor) return;
  float px[4], py[4], pz[4];
  row_points(F, m.v, r, px, py, pz);
  const int naz = F.width, nel = F.height;
  float rr[4], fx[4], fy[4], d00[4], d10[4], d01[4], d11[4];
  bool ok[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    rr[i] = __fsqrt_rn(__fmaf_rn(px[i], px[i], __fmaf_rn(py[i], py[i], __fmul_rn(pz[i], pz[i]))));
    const float rho = __fsqrt_rn(__fmaf_rn(px[i], px[i], __fmul_rn(py[i], py[i])));
    const float th = atan2_dec(py[i], px[i]);
    const float ph = atan2_dec(rho, pz[i]);
    const float u = __fmul_rn(__fsub_rn(th, F.theta_start), F.alpha);
    const float v = __fmul_rn(__fsub_rn(ph, F.phi_start), F.beta);
    ok[i] = rr[i] > 0.0f;
    d00[i] = d10[i] = d01[i] = d11[i] = 0.0f;
    if (m.lidar_nearest) {
      const float ku = floorf(u), jv = floorf(v);
      fx[i] = fy[i] = 0.0f;
      ok[i] = ok[i] && jv >= 0.0f && jv <= (float)(nel - 1) && ku >= -1.0f && ku <= (float)naz;
      if (ok[i]) d00[i] = __ldg(F.depth + (int)jv * naz + wrap_az((int)ku, naz));
    } else {
      const float uu = __fsub_rn(u, 0.5f), vv = __fsub_rn(v, 0.5f);
      const float k0f = floorf(uu), j0f = floorf(vv);
      fx[i] = __fsub_rn(uu, k0f);
      fy[i] = __fsub_rn(vv, j0f);
      ok[i] = ok[i] && j0f >= 0.0f && j0f <= (float)(nel - 2) && k0f >= -1.0f && k0f <= (float)naz;
      if (ok[i]) {
        const int k0 = wrap_az((int)k0f, naz), k1 = k0 + 1 == naz ? 0 : k0 + 1;
        const float* row0 = F.depth + (int)j0f * naz;
        const float* row1 = row0 + naz;
        d00[i] = __ldg(row0 + k0);
        d10[i] = __ldg(row0 + k1);
        d01[i] = __ldg(row1 + k0);
        d11[i] = __ldg(row1 + k1);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!ok[i]) continue;
    float d;
    if (m.lidar_nearest) {
      d = d00[i];
      if (!lidar_valid(F, d)) continue;
    } else {
      if (!(lidar_valid(F, d00[i]) && lidar_valid(F, d10[i]) && lidar_valid(F, d01[i]) &&
            lidar_valid(F, d11[i])))
        continue;
      const float hi = fmaxf(fmaxf(d00[i], d10[i]), fmaxf(d01[i], d11[i]));
      const float lo = fminf(fminf(d00[i], d10[i]), fminf(d01[i], d11[i]));
      if (__fsub_rn(hi, lo) > m.guard) continue;
      const float top = __fmaf_rn(fx[i], __fsub_rn(d10[i], d00[i]), d00[i]);
      const float bot = __fmaf_rn(fx[i], __fsub_rn(d11[i], d01[i]), d01[i]);
      d = __fmaf_rn(fy[i], __fsub_rn(bot, top), top);
    }
    const float dp = __fsub_rn(d, rr[i]);
    if (dp < -m.tau) continue;
    apply<STORAGE, WEIGHTED>(m, D[i], W[i], rr[i], dp);
    ++upd;
  }
}

// Shared memory of the integration workers of a CTA: G groups of
// kIntegrateThreads threads, each group working on its own work-list
// entries.
template <int NF, int NM, int G>
struct IntegSmem {
  uint32_t begin[NM + 1];         // first entry of each map's list in the batch's work
  unsigned long long upd[NM];     // voxel updates per map
  unsigned long long pairs[NM];   // (block, frame) pairs per map
  uint32_t next[G][2];            // per group: the entry in hand and the next one
  FrameProj fp[NF];
};

// Barrier of the kIntegrateThreads threads of worker group g: the CTA
// barrier when the CTA is one group, else hardware barrier 1 + g.
template <int G>
__device__ __forceinline__ void group_sync(int g) {
  if (G == 1) {
    __syncthreads();
  } else if (g == 0) {
    asm volatile("bar.sync 1, %0;" ::"n"(kIntegrateThreads) : "memory");
  } else {
    asm volatile("bar.sync 2, %0;" ::"n"(kIntegrateThreads) : "memory");
  }
}

// Entry metadata: COHERENT loads bypass L1, for a kernel that reads
// metadata that other CTAs of the same launch wrote.
template <bool COHERENT, class T>
__device__ __forceinline__ T meta_load(const T* a) {
  if (COHERENT) return __ldcg(a);
  return *a;
}

// The integration of a batch's work list: every entry is a hash slot met by
// some frames of the batch; its block's 512 voxels are held in registers (4
// per thread) across those frames, in batch order, and written back once.
// Entries are handed out dynamically (blocks differ in their frame counts);
// next[g] is double-buffered so one group barrier per entry suffices.  The
// last CTA to finish resets every map's work list for the next batch.
template <int NF, int NM, int G, bool COHERENT, int STORAGE, bool PINHOLE_ONLY, bool WEIGHTED, bool FAST>
__device__ __forceinline__ void integrate_entries(const BatchParams<NF, NM>& p, IntegSmem<NF, NM, G>& sm) {
  static_assert(G == 1 || G == 2, "one or two worker groups per CTA");
  const int g = G == 1 ? 0 : (int)threadIdx.x / kIntegrateThreads;
  const int t = G == 1 ? (int)threadIdx.x : (int)threadIdx.x % kIntegrateThreads;
  if (threadIdx.x < NM) sm.upd[threadIdx.x] = sm.pairs[threadIdx.x] = 0ull;
  for (int f = threadIdx.x; f < p.n_frames; f += G * kIntegrateThreads)
    if (p.fr[f].kind == kSensorPinhole) stage_frame(p.fr[f], sm.fp[f]);
  if (t == 0) sm.next[g][0] = blockIdx.x * G + g;
  if (threadIdx.x == 0) {
    // the batch's work = the concatenation of every map's list
    uint32_t acc = 0;
    for (int k = 0; k < p.n_maps; ++k) {
      sm.begin[k] = acc;
      acc += min(__ldcg(p.maps[k].ctl), p.maps[k].list_cap);
    }
    sm.begin[p.n_maps] = acc;
  }
  __syncthreads();
  const uint32_t n = sm.begin[p.n_maps];
  // this thread's voxels: x = lx0 .. lx0 + 3 at (ly, lz)
  const int lx0 = (t & 1) * 4, ly = (t >> 1) & 7, lz = t >> 4;

  for (uint32_t it = 0;; ++it) {
    const uint32_t e = sm.next[g][it & 1u];
    if (e >= n) break;
    if (t == 0) sm.next[g][(it + 1) & 1u] = gridDim.x * G + atomicAdd(p.maps[0].ctl + 2, 1u);
    // every thread reads the entry's metadata itself (same addresses across
    // the group), so no warp waits on another before its voxel loads
    int mi = 0;
    while (mi + 1 < p.n_maps && e >= sm.begin[mi + 1]) ++mi;
    const MapDev& m = NM == 1 ? p.maps[0] : p.maps[mi];
    const uint32_t slot = meta_load<COHERENT>(m.list + (e - sm.begin[mi]));
    const int val = meta_load<COHERENT>(m.vals + slot);
    const uint32_t slot_mask = meta_load<COHERENT>(m.mask + slot);
    const unsigned long long slot_key = meta_load<COHERENT>(m.keys + slot);
    const bool fresh = val <= -2;
    const int pool = fresh ? -val - 2 : val;
    unsigned long long my_upd = 0;
    if (val != -1) {
      float D[4], W[4], G4[4], B[4];
      if (fresh) {
#pragma unroll
        for (int i = 0; i < 4; ++i) { D[i] = 0.0f; W[i] = 0.0f; G4[i] = 0.0f; B[i] = 0.0f; }
      } else {
        Voxels4<STORAGE>::load(m, pool, t, D, W, G4, B);
      }
      const int bx = key_coord(slot_key, 0), by = key_coord(slot_key, 1), bz = key_coord(slot_key, 2);
      const VoxelRow vr{bx, by, bz, lx0, ly, lz};
      uint32_t bits = slot_mask;
      while (bits) {
        // bit k of the mask is frame k of the batch; frames apply in batch
        // order.  Two consecutive pinhole frames issue all their depth loads
        // before the first update (longer runs measured slower: the unrolled
        // code outgrows the instruction cache).
        int fq[4];
        int nq = 0;
        bool go = true;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          fq[q] = -1;
          if (go && bits) {
            const int f = __ffs(bits) - 1;
            if (PINHOLE_ONLY || p.fr[f].kind == kSensorPinhole) {
              fq[q] = f;
              ++nq;
              bits &= bits - 1u;
            } else {
              go = false;
            }
          }
        }
        fq[2] = fq[3] = -1;
        if (nq == 2)
          fuse_pinhole<2, STORAGE, WEIGHTED, FAST, PINHOLE_ONLY>(p, sm.fp, fq, m, vr, D, W, G4, B, my_upd);
        else if (nq == 1)
          fuse_pinhole<1, STORAGE, WEIGHTED, FAST, PINHOLE_ONLY>(p, sm.fp, fq, m, vr, D, W, G4, B, my_upd);
        else if (!PINHOLE_ONLY) {
          const int f = __ffs(bits) - 1;  // a LiDAR frame
          bits &= bits - 1u;
          fuse_lidar<STORAGE, WEIGHTED>(p.fr[f], m, vr, D, W, my_upd);
        }
      }
      Voxels4<STORAGE>::store(m, pool, t, D, W, G4, B);
    }
    // per-map update count: warp sums into a shared per-map counter
    for (int o = 16; o > 0; o >>= 1) my_upd += __shfl_down_sync(0xffffffffu, my_upd, o);
    if ((t & 31) == 0 && my_upd) atomicAdd(&sm.upd[mi], my_upd);
    group_sync<G>(g);  // every warp of the group has read this entry's metadata
    if (t == 0) {
      atomicAdd(&sm.pairs[mi], (unsigned long long)__popc(slot_mask));
      m.mask[slot] = 0u;
      if (fresh) m.vals[slot] = pool;
      if (m.dirty && val != -1) m.dirty[pool] = kDirtyEsdf | kDirtyMesh;
    }
  }
  if (p.overlap) allow_next_grid();
  __syncthreads();
  if (threadIdx.x < p.n_maps && sm.upd[threadIdx.x])
    atomicAdd(p.maps[threadIdx.x].counters + kCntUpdates, sm.upd[threadIdx.x]);
  if (threadIdx.x < p.n_maps && sm.pairs[threadIdx.x])
    atomicAdd(p.maps[threadIdx.x].counters + kCntPairs, sm.pairs[threadIdx.x]);
  // the last CTA to finish resets every map's work list for the next batch
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(p.maps[0].ctl + 1, 1u);
    if (done == gridDim.x - 1) {
      for (int k = 0; k < p.n_maps; ++k) {
        atomicAdd(p.maps[k].counters + kCntVisits, (unsigned long long)(sm.begin[k + 1] - sm.begin[k]));
        atomicAdd(p.maps[k].counters + kCntLaunches, 1ull);
        p.maps[k].ctl[0] = 0u;
      }
      p.maps[0].ctl[1] = 0u;
      p.maps[0].ctl[2] = 0u;
      p.maps[0].ctl[3] = 0u;  // the fused kernel's barrier count
    }
  }
}

template <int NF, int NM, int STORAGE, bool PINHOLE_ONLY, bool WEIGHTED, bool FAST = false>
__global__ void __launch_bounds__(kIntegrateThreads)
    integrate_kernel(const __grid_constant__ BatchParams<NF, NM> p) {
  __shared__ IntegSmem<NF, NM, 1> sm;
  if (p.overlap) wait_prev_grid();
  integrate_entries<NF, NM, 1, false, STORAGE, PINHOLE_ONLY, WEIGHTED, FAST>(p, sm);
}

// ------------------------------------------- one launch per batch (fused)

// Bounded waits give up after this many nanoseconds of the global timer.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int load_acquire(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident): thread 0 of
// every CTA arrives on *count, then waits until `expected` CTAs have arrived,
// for at most kWaitLimitNs.  A wait that runs out sets kStTimeout in *status
// (the map's sticky status) and makes the CTA return false.
__device__ __noinline__ bool grid_wait(unsigned int* count, unsigned int expected, unsigned long long* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while (load_acquire(count) < expected) {
      if (global_ns() - t0 > kWaitLimitNs) {
        atomicOr(status, (unsigned long long)kStTimeout);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kFusedThreads = kAllocThreads;  // two integration worker groups
static_assert(kFusedThreads == 2 * kIntegrateThreads, "fused CTA = two integration groups");

template <int NF, int NM, int TH>
union FusedSmem {
  AllocSmem<TH> a;
  IntegSmem<NF, NM, 2> i;
};

// Allocation and integration of one batch in one persistent, cooperative
// launch: the CTAs walk every allocation tile of the batch (grid-stride),
// meet at a bounded grid-wide wait (the integration reads the work list,
// slot masks and pool indices that every tile wrote), then integrate the
// work list as two groups of kIntegrateThreads per CTA.  Single-map
// batches, TSDF storage, constant weighting, no walk statistics.
// Four resident CTAs per SM (64 registers): the rig's fused step measured
// 16.1 ms per 1,000 frames against 18.2 ms with three.
template <int NF, int NM, int TH, int STORAGE, bool PINHOLE_ONLY, bool FAST>
__global__ void __launch_bounds__(kFusedThreads, 4)
    fused_kernel(const __grid_constant__ BatchParams<NF, NM> p) {
  __shared__ FusedSmem<NF, NM, TH> sm;
  for (int cta = blockIdx.x; cta < p.alloc_ctas; cta += gridDim.x)
    alloc_tile<NF, NM, TH, PINHOLE_ONLY, false, FAST, true>(p, cta, sm.a);
  if (!grid_wait(p.maps[0].ctl + 3, gridDim.x + (unsigned)p.wait_extra, p.maps[0].counters + kCntStatus))
    return;  // timed out: integration skipped, the map reports TSDF_ERR_TIMEOUT
  integrate_entries<NF, NM, 2, true, STORAGE, PINHOLE_ONLY, false, FAST>(p, sm.i);
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
        if (STORAGE == kStorageOcc) {
          outD = reinterpret_cast<const float*>(m.pool)[(size_t)val * 512 + l];
        } else if (STORAGE == kStorageF32) {
          const float2 v = reinterpret_cast<const float2*>(m.pool)[(size_t)val * 512 + l];
          outD = v.x;
          outW = v.y;
        } else if (STORAGE == kStorageX16) {
          const uint32_t w = reinterpret_cast<const uint32_t*>(m.pool)[(size_t)val * 512 + l];
          outD = x16_dist(w, m.x16_unit);
          outW = x16_weight(w);
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

// Colour of the voxel holding each point: r, g, b and the colour weight;
// zeros where no block or no colour update exists.
__global__ void query_color_kernel(const MapDev m, const float* __restrict__ pts, int64_t n,
                                   float* __restrict__ rgb, float* __restrict__ weight) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
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
        out = reinterpret_cast<const float4*>(m.pool)[(size_t)val * 512 + l];
      }
    }
  }
  rgb[3 * i] = out.x;
  rgb[3 * i + 1] = out.y;
  rgb[3 * i + 2] = out.z;
  weight[i] = out.w;
}

// Occupancy decay over every allocated block: log-odds above 0 drop by
// d_occ, below 0 rise by d_free, neither crossing 0.  The pool's first
// min(blocks, max_blocks) blocks are exactly the allocated ones; a thread
// handles four voxels (one 16-byte word) per step of a grid-stride loop.
__global__ void decay_kernel(const MapDev m, float d_occ, float d_free) {
  const unsigned long long nb =
      min((unsigned long long)m.max_blocks, __ldcg(m.counters + kCntBlocks));
  const size_t n4 = (size_t)nb * 128;
  float4* pool = reinterpret_cast<float4*>(m.pool);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x) {
    float4 l = pool[i];
    const float4 before = l;
    float* c = &l.x;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      c[k] = c[k] > 0.0f ? fmaxf(c[k] - d_occ, 0.0f) : (c[k] < 0.0f ? fminf(c[k] + d_free, 0.0f) : c[k]);
    pool[i] = l;
    // a changed block is due for the next ESDF update and mesh extraction
    // (all writers of a block's flag byte set the same bits)
    if (m.dirty && (l.x != before.x || l.y != before.y || l.z != before.z || l.w != before.w))
      m.dirty[i / 128] |= kDirtyEsdf | kDirtyMesh;
  }
}

__global__ void reset_kernel(const MapDev m, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    m.keys[i] = kEmptyKey;
    m.vals[i] = -1;
    m.mask[i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < kNumCounters) m.counters[threadIdx.x] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x < 4) m.ctl[threadIdx.x] = 0u;
}

}  // namespace

// True when every frame of the batch is a pinhole camera: the kernels are
// then launched without their LiDAR code (smaller, fewer branches).
template <int NF, int NM>
bool pinhole_only(const BatchParams<NF, NM>& p) {
  for (int f = 0; f < p.n_frames; ++f)
    if (p.fr[f].kind != kSensorPinhole) return false;
  return true;
}

// Every frame's band segments meet fewer than kMaxCells blocks (host check).
template <int NF, int NM>
bool short_walks(const BatchParams<NF, NM>& p) {
  for (int f = 0; f < p.n_frames; ++f)
    if (!p.fr[f].short_walks) return false;
  return true;
}

// Launch kernel k; with p.overlap as a programmatic dependent launch.
template <class P>
cudaError_t launch_k(void (*k)(P), dim3 g, dim3 b, cudaStream_t s, const P& p) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = p.overlap ? at : nullptr;
  cfg.numAttrs = p.overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, p);
}

template <int NF, int NM>
cudaError_t launch_band_alloc(const BatchParams<NF, NM>& p, int n_ctas, int tile_h, cudaStream_t s) {
  if (n_ctas <= 0) return cudaSuccess;
  const bool ph = pinhole_only(p);
  bool st = false;
  for (int k = 0; k < p.n_maps; ++k) st = st || p.maps[k].walk_stats != 0;
  const dim3 g(n_ctas), b(kAllocThreads);
  if (st) {  // diagnostics: one generic variant per tile height
    if (tile_h == kTileHBig)
      return launch_k(band_alloc_kernel<NF, NM, kTileHBig, false, true, false, true>, g, b, s, p);
    else
      return launch_k(band_alloc_kernel<NF, NM, kTileHSmall, false, true, false, true>, g, b, s, p);
  }
  if (!short_walks(p)) {  // segments that may reach the cap: one generic variant per tile height
    if (tile_h == kTileHBig)
      return launch_k(band_alloc_kernel<NF, NM, kTileHBig, false, false, false, true>, g, b, s, p);
    else
      return launch_k(band_alloc_kernel<NF, NM, kTileHSmall, false, false, false, true>, g, b, s, p);
  }
  const bool fast = p.fast_rcp != 0;
  if (tile_h == kTileHBig) {
    if (ph) return fast ? launch_k(band_alloc_kernel<NF, NM, kTileHBig, true, false, true, false>, g, b, s, p)
                        : launch_k(band_alloc_kernel<NF, NM, kTileHBig, true, false, false, false>, g, b, s, p);
    return fast ? launch_k(band_alloc_kernel<NF, NM, kTileHBig, false, false, true, false>, g, b, s, p)
                : launch_k(band_alloc_kernel<NF, NM, kTileHBig, false, false, false, false>, g, b, s, p);
  }
  if (ph) return fast ? launch_k(band_alloc_kernel<NF, NM, kTileHSmall, true, false, true, false>, g, b, s, p)
                      : launch_k(band_alloc_kernel<NF, NM, kTileHSmall, true, false, false, false>, g, b, s, p);
  return fast ? launch_k(band_alloc_kernel<NF, NM, kTileHSmall, false, false, true, false>, g, b, s, p)
              : launch_k(band_alloc_kernel<NF, NM, kTileHSmall, false, false, false, false>, g, b, s, p);
}

template <int NF, int NM>
cudaError_t launch_integrate(const BatchParams<NF, NM>& p, int n_ctas, cudaStream_t s) {
  // all maps of a batch share one storage type (checked by the host API)
  // colour maps take pinhole frames only (checked by the host API)
  const bool ph = pinhole_only(p);
  const int st = p.maps[0].storage;
  // the weighted update with weighting 0 is the constant-weight update, so
  // one weighted map selects the weighted kernel for the whole batch
  bool wt = false;
  for (int k = 0; k < p.n_maps; ++k) wt = wt || p.maps[k].weighting != 0;
  const dim3 g(n_ctas), b(kIntegrateThreads);
  // FAST: pinhole reciprocals by rcp_dec<true> (the host checked their range)
  const bool fast = p.fast_rcp != 0;
#define GBT_INTEG(ST, PH) \
  (fast ? launch_k(integrate_kernel<NF, NM, ST, PH, false, true>, g, b, s, p) \
        : launch_k(integrate_kernel<NF, NM, ST, PH, false, false>, g, b, s, p))
  if (st == kStorageColor) return GBT_INTEG(kStorageColor, true);
  if (st == kStorageOcc) return ph ? GBT_INTEG(kStorageOcc, true) : GBT_INTEG(kStorageOcc, false);
  if (st == kStorageX16) {
    if (wt) return launch_k(integrate_kernel<NF, NM, kStorageX16, false, true>, g, b, s, p);
    return ph ? GBT_INTEG(kStorageX16, true) : GBT_INTEG(kStorageX16, false);
  }
  if (st == kStorageF16) {
    if (wt) return launch_k(integrate_kernel<NF, NM, kStorageF16, false, true>, g, b, s, p);
    return ph ? GBT_INTEG(kStorageF16, true) : GBT_INTEG(kStorageF16, false);
  }
  if (wt) return launch_k(integrate_kernel<NF, NM, kStorageF32, false, true>, g, b, s, p);
  return ph ? GBT_INTEG(kStorageF32, true) : GBT_INTEG(kStorageF32, false);
#undef GBT_INTEG
}

// The fused kernel of a tile height for a storage and sensor mix, launched
// cooperatively with as many CTAs as can be resident at once.
template <int NF, int NM, int TH>
cudaError_t launch_fused_th(const BatchParams<NF, NM>& p, int st, bool ph, cudaStream_t s) {
  void (*k)(BatchParams<NF, NM>) = nullptr;
  const bool fast = p.fast_rcp != 0;
#define GBT_FUSED(ST) \
  (ph ? (fast ? fused_kernel<NF, NM, TH, ST, true, true> : fused_kernel<NF, NM, TH, ST, true, false>) \
      : (fast ? fused_kernel<NF, NM, TH, ST, false, true> : fused_kernel<NF, NM, TH, ST, false, false>))
  int si = 0;
  if (st == kStorageF32) {
    k = GBT_FUSED(kStorageF32);
    si = 0;
  } else if (st == kStorageF16) {
    k = GBT_FUSED(kStorageF16);
    si = 1;
  } else {
    k = GBT_FUSED(kStorageX16);
    si = 2;
  }
#undef GBT_FUSED
  static int per_sm[3][2][2] = {};  // resident CTAs per SM of each variant (all devices are alike here)
  int& n = per_sm[si][ph ? 1 : 0][fast ? 1 : 0];
  if (n == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFusedThreads, 0) != cudaSuccess) {
    n = 0;
    return cudaGetLastError();
  }
  if (n <= 0) return cudaErrorNotSupported;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaGetLastError();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n * sms);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid-wide wait can complete
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, p);
}

template <int NF, int NM>
cudaError_t launch_fused(const BatchParams<NF, NM>& p, int tile_h, cudaStream_t s) {
  const MapDev& m0 = p.maps[0];
  if (NM != 1 || p.n_maps != 1 || p.overlap || m0.walk_stats || m0.weighting != 0) return cudaErrorNotSupported;
  const int st = m0.storage;
  if (st != kStorageF32 && st != kStorageF16 && st != kStorageX16) return cudaErrorNotSupported;
  if (p.alloc_ctas <= 0) return cudaErrorNotSupported;
  const bool ph = pinhole_only(p);
  return tile_h == kTileHBig ? launch_fused_th<NF, NM, kTileHBig>(p, st, ph, s)
                             : launch_fused_th<NF, NM, kTileHSmall>(p, st, ph, s);
}

template cudaError_t launch_fused<kMaxFrames, 1>(const BatchParams<kMaxFrames, 1>&, int, cudaStream_t);
template cudaError_t launch_band_alloc<1, 1>(const BatchParams<1, 1>&, int, int, cudaStream_t);
template cudaError_t launch_band_alloc<kMaxFrames, kMaxMaps>(const BatchParams<kMaxFrames, kMaxMaps>&,
                                                             int, int, cudaStream_t);
template cudaError_t launch_integrate<1, 1>(const BatchParams<1, 1>&, int, cudaStream_t);
template cudaError_t launch_band_alloc<kMaxFrames, 1>(const BatchParams<kMaxFrames, 1>&, int, int,
                                                     cudaStream_t);
template cudaError_t launch_integrate<kMaxFrames, 1>(const BatchParams<kMaxFrames, 1>&, int, cudaStream_t);
template cudaError_t launch_integrate<kMaxFrames, kMaxMaps>(const BatchParams<kMaxFrames, kMaxMaps>&,
                                                            int, cudaStream_t);

cudaError_t launch_query(const MapDev& m, const float* pts, int64_t n, float* dist, float* weight,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (m.storage == kStorageOcc)
    query_kernel<kStorageOcc><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  else if (m.storage == kStorageF16)
    query_kernel<kStorageF16><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  else if (m.storage == kStorageX16)
    query_kernel<kStorageX16><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  else
    query_kernel<kStorageF32><<<blocks, threads, 0, s>>>(m, pts, n, dist, weight);
  return cudaGetLastError();
}

cudaError_t launch_query_color(const MapDev& m, const float* pts, int64_t n, float* rgb, float* weight,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  query_color_kernel<<<blocks, threads, 0, s>>>(m, pts, n, rgb, weight);
  return cudaGetLastError();
}

cudaError_t launch_decay(const MapDev& m, float d_occ, float d_free, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  decay_kernel<<<sms * 8, 256, 0, s>>>(m, d_occ, d_free);
  return cudaGetLastError();
}

cudaError_t launch_reset(const MapDev& m, uint32_t cap, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  reset_kernel<<<sms * 4, 256, 0, s>>>(m, cap);
  return cudaGetLastError();
}

namespace {
template <class K>
int occupancy(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kIntegrateThreads, 0) != cudaSuccess)
    n = 0;
  return n;
}
}  // namespace

// Resident integration CTAs per SM: the smallest over the kernel variants a
// map of this storage can launch (the grid is persistent).
int integrate_ctas_per_sm(int storage) {
  constexpr int F = kMaxFrames, M = kMaxMaps;
  int n;
  if (storage == kStorageColor)
    n = occupancy(integrate_kernel<F, M, kStorageColor, true, false>);
  else if (storage == kStorageOcc)
    n = std::min(occupancy(integrate_kernel<F, M, kStorageOcc, true, false>),
                 occupancy(integrate_kernel<F, M, kStorageOcc, false, false>));
  else if (storage == kStorageX16)
    n = std::min({occupancy(integrate_kernel<F, M, kStorageX16, true, false>),
                  occupancy(integrate_kernel<F, M, kStorageX16, false, false>),
                  occupancy(integrate_kernel<F, M, kStorageX16, false, true>)});
  else if (storage == kStorageF16)
    n = std::min({occupancy(integrate_kernel<F, M, kStorageF16, true, false>),
                  occupancy(integrate_kernel<F, M, kStorageF16, false, false>),
                  occupancy(integrate_kernel<F, M, kStorageF16, false, true>)});
  else
    n = std::min({occupancy(integrate_kernel<F, M, kStorageF32, true, false>),
                  occupancy(integrate_kernel<F, M, kStorageF32, false, false>),
                  occupancy(integrate_kernel<F, M, kStorageF32, false, true>)});
  return n > 0 ? n : 4;
}

}  // namespace gbt
