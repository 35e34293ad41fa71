// ESDF layer kernels (Sec. IV-C) and the map import kernel, sm_103a.
//
// The ESDF layer is indexed like the TSDF pool: block p of the pool has the
// 512 voxel state words st[p * 512 ..].  One update runs the stages of
// Sec. IV-C in order:
//
//   esdf_mark_kernel   mark sites in the blocks changed since the last
//                      update (the dirty flags the integration sets) and
//                      reset voxels whose site status, observation or side
//                      changed; collect the update set and the blocks where
//                      a site disappeared (occupancy layers: the face-
//                      neighbour table first, then esdf_occ_spread_kernel
//                      and esdf_occ_mark_kernel, whose site test reads
//                      across block faces)
//   esdf_clear_kernel  in every block near one of the latter, drop parents
//                      that are no longer sites
//   esdf_nbr_kernel    the face-neighbour table of every block
//   then, until the update set is empty (the host enqueues four iterations
//   at a time and reads the set size after them):
//   esdf_sweep_kernel  six in-block sweeps (+x, -x, +y, -y, +z, -z) of every
//                      block of the update set, in shared memory; the block
//                      and its existing face neighbours join the tlist
//   esdf_pull_kernel   every tlist block tries, on its faces, the parents of
//                      the adjacent voxels across the faces, reading the
//                      states as they were before this step; results go to
//                      st2
//   esdf_apply_kernel  copy back the blocks that changed; they form the next
//                      update set
//
// All distance arithmetic is on integer offsets (squared lengths), so the
// result is exact and does not depend on the order in which CTAs run.
#include <cmath>

#include "tsdf_internal.cuh"

namespace gbt {
namespace {

constexpr int kEsdfThreads = 128;  // threads per CTA (4 voxels each, or 4 warps of 16)

__device__ __forceinline__ int off_comp(uint32_t s, int axis) {
  const int raw = (int)((s >> (9 * axis)) & 511u);
  return raw >= 256 ? raw - 512 : raw;
}

__device__ __forceinline__ int dist2(uint32_t s) {
  const int x = off_comp(s, 0), y = off_comp(s, 1), z = off_comp(s, 2);
  return x * x + y * y + z * z;
}

// Voxel p tries the parent of its neighbour q, which lies at p + (dx, dy, dz):
// taken if p is observed and not a site, q has a parent, and the offset from
// p to that parent is within max_dist and strictly shorter than p's own.
__device__ __forceinline__ bool relax(uint32_t& p, uint32_t q, int dx, int dy, int dz, int max2) {
  if (!(p & kEsdfObs) || (p & kEsdfSite) || !(q & kEsdfPar)) return false;
  const int cx = off_comp(q, 0) + dx, cy = off_comp(q, 1) + dy, cz = off_comp(q, 2) + dz;
  const int c2 = cx * cx + cy * cy + cz * cz;
  if (c2 > max2) return false;
  if ((p & kEsdfPar) && c2 >= dist2(p)) return false;
  p = (p & ~kEsdfOffMask) | kEsdfPar | ((uint32_t)cx & 511u) | (((uint32_t)cy & 511u) << 9) |
      (((uint32_t)cz & 511u) << 18);
  return true;
}

__device__ __forceinline__ uint32_t n_blocks(const MapDev& m) {
  return (uint32_t)min((unsigned long long)m.max_blocks, __ldcg(m.counters + kCntBlocks));
}

// Pool index of the block with coordinates (x, y, z), or -1.
__device__ __forceinline__ int pool_of(const MapDev& m, int x, int y, int z) {
  const int slot = hash_find(m, pack_key(x, y, z));
  if (slot < 0) return -1;
  const int val = m.vals[slot];
  return val >= 0 ? val : -1;
}

// Append block p to an update set (list, size) unless this generation has it already.
__device__ __forceinline__ void add_update(const EsdfDev& e, uint32_t* list, uint32_t* size,
                                           uint32_t p, uint32_t gen) {
  if (atomicExch(e.stamp_s + p, gen) != gen) list[atomicAdd(size, 1u)] = p;
}

// Hashed bitmaps of the blocks where a site disappeared (lost-site blocks)
// and of their coarse cells (cubes of G = R + 1 blocks, R the reach of a
// parent in blocks), written by the mark stage for the clear stage.
constexpr int kNearBits = kEsdfBitWords * 32;
constexpr int kCoordBias = 1 << 21;  // block coordinates + bias >= 0

__device__ __forceinline__ uint32_t near_bit(int cx, int cy, int cz) {
  return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & (kNearBits - 1);
}

__device__ __forceinline__ int parent_reach(const EsdfDev& e) { return (e.max_dist + 7) / 8 + 1; }

__device__ __forceinline__ bool bit_set(const uint32_t* bits, uint32_t b) {
  return (__ldg(bits + (b >> 5)) >> (b & 31)) & 1u;
}

// ------------------------------------------------------------- mark sites

// New state of a voxel from its observation, site and side: a new site
// takes itself as parent; a voxel that stops being a site, becomes
// observed or changes sides loses its parent (lost: a site disappeared).
__device__ __forceinline__ uint32_t marked_state(uint32_t old, bool obs, bool site, bool inside, bool& lost) {
  if (site) return kEsdfObs | kEsdfSite | kEsdfPar | (inside ? kEsdfInside : 0u);
  if (old & kEsdfSite) {
    lost = true;
    return obs ? (kEsdfObs | (inside ? kEsdfInside : 0u)) : 0u;
  }
  if (!obs) return 0u;
  if (!(old & kEsdfObs) || ((old & kEsdfInside) != 0u) != inside) return kEsdfObs | (inside ? kEsdfInside : 0u);
  return old;
}

// Update-set and lost-site bookkeeping of a marked block (lane 0).
__device__ __forceinline__ void mark_done(const MapDev& m, const EsdfDev& e, uint32_t p, uint32_t gen, bool any,
                                          bool lost) {
  if (any) add_update(e, e.list[0], e.cnt, p, gen);
  if (lost) {
    e.clist[atomicAdd(e.cnt + 2, 1u)] = p;
    const unsigned long long key = m.block_keys[p];
    const int G = parent_reach(e) + 1;
    const int cx = key_coord(key, 0) + kCoordBias, cy = key_coord(key, 1) + kCoordBias,
              cz = key_coord(key, 2) + kCoordBias;
    const uint32_t l = near_bit(cx, cy, cz), c = near_bit(cx / G, cy / G, cz / G);
    atomicOr(e.bits + (l >> 5), 1u << (l & 31));
    atomicOr(e.bits + kEsdfBitWords + (c >> 5), 1u << (c & 31));
  }
}

// One warp per pool block, 16 voxels per lane (voxels 128 j + 4 lane + i),
// read and written as 16-byte vectors.
__global__ void __launch_bounds__(kEsdfThreads)
    esdf_mark_kernel(const MapDev m, const EsdfDev e, uint32_t gen) {
  constexpr int kWarps = kEsdfThreads / 32;
  const uint32_t nb = n_blocks(m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t p = blockIdx.x * kWarps + warp; p < nb; p += gridDim.x * kWarps) {
    if (!(m.dirty[p] & kDirtyEsdf)) continue;  // same value for every lane
    uint4* stb = reinterpret_cast<uint4*>(e.st + (size_t)p * 512) + lane;
    bool any = false, lost = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float D[4], W[4];
      if (m.storage == kStorageF16) {
        const uint4 raw = reinterpret_cast<const uint4*>(m.pool)[(size_t)p * 128 + 32 * j + lane];
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __half2 h = *reinterpret_cast<const __half2*>(&w4[i]);
          D[i] = __low2float(h) * m.tau;
          W[i] = __high2float(h);
        }
      } else if (m.storage == kStorageX16) {
        const uint4 raw = reinterpret_cast<const uint4*>(m.pool)[(size_t)p * 128 + 32 * j + lane];
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          D[i] = x16_dist(w4[i], m.x16_unit);
          W[i] = x16_weight(w4[i]);
        }
      } else {
        const float4* src = reinterpret_cast<const float4*>(m.pool) + (size_t)p * 256 + 64 * j + 2 * lane;
        const float4 a = src[0], b = src[1];
        D[0] = a.x; W[0] = a.y; D[1] = a.z; W[1] = a.w;
        D[2] = b.x; W[2] = b.y; D[3] = b.z; W[3] = b.w;
      }
      const uint4 o4 = stb[32 * j];
      const uint32_t old[4] = {o4.x, o4.y, o4.z, o4.w};
      uint32_t nw[4];
      bool changed = false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool obs = W[i] >= e.min_weight;
        nw[i] = marked_state(old[i], obs, obs && fabsf(D[i]) <= e.site_eps, obs && D[i] < 0.0f, lost);
        changed = changed || nw[i] != old[i];
      }
      if (changed) stb[32 * j] = make_uint4(nw[0], nw[1], nw[2], nw[3]);
      any = any || changed;
    }
    any = __any_sync(0xffffffffu, any);  // also: every lane has read dirty[p]
    lost = __any_sync(0xffffffffu, lost);
    if (lane == 0) {
      m.dirty[p] &= (uint8_t)~kDirtyEsdf;
      mark_done(m, e, p, gen, any, lost);
    }
  }
}

// Occupancy layers (Sec. IV-C: an occupancy voxel is a site if it is
// adjacent to free voxels).  Log-odds l > 0 is occupied, l < 0 free, l = 0
// unknown (never observed, or decayed back to probability 1/2); observed =
// occupied or free, inside = occupied, site = occupied with a free voxel
// among its six face neighbours.  Neighbours across a block face are read
// through the face-neighbour table (a missing block is unknown), so a block
// is marked when it changed or one of its face neighbours did.

// Flag the face neighbours of every changed block.  Every writer of a byte
// here sets the same bit, so the unsynchronised read-modify-writes agree.
__global__ void esdf_occ_spread_kernel(const MapDev m, const EsdfDev e) {
  const uint32_t nb = n_blocks(m);
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nb; p += gridDim.x * blockDim.x) {
    if (!(m.dirty[p] & kDirtyEsdf)) continue;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int q = e.nbr[6 * p + f];
      if (q >= 0) m.dirty[q] |= kDirtyNbr;
    }
  }
}

// One warp per flagged block: the block's log-odds staged in shared memory,
// 16 voxels per lane (voxels 128 j + 4 lane + i) as in esdf_mark_kernel.
__global__ void __launch_bounds__(kEsdfThreads)
    esdf_occ_mark_kernel(const MapDev m, const EsdfDev e, uint32_t gen) {
  constexpr int kWarps = kEsdfThreads / 32;
  __shared__ __align__(16) float s_l[kWarps][512];
  const uint32_t nb = n_blocks(m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* pool = reinterpret_cast<const float*>(m.pool);
  float* sl = s_l[warp];
  for (uint32_t p = blockIdx.x * kWarps + warp; p < nb; p += gridDim.x * kWarps) {
    if (!(m.dirty[p] & (kDirtyEsdf | kDirtyNbr))) continue;  // same value for every lane
#pragma unroll
    for (int j = 0; j < 4; ++j)
      reinterpret_cast<float4*>(sl)[32 * j + lane] = reinterpret_cast<const float4*>(pool)[(size_t)p * 128 + 32 * j + lane];
    const int mine = lane < 6 ? e.nbr[6 * p + lane] : -1;
    int q[6];  // face neighbours -x, +x, -y, +y, -z, +z
#pragma unroll
    for (int f = 0; f < 6; ++f) q[f] = __shfl_sync(0xffffffffu, mine, f);
    __syncwarp();
    uint4* stb = reinterpret_cast<uint4*>(e.st + (size_t)p * 512) + lane;
    bool any = false, lost = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 o4 = stb[32 * j];
      const uint32_t old[4] = {o4.x, o4.y, o4.z, o4.w};
      uint32_t nw[4];
      bool changed = false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = 128 * j + 4 * lane + i;
        const int c[3] = {l & 7, (l >> 3) & 7, l >> 6};
        const float v = sl[l];
        bool free_nbr = false;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int axis = f >> 1, d = (f & 1) ? 1 : -1, stride = axis == 0 ? 1 : (axis == 1 ? 8 : 64);
          const int cn = c[axis] + d;
          float w;
          if (cn >= 0 && cn < 8) w = sl[l + d * stride];
          else w = q[f] >= 0 ? pool[(size_t)q[f] * 512 + l - d * 7 * stride] : 0.0f;
          free_nbr = free_nbr || w < 0.0f;
        }
        const bool obs = v != 0.0f, inside = v > 0.0f;
        nw[i] = marked_state(old[i], obs, inside && free_nbr, inside, lost);
        changed = changed || nw[i] != old[i];
      }
      if (changed) stb[32 * j] = make_uint4(nw[0], nw[1], nw[2], nw[3]);
      any = any || changed;
    }
    any = __any_sync(0xffffffffu, any);  // also: every lane is done with sl and dirty[p]
    lost = __any_sync(0xffffffffu, lost);
    if (lane == 0) {
      m.dirty[p] &= (uint8_t)~(kDirtyEsdf | kDirtyNbr);
      mark_done(m, e, p, gen, any, lost);
    }
  }
}

// ---------------------------------------------------------- clear invalid

// Between updates every parent is a site, and sites disappear only in the
// lost-site blocks.  A block is checked if a marked coarse cell is among the
// 27 around its own (every block within R of a lost-site block is), and in
// it a parent is looked up only if its block's bit is set.  Bitmap
// collisions only add checks of parents that are still sites, which change
// nothing.
// One warp per pool block, 16 voxels per lane (voxels 128 j + 4 lane + i).
__global__ void __launch_bounds__(kEsdfThreads)
    esdf_clear_kernel(const MapDev m, const EsdfDev e, uint32_t gen) {
  constexpr int kWarps = kEsdfThreads / 32;
  const uint32_t nc = __ldcg(e.cnt + 2);
  if (nc == 0) return;
  const uint32_t nb = n_blocks(m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = parent_reach(e) + 1;  // coarse cell edge in blocks
  const uint32_t* lost_bits = e.bits;
  const uint32_t* cell_bits = e.bits + kEsdfBitWords;
  unsigned long long my_cleared = 0;
  for (uint32_t p = blockIdx.x * kWarps + warp; p < nb; p += gridDim.x * kWarps) {
    const unsigned long long key = m.block_keys[p];
    const int bx = key_coord(key, 0), by = key_coord(key, 1), bz = key_coord(key, 2);
    bool near = false;
    if (lane < 27) {
      const uint32_t b = near_bit((bx + kCoordBias) / G + lane % 3 - 1, (by + kCoordBias) / G + (lane / 3) % 3 - 1,
                                  (bz + kCoordBias) / G + lane / 9 - 1);
      near = bit_set(cell_bits, b);
    }
    if (!__any_sync(0xffffffffu, near)) continue;
    uint4* blk = reinterpret_cast<uint4*>(e.st + (size_t)p * 512) + lane;
    uint32_t v[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 a = blk[32 * j];
      v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
    }
    bool any = false;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = 128 * j + 4 * lane + i;
        const uint32_t s = v[4 * j + i];
        if (!(s & kEsdfPar) || (s & kEsdfSite)) continue;
        // parent voxel in global voxel coordinates, then its block and index
        const int gx = 8 * bx + (l & 7) + off_comp(s, 0);
        const int gy = 8 * by + ((l >> 3) & 7) + off_comp(s, 1);
        const int gz = 8 * bz + (l >> 6) + off_comp(s, 2);
        const int pbx = gx >> 3, pby = gy >> 3, pbz = gz >> 3;
        const uint32_t lb = near_bit(pbx + kCoordBias, pby + kCoordBias, pbz + kCoordBias);
        if (!bit_set(lost_bits, lb)) continue;  // its block lost no site
        const int pp = (pbx == bx && pby == by && pbz == bz) ? (int)p : pool_of(m, pbx, pby, pbz);
        const bool ok = pp >= 0 &&
                        (e.st[(size_t)pp * 512 + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7)] & kEsdfSite);
        if (!ok) {
          e.st[(size_t)p * 512 + l] = s & ~(kEsdfPar | kEsdfOffMask);
          ++my_cleared;
          any = true;
        }
      }
    if (__any_sync(0xffffffffu, any) && lane == 0) add_update(e, e.list[0], e.cnt, p, gen);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_cleared += __shfl_down_sync(0xffffffffu, my_cleared, o);
  if (lane == 0 && my_cleared) atomicAdd(e.stats, my_cleared);
}

// ------------------------------------------------------------ lower ESDF

// Face-neighbour table of every pool block (the block set does not change
// during an update).
__global__ void esdf_nbr_kernel(const MapDev m, const EsdfDev e) {
  const uint32_t nb = n_blocks(m);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < 6u * nb; k += gridDim.x * blockDim.x) {
    const uint32_t p = k / 6u;
    const int f = (int)(k - 6u * p);
    const unsigned long long key = m.block_keys[p];
    const int d = (f & 1) ? 1 : -1;
    e.nbr[k] = pool_of(m, key_coord(key, 0) + (f >> 1 == 0 ? d : 0), key_coord(key, 1) + (f >> 1 == 1 ? d : 0),
                       key_coord(key, 2) + (f >> 1 == 2 ? d : 0));
  }
}

// In-block sweeps keep the block in shared memory padded to 9 words per
// x-row and 72 per z-slice, so that the lines of every axis are read with at
// most two-way bank conflicts, with each voxel's squared parent distance
// beside its state.
constexpr int kSweepRow = 9, kSweepSlice = 72;
constexpr int kSweepWords = 7 + 7 * kSweepRow + 7 * kSweepSlice + 1;

__device__ __forceinline__ int sweep_idx(int l) {
  return (l & 7) + kSweepRow * ((l >> 3) & 7) + kSweepSlice * (l >> 6);
}

// relax() for a neighbour q on axis AXIS at p + D (D = +-1), with the squared
// lengths carried along: q's candidate offset differs from q's own in the
// AXIS component only, so its squared length is q2 + 2 D o + 1.  Same
// decisions and the same resulting state as relax().
template <int AXIS, int D>
__device__ __forceinline__ void relax_line(uint32_t& ps, int& p2, uint32_t qs, int q2, int max2) {
  const int oq = off_comp(qs, AXIS);
  const int c2 = q2 + 2 * D * oq + 1;
  const bool take = (ps & (kEsdfObs | kEsdfSite)) == kEsdfObs && (qs & kEsdfPar) && c2 <= max2 &&
                    (!(ps & kEsdfPar) || c2 < p2);
  if (take) {
    ps = (ps & ~kEsdfOffMask) | kEsdfPar | (qs & kEsdfOffMask & ~(511u << (9 * AXIS))) |
         (((uint32_t)(oq + D) & 511u) << (9 * AXIS));
    p2 = c2;
  }
}

// Both sweeps along AXIS of one line of eight voxels (first i = 1 .. 7, each
// voxel trying its predecessor's parent, then i = 6 .. 0, each trying its
// successor's), in registers.
template <int AXIS>
__device__ __forceinline__ void sweep_line(uint32_t* s, int* s2, int base, int max2) {
  constexpr int stride = AXIS == 0 ? 1 : (AXIS == 1 ? kSweepRow : kSweepSlice);
  uint32_t w[8];
  int d2[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    w[i] = s[base + stride * i];
    d2[i] = s2[base + stride * i];
  }
#pragma unroll
  for (int i = 1; i < 8; ++i) relax_line<AXIS, -1>(w[i], d2[i], w[i - 1], d2[i - 1], max2);
#pragma unroll
  for (int i = 6; i >= 0; --i) relax_line<AXIS, 1>(w[i], d2[i], w[i + 1], d2[i + 1], max2);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    s[base + stride * i] = w[i];
    s2[base + stride * i] = d2[i];
  }
}

// Six in-block sweeps of every block of the current update set (+x, -x,
// +y, -y, +z, -z).  64 threads sweep the 64 lines of an axis, one line
// each.  Afterwards the block and its existing face neighbours join this
// iteration's tlist.  Thread 0 of CTA 0 zeroes the next update set's size
// first (that set was consumed by the previous iteration).
__global__ void __launch_bounds__(64)
    esdf_sweep_kernel(const EsdfDev e, const uint32_t* __restrict__ list, const uint32_t* size,
                      uint32_t* zero_next, uint32_t* tlist, uint32_t* tsize, uint32_t gen_t) {
  __shared__ uint32_t s[kSweepWords];
  __shared__ int s2[kSweepWords];
  const uint32_t n = __ldcg(size);
  const int t = threadIdx.x;
  if (blockIdx.x == 0 && t == 0) {
    *zero_next = 0u;
    if (n) {
      atomicAdd(e.stats + 1, 1ull);
      atomicAdd(e.stats + 2, (unsigned long long)n);
    }
  }
  const int max2 = e.max_dist * e.max_dist;
  const int a = t & 7, c = t >> 3;  // the line's coordinates on the two other axes, in axis order
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    const uint32_t p = list[k];
    uint32_t* g = e.st + (size_t)p * 512;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t v = g[t + 64 * i];
      s[sweep_idx(t + 64 * i)] = v;
      s2[sweep_idx(t + 64 * i)] = dist2(v);
    }
    __syncthreads();
    sweep_line<0>(s, s2, kSweepRow * a + kSweepSlice * c, max2);
    __syncthreads();
    sweep_line<1>(s, s2, a + kSweepSlice * c, max2);
    __syncthreads();
    sweep_line<2>(s, s2, a + kSweepRow * c, max2);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) g[t + 64 * i] = s[sweep_idx(t + 64 * i)];
    if (t < 7) {
      const int q = t == 6 ? (int)p : e.nbr[6 * (size_t)p + t];
      if (q >= 0 && atomicExch(e.stamp_t + q, gen_t) != gen_t) tlist[atomicAdd(tsize, 1u)] = (uint32_t)q;
    }
  }
}

// Face exchange: each voxel on a face of the block tries the parent of the
// voxel across that face in the neighbouring block, faces in -x, +x, -y,
// +y, -z, +z order; reads st only, writes the block to st2 if it changed.
__global__ void __launch_bounds__(kEsdfThreads)
    esdf_pull_kernel(const EsdfDev e, const uint32_t* __restrict__ tlist, const uint32_t* tsize) {
  __shared__ int s_nb[6];
  const uint32_t n = __ldcg(tsize);
  const int t = threadIdx.x;
  const int max2 = e.max_dist * e.max_dist;
  if (blockIdx.x == 0 && t == 0 && n) atomicAdd(e.stats + 3, (unsigned long long)n);
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    const uint32_t p = tlist[k];
    __syncthreads();
    if (t < 6) s_nb[t] = e.nbr[6 * (size_t)p + t];
    __syncthreads();
    uint32_t v[4];
    bool any = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = 4 * t + i;
      const int x = l & 7, y = (l >> 3) & 7, z = l >> 6;
      const int c[3] = {x, y, z};
      v[i] = e.st[(size_t)p * 512 + l];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int axis = f >> 1;
        const int mine = (f & 1) ? 7 : 0;
        if (c[axis] != mine || s_nb[f] < 0) continue;
        const int ql = l + (axis == 0 ? 1 : (axis == 1 ? 8 : 64)) * (7 - 2 * mine);
        const uint32_t q = e.st[(size_t)s_nb[f] * 512 + ql];
        const int d = (f & 1) ? 1 : -1;
        any |= relax(v[i], q, axis == 0 ? d : 0, axis == 1 ? d : 0, axis == 2 ? d : 0, max2);
      }
    }
    any = __syncthreads_or(any);
    if (any) {
      uint4* dst = reinterpret_cast<uint4*>(e.st2 + (size_t)p * 512) + t;
      *dst = make_uint4(v[0], v[1], v[2], v[3]);
    }
    if (t == 0) e.tchanged[k] = any ? 1 : 0;
  }
}

// Copy the changed blocks back; they form the next update set.  One warp
// per tlist entry, four 16-byte vectors per lane.  Thread 0 of CTA 0 zeroes
// the other tlist's size (used by the previous iteration, filled by the
// next one).
__global__ void __launch_bounds__(kEsdfThreads)
    esdf_apply_kernel(const EsdfDev e, const uint32_t* __restrict__ tlist, const uint32_t* tsize,
                      uint32_t* zero_tsize, uint32_t* next, uint32_t* next_size, uint32_t gen_next) {
  constexpr int kWarps = kEsdfThreads / 32;
  const uint32_t n = __ldcg(tsize);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) *zero_tsize = 0u;
  for (uint32_t k = blockIdx.x * kWarps + warp; k < n; k += gridDim.x * kWarps) {
    if (!e.tchanged[k]) continue;
    const uint32_t p = tlist[k];
    uint4* dst = reinterpret_cast<uint4*>(e.st + (size_t)p * 512) + lane;
    const uint4* src = reinterpret_cast<const uint4*>(e.st2 + (size_t)p * 512) + lane;
    uint4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = src[32 * j];
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[32 * j] = v[j];
    if (lane == 0) add_update(e, next, next_size, p, gen_next);
  }
}

// ---------------------------------------------------------------- query

// Signed distance (m) at each point: the parent offset's length times the
// voxel size, negative inside; max_dist for an observed voxel without a
// parent; NaN for an unknown voxel or a point outside every block.
__global__ void esdf_query_kernel(const MapDev m, const EsdfDev e, const float* __restrict__ pts,
                                  int64_t n, float* __restrict__ dist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float out = __int_as_float(0x7fc00000);
  const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
  const float gx = floorf(__fdiv_rn(x, m.v)), gy = floorf(__fdiv_rn(y, m.v)), gz = floorf(__fdiv_rn(z, m.v));
  const float lim = 8.0f * 1048576.0f;
  if (fabsf(gx) < lim && fabsf(gy) < lim && fabsf(gz) < lim) {
    const int ix = (int)gx, iy = (int)gy, iz = (int)gz;
    const int p = pool_of(m, ix >> 3, iy >> 3, iz >> 3);
    if (p >= 0) {
      const uint32_t s = e.st[(size_t)p * 512 + (ix & 7) + 8 * (iy & 7) + 64 * (iz & 7)];
      if (s & kEsdfObs) {
        const float d = (s & kEsdfPar) ? sqrtf((float)dist2(s)) : (float)e.max_dist;
        out = ((s & kEsdfInside) ? -d : d) * m.v;
      }
    }
  }
  dist[i] = out;
}

// ---------------------------------------------------------------- import

// One CTA per input block: find or insert its key (a new key takes the next
// pool block), write its voxels in the map's storage, mark it changed.
__global__ void __launch_bounds__(kEsdfThreads)
    import_kernel(const MapDev m, const int32_t* __restrict__ keys, const float* __restrict__ D,
                  const float* __restrict__ W, int64_t n) {
  __shared__ int s_pool;
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    __syncthreads();
    if (t == 0) {
      const unsigned long long key = pack_key(keys[3 * b], keys[3 * b + 1], keys[3 * b + 2]);
      int pool = -1;
      uint32_t slot = hash_key(key) & m.cap_mask;
      for (uint32_t probe = 0; probe <= m.cap_mask; ++probe) {
        const unsigned long long old = atomicCAS(m.keys + slot, kEmptyKey, key);
        if (old == kEmptyKey) {
          const unsigned long long q = atomicAdd(m.counters + kCntBlocks, 1ull);
          if (q < (unsigned long long)m.max_blocks) {
            m.block_keys[q] = key;
            m.vals[slot] = (int)q;
            pool = (int)q;
          } else {
            m.vals[slot] = -1;
            atomicOr(m.counters + kCntStatus, (unsigned long long)kStPoolFull);
          }
          break;
        }
        if (old == key) {
          pool = m.vals[slot];
          break;
        }
        slot = (slot + 1) & m.cap_mask;
        if (probe == m.cap_mask) atomicOr(m.counters + kCntStatus, (unsigned long long)kStHashFull);
      }
      s_pool = pool;
    }
    __syncthreads();
    const int pool = s_pool;
    if (pool < 0) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int l = 4 * t + i;
      const float d = D[b * 512 + l], w = W[b * 512 + l];
      if (m.storage == kStorageOcc) {
        reinterpret_cast<float*>(m.pool)[(size_t)pool * 512 + l] = d;
      } else if (m.storage == kStorageF16) {
        reinterpret_cast<__half2*>(m.pool)[(size_t)pool * 512 + l] = __floats2half2_rn(d * m.inv_tau, w);
      } else if (m.storage == kStorageX16) {
        reinterpret_cast<uint32_t*>(m.pool)[(size_t)pool * 512 + l] = x16_pack(d, w, m.x16_scale);
      } else {
        reinterpret_cast<float2*>(m.pool)[(size_t)pool * 512 + l] = make_float2(d, w);
      }
    }
    if (t == 0 && m.dirty) m.dirty[pool] = kDirtyEsdf | kDirtyMesh;
  }
}

int grid_for(int per_sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms) * per_sm;
}

}  // namespace

cudaError_t launch_esdf_mark(const MapDev& m, const EsdfDev& e, uint32_t gen, cudaStream_t s) {
  if (m.storage == kStorageOcc) {
    // occupancy sites read across block faces: the neighbour table first
    esdf_nbr_kernel<<<grid_for(4), 256, 0, s>>>(m, e);
    esdf_occ_spread_kernel<<<grid_for(4), 256, 0, s>>>(m, e);
    esdf_occ_mark_kernel<<<grid_for(16), kEsdfThreads, 0, s>>>(m, e, gen);
  } else {
    esdf_mark_kernel<<<grid_for(16), kEsdfThreads, 0, s>>>(m, e, gen);
  }
  return cudaGetLastError();
}

cudaError_t launch_esdf_clear(const MapDev& m, const EsdfDev& e, uint32_t gen, cudaStream_t s) {
  esdf_clear_kernel<<<grid_for(10), kEsdfThreads, 0, s>>>(m, e, gen);  // 48 registers: 10 CTAs per SM
  if (m.storage != kStorageOcc) esdf_nbr_kernel<<<grid_for(4), 256, 0, s>>>(m, e);  // built before marking otherwise
  return cudaGetLastError();
}

// One lowering iteration (update set `cur`, tlist `cur`): sweep and build
// the tlist, exchange faces, apply.  With an empty current set every kernel
// returns at once.
cudaError_t launch_esdf_iteration(const MapDev& m, const EsdfDev& e, int cur, uint32_t gen_t,
                                  uint32_t gen_next, cudaStream_t s) {
  uint32_t* list = cur ? e.list[1] : e.list[0];
  uint32_t* next = cur ? e.list[0] : e.list[1];
  uint32_t* tl = cur ? e.tlist[1] : e.tlist[0];
  uint32_t* tsize = e.cnt + 3 + cur;
  // latency-bound stages: enough resident warps per SM to overlap the
  // blocks' loads (sweep 40 registers x 64 threads, pull 32 x 128)
  esdf_sweep_kernel<<<grid_for(24), 64, 0, s>>>(e, list, e.cnt + cur, e.cnt + (1 - cur), tl, tsize, gen_t);
  esdf_pull_kernel<<<grid_for(16), kEsdfThreads, 0, s>>>(e, tl, tsize);
  esdf_apply_kernel<<<grid_for(16), kEsdfThreads, 0, s>>>(e, tl, tsize, e.cnt + 3 + (1 - cur), next,
                                                          e.cnt + (1 - cur), gen_next);
  (void)m;
  return cudaGetLastError();
}

cudaError_t launch_esdf_query(const MapDev& m, const EsdfDev& e, const float* pts, int64_t n,
                              float* dist, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  esdf_query_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(m, e, pts, n, dist);
  return cudaGetLastError();
}

cudaError_t launch_import(const MapDev& m, const int32_t* keys, const float* D, const float* W,
                          int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  import_kernel<<<grid_for(8), kEsdfThreads, 0, s>>>(m, keys, D, W, n);
  return cudaGetLastError();
}

}  // namespace gbt
