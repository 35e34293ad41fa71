// Internal device-side data layout of the GB300 TSDF library (not part of the
// C ABI).  One map = a block hash (Sec. IV-A: integer block coordinates ->
// 8x8x8-voxel block) plus a pool of blocks stored contiguously in HBM.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gbt {

constexpr int kBlockVoxels = 512;      // 8 x 8 x 8, x fastest
constexpr int kMaxCells = 32;          // cap on blocks met by one band segment
constexpr int kMaxFrames = 32;         // frames per batch (one bit each in the slot mask)
constexpr int kMaxMaps = 16;           // maps per batch
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kAllocThreads = 256;     // threads per allocation CTA
constexpr int kTileW = 32;             // allocation CTA = one 32 x (16 or 32) pixel tile
constexpr int kTileHSmall = 16;        // small launches: more CTAs
constexpr int kTileHBig = 32;          // large launches: fewer, fuller CTAs
constexpr int kBigTilePixels = 1 << 21;  // pixels per launch from which big tiles are used
constexpr int kSetBits = 10;           // CTA-local block-key set: 1024 slots
constexpr int kSetSize = 1 << kSetBits;
constexpr int kSetProbes = 32;
constexpr int kIntegrateThreads = 128; // 4 voxels per thread

// Per-map u64 counters.
enum : int {
  kCntBlocks = 0,   // pool blocks handed out (may exceed max_blocks when full)
  kCntUpdates = 1,  // voxel updates
  kCntStatus = 2,   // sticky status bits
  kCntVisits = 3,   // work-list entries consumed by integration launches
  kCntLaunches = 4, // integration launches
  kCntSegments = 5, // band segments walked by the allocator (valid pixels in range)
  kCntCells = 6,    // cells emitted by those walks (with repeats across pixels)
  kCntPairs = 7,    // (block, frame) pairs integrated: 512 voxel projections each
  kNumCounters = 8
};
// Sticky status bits.
enum : unsigned long long { kStPoolFull = 1, kStHashFull = 2, kStListFull = 4, kStTimeout = 8 };

enum : int { kSensorPinhole = 0, kSensorLidar = 1 };
// Voxel storage: TSDF {D, W} as FP32, as FP16 (D / tau) or as 16-bit fixed
// point (D / tau) with an FP16 weight, occupancy log-odds as one FP32 value,
// or colour {r, g, b, W} as four FP32 values.  The first three codes are the
// ABI's TSDF_STORAGE_* values.
enum : int { kStorageF32 = 0, kStorageF16 = 1, kStorageX16 = 2, kStorageOcc = 3, kStorageColor = 4 };

// 16-bit fixed-point TSDF voxel (one 32-bit word): D / tau as a signed
// fraction with kX16Steps steps per tau in the low half (round to nearest,
// saturating at +-tau), W as an FP16 number in the high half.
constexpr float kX16Steps = 32767.0f;
__host__ __device__ __forceinline__ float x16_dist(uint32_t word, float unit) {
  return (float)(int16_t)(uint16_t)(word & 0xFFFFu) * unit;
}
__host__ __device__ __forceinline__ float x16_weight(uint32_t word) {
  __half_raw r;
  r.x = (unsigned short)(word >> 16);
  return __half2float(__half(r));
}
__device__ __forceinline__ uint32_t x16_pack(float D, float W, float scale) {
  const float q = fminf(fmaxf(__fmul_rn(D, scale), -kX16Steps), kX16Steps);
  const int qi = __float2int_rn(q);
  const __half h = __float2half_rn(W);
  return ((uint32_t)qi & 0xFFFFu) | ((uint32_t)__half_as_ushort(h) << 16);
}

// Device view of one map.  The work list holds the hash slots met by the
// frames of the batch in flight; the integration launch consumes it and its
// last CTA resets the list length.  vals[slot]: pool index >= 0; -1 = no pool block
// (pool was full); <= -2 = block allocated by the current batch, pool index
// -v - 2, contents not yet initialised.
struct MapDev {
  unsigned long long* keys;       // [cap] packed block keys, kEmptyKey = free
  int32_t* vals;                  // [cap]
  uint32_t* mask;                 // [cap] frames of the current batch meeting the block
  void* pool;                     // [max_blocks][512] float2 {D, W}, __half2 {D/tau, W} or
                                  // fixed-point words (x16_pack)
  unsigned long long* block_keys; // [max_blocks] key of each pool block
  unsigned long long* counters;   // [kNumCounters]; kCntSegments and kCntCells are
                                  // written only when walk_stats != 0
  int32_t walk_stats;             // count band segments and cells (diagnostic)
  uint32_t* list;                 // [list_cap] slots met by the current batch
  unsigned int* ctl;              // [0] list length, [1] finished integration CTAs,
                                  // [2] entries handed out (first map of a batch)
  uint32_t list_cap;
  uint32_t cap_mask;              // hash capacity - 1 (power of two)
  int32_t max_blocks;
  int32_t storage;
  int32_t lidar_nearest;
  float v;                        // voxel edge (m)
  float tau;                      // truncation distance, (float)(trunc * (double)v)
  float inv_tau;
  float x16_scale, x16_unit;      // fixed-point storage: steps per metre, metres per step
  float wmax;
  float guard;                    // LiDAR bilinear guard (m)
  float l_occ, l_free;            // occupancy layer: log-odds added per update
  int32_t weighting;              // TSDF weight: bit 0 inverse square depth, bit 1 drop-off
  float dropoff;                  // drop-off start behind the surface (m)
  uint8_t* dirty;                 // [max_blocks] kDirtyEsdf / kDirtyMesh: changed since the
                                  // last ESDF update / mesh extraction (may be null)
};
// kDirtyNbr: a face neighbour changed (occupancy ESDF sites read across faces)
enum : uint8_t { kDirtyEsdf = 1, kDirtyMesh = 2, kDirtyNbr = 4 };

// ESDF layer of a map (Sec. IV-C), indexed like the pool.  State word per
// voxel: parent offset x, y, z as 9-bit two's complement in bits 0-8, 9-17,
// 18-26; kEsdfObs, kEsdfSite, kEsdfPar (has a parent), kEsdfInside.
constexpr uint32_t kEsdfObs = 1u << 27, kEsdfSite = 1u << 28, kEsdfPar = 1u << 29,
                   kEsdfInside = 1u << 30;
constexpr uint32_t kEsdfOffMask = (1u << 27) - 1u;
constexpr int kEsdfBitWords = (1 << 16) / 32;
struct EsdfDev {
  uint32_t* st;         // [max_blocks][512] voxel states
  uint32_t* st2;        // [max_blocks][512] states produced by a face exchange
  uint32_t* list[2];    // [max_blocks] update sets (current, next)
  uint32_t* tlist[2];   // [max_blocks] update set and its face neighbours (alternate
                        // iterations use alternate lists)
  uint32_t* clist;      // [max_blocks] blocks where a site disappeared
  uint32_t* stamp_s;    // [max_blocks] generation that put the block in an update set
  uint32_t* stamp_t;    // [max_blocks] generation that put the block in a tlist
  uint8_t* tchanged;    // [max_blocks] per tlist entry: the exchange changed the block
  int32_t* nbr;         // [max_blocks][6] pool index of each face neighbour (-x, +x, -y,
                        // +y, -z, +z), -1 if none; rebuilt by every update
  uint32_t* bits;       // [2][kEsdfBitWords] hashed bitmaps of the clist blocks and of their
                        // coarse cells, rebuilt by every update
  uint32_t* cnt;        // [0], [1] update set sizes, [2] clist size, [3], [4] tlist sizes
  unsigned long long* stats;    // [0] voxels whose parent stopped being a site, [1] lowering
                                // iterations, [2] blocks swept, [3] blocks in face exchanges
  float site_eps, min_weight;
  int32_t max_dist;     // voxels, <= 255
};

// One frame as the kernels see it.  Geometry is anchor-relative: a is the
// block holding the sensor origin; Rcl, tloc map anchor-local voxel centres
// into the sensor frame; M, o map sensor rays into anchor-relative block
// units.  All FP32 values are rounded once from FP64 on the host.
struct FrameDev {
  int32_t kind, map, width, height;
  const float* depth;
  const uint32_t* rgba;  // colour layer: registered colour image (r in the low byte)
  const float* tab;      // LiDAR: cos/sin of beam azimuths [2*n_az], then polar [2*n_el]
  float fu, fv, cu, cv;  // pinhole
  float theta_start, phi_start, alpha, beta, min_range, max_range;  // LiDAR
  float Rcl[9], tloc[3];
  float M[9], o[3];
  int32_t a[3];
  int32_t blk_begin;     // first allocation CTA of this frame
  int32_t bit;           // bit of this frame in the slot masks = its index in the batch
  int32_t fast_rcp;      // host check: this frame's inverted decision values are in [2^-126, 2^126]
  int32_t short_walks;   // host check: this frame's band segments meet fewer than kMaxCells blocks
};

template <int NF, int NM>
struct BatchParams {
  int32_t n_frames;
  int32_t n_maps;
  int32_t overlap;     // launched as a programmatic dependent of the stream's previous kernel
  int32_t alloc_ctas;  // allocation tiles of the batch (the fused kernel loops over them)
  int32_t wait_extra;  // test hook: the fused kernel's grid wait expects this many extra CTAs
  int32_t fast_rcp;    // every reciprocal of the batch's decisions lies in [2^-126, 2^126] or is not taken
  MapDev maps[NM];
  FrameDev fr[NF];
};

// Block key: three 21-bit fields holding coordinate + 2^20 (x lowest), so a
// unit step along an axis is a plain add of 1 << (21 * axis) to the key.
// Bit 63 is always 0, so no key equals kEmptyKey.
constexpr int kKeyBias = 1 << 20;
__host__ __device__ __forceinline__ constexpr unsigned long long pack_key(int x, int y, int z) {
  return (unsigned long long)(unsigned)(x + kKeyBias) |
         ((unsigned long long)(unsigned)(y + kKeyBias) << 21) |
         ((unsigned long long)(unsigned)(z + kKeyBias) << 42);
}
__host__ __device__ __forceinline__ int key_coord(unsigned long long k, int axis) {
  return (int)((k >> (21 * axis)) & 0x1FFFFF) - kKeyBias;
}
// 64-bit finaliser (MurmurHash3 fmix64) for slot selection.
__host__ __device__ __forceinline__ uint32_t hash_key(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)k;
}

// Launchers (kernels.cu).
// Slot of `key` in the hash, or -1 (linear probing, bounded by the table size).
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

template <int NF, int NM>
cudaError_t launch_band_alloc(const BatchParams<NF, NM>& p, int n_ctas, int tile_h, cudaStream_t s);
template <int NF, int NM>
cudaError_t launch_integrate(const BatchParams<NF, NM>& p, int n_ctas, cudaStream_t s);
// Allocation and integration of one batch in a single cooperative launch;
// cudaErrorNotSupported for batches it does not cover (the caller then
// launches the two kernels).
template <int NF, int NM>
cudaError_t launch_fused(const BatchParams<NF, NM>& p, int tile_h, cudaStream_t s);
cudaError_t launch_query_color(const MapDev& m, const float* pts, int64_t n, float* rgb, float* weight,
                               cudaStream_t s);
cudaError_t launch_query(const MapDev& m, const float* pts, int64_t n, float* dist, float* weight,
                         cudaStream_t s);
cudaError_t launch_reset(const MapDev& m, uint32_t cap, cudaStream_t s);
cudaError_t launch_decay(const MapDev& m, float d_occ, float d_free, cudaStream_t s);
// ESDF stages (esdf.cu); `cur` selects the current update set.
cudaError_t launch_esdf_mark(const MapDev& m, const EsdfDev& e, uint32_t gen, cudaStream_t s);
cudaError_t launch_esdf_clear(const MapDev& m, const EsdfDev& e, uint32_t gen, cudaStream_t s);
cudaError_t launch_esdf_iteration(const MapDev& m, const EsdfDev& e, int cur, uint32_t gen_t,
                                  uint32_t gen_next, cudaStream_t s);
cudaError_t launch_esdf_query(const MapDev& m, const EsdfDev& e, const float* pts, int64_t n,
                              float* dist, cudaStream_t s);
cudaError_t launch_import(const MapDev& m, const int32_t* keys, const float* D, const float* W,
                          int64_t n, cudaStream_t s);

// Marching-cubes case table: triangles (edge numbers) of each inside mask.
struct MeshTable {
  uint8_t count[256];
  int8_t edges[256][15];
};
// Meshing scratch of a map, allocated by the first extraction.
struct MeshDev {
  uint32_t* list;     // [max_blocks] blocks to mesh
  uint32_t* stamp;    // [max_blocks] generation that listed the block
  unsigned long long* cnt;  // [0] list size, [1] triangles produced
};
cudaError_t launch_mesh(const MapDev& m, const MeshDev& md, const MeshTable& table, int changed_only,
                        uint32_t gen, float min_weight, float* pos, int32_t* keys, int32_t* cubes,
                        int64_t cap, cudaStream_t s);
int integrate_ctas_per_sm(int storage);

}  // namespace gbt
