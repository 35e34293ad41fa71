// Marching-cubes meshing of TSDF blocks (Sec. IV-B: updated blocks are
// meshed with a parallel Marching Cubes), sm_103a.
//
//  mesh_list_kernel  the blocks to mesh: every block, or every block changed
//                    since the last extraction together with the seven
//                    blocks whose cubes reach into it (-x, -y, -z sides)
//  mesh_kernel       one warp per listed block: the block's 8^3 voxels and
//                    the +x / +y / +z faces, edges and corner of its
//                    neighbours (9^3 values) are staged in the warp's part
//                    of shared memory; each lane classifies two lines of
//                    eight cubes along x with the case table (held in
//                    shared memory: lanes index it by their own cases); the
//                    warp reserves the block's output with one atomic (a
//                    scan of the lanes' triangle counts), lists the cubes
//                    with triangles and deals them out across its lanes
//
// A cube joins voxel centres g .. g + (1, 1, 1) and belongs to the block
// holding g; it is meshed only if its eight corners exist and are observed.
// Vertices are interpolated in FP32 on the edge from its lower corner.
#include "tsdf_internal.cuh"

namespace gbt {
namespace {

constexpr int kMeshWarps = 4;                    // blocks meshed at once per CTA
constexpr int kSide = 9;                         // staged values per axis
constexpr int kStaged = kSide * kSide * kSide;   // 729
constexpr int kHalo = kStaged - 512;             // 217 values of the neighbours

__device__ __forceinline__ int pool_at(const MapDev& m, int x, int y, int z) {
  const int slot = hash_find(m, pack_key(x, y, z));
  if (slot < 0) return -1;
  const int val = m.vals[slot];
  return val >= 0 ? val : -1;
}

__device__ __forceinline__ void add_block(const MeshDev& md, uint32_t p, uint32_t gen) {
  if (atomicExch(md.stamp + p, gen) != gen) md.list[atomicAdd(md.cnt, 1ull)] = p;
}

__global__ void mesh_list_kernel(const MapDev m, const MeshDev md, int changed_only, uint32_t gen) {
  const uint32_t nb = (uint32_t)min((unsigned long long)m.max_blocks, __ldcg(m.counters + kCntBlocks));
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nb; p += gridDim.x * blockDim.x) {
    if (!changed_only) {
      add_block(md, p, gen);
      continue;
    }
    if (!(m.dirty[p] & kDirtyMesh)) continue;
    m.dirty[p] &= (uint8_t)~kDirtyMesh;
    const unsigned long long key = m.block_keys[p];
    const int bx = key_coord(key, 0), by = key_coord(key, 1), bz = key_coord(key, 2);
    for (int c = 0; c < 8; ++c) {
      const int q = c == 0 ? (int)p : pool_at(m, bx - (c & 1), by - ((c >> 1) & 1), bz - ((c >> 2) & 1));
      if (q >= 0) add_block(md, (uint32_t)q, gen);
    }
  }
}

// TSDF value of voxel l of pool block q and whether it is observed
// (W >= min_weight); a missing block (q < 0) is unobserved.
__device__ __forceinline__ float staged_voxel(const MapDev& m, int q, int l, float min_weight, bool& ok) {
  ok = false;
  if (q < 0) return 0.0f;
  float d, w;
  if (m.storage == kStorageF16) {
    const __half2 h = reinterpret_cast<const __half2*>(m.pool)[(size_t)q * 512 + l];
    d = __low2float(h) * m.tau;
    w = __high2float(h);
  } else if (m.storage == kStorageX16) {
    const uint32_t word = reinterpret_cast<const uint32_t*>(m.pool)[(size_t)q * 512 + l];
    d = x16_dist(word, m.x16_unit);
    w = x16_weight(word);
  } else {
    const float2 v = reinterpret_cast<const float2*>(m.pool)[(size_t)q * 512 + l];
    d = v.x;
    w = v.y;
  }
  ok = w >= min_weight;
  return d;
}

__global__ void __launch_bounds__(kMeshWarps * 32, 8)
    mesh_kernel(const MapDev m, const MeshDev md, const __grid_constant__ MeshTable tab, float min_weight,
                float* __restrict__ out_pos, int32_t* __restrict__ out_keys,
                int32_t* __restrict__ out_cube, int64_t cap) {
  __shared__ float s_d[kMeshWarps][kStaged];         // D at staged (x, y, z), x fastest
  __shared__ uint8_t s_ok[kMeshWarps][kStaged + 7];  // observed
  __shared__ uint32_t s_list[kMeshWarps][512];       // the block's cubes with triangles
  __shared__ uint8_t s_count[256];
  __shared__ int8_t s_edges[256 * 15];
  {
    const uint8_t* src = reinterpret_cast<const uint8_t*>(&tab);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_count[i] = src[i];
    for (int i = threadIdx.x; i < 256 * 15; i += blockDim.x) s_edges[i] = (int8_t)src[256 + i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sd = s_d[warp];
  uint8_t* sok = s_ok[warp];
  uint32_t* list = s_list[warp];
  const uint32_t n = (uint32_t)__ldcg(md.cnt);
  for (uint32_t k = blockIdx.x * kMeshWarps + warp; k < n; k += gridDim.x * kMeshWarps) {
    const uint32_t p = md.list[k];
    const unsigned long long key = m.block_keys[p];
    const int bx = key_coord(key, 0), by = key_coord(key, 1), bz = key_coord(key, 2);
    // pool block of the block (lane 0) and of its neighbour at offset
    // (lane & 1, lane >> 1 & 1, lane >> 2) for lanes 1 .. 7
    const int nbq = lane == 0 ? (int)p
                    : (lane < 8 ? pool_at(m, bx + (lane & 1), by + ((lane >> 1) & 1), bz + (lane >> 2)) : -1);
    __syncwarp();  // the previous block's reads of the staging are done
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int l = lane + 32 * it;
      const int i = (l & 7) + kSide * ((l >> 3) & 7) + kSide * kSide * (l >> 6);
      bool ok;
      sd[i] = staged_voxel(m, (int)p, l, min_weight, ok);
      sok[i] = ok ? 1 : 0;
    }
    // the 217 halo values: the +x, +y and +z faces (64 each), the three
    // edges (8 each) and the corner
#pragma unroll
    for (int it = 0; it < (kHalo + 31) / 32; ++it) {
      const int h = lane + 32 * it;
      const int a = h & 7, b = (h >> 3) & 7;
      int nb, sx, sy, sz, l;
      if (h < 64) {
        nb = 1; sx = 8; sy = a; sz = b; l = 8 * a + 64 * b;
      } else if (h < 128) {
        nb = 2; sx = a; sy = 8; sz = b; l = a + 64 * b;
      } else if (h < 192) {
        nb = 4; sx = a; sy = b; sz = 8; l = a + 8 * b;
      } else if (h < 200) {
        nb = 3; sx = 8; sy = 8; sz = a; l = 64 * a;
      } else if (h < 208) {
        nb = 5; sx = 8; sy = a; sz = 8; l = 8 * a;
      } else if (h < 216) {
        nb = 6; sx = a; sy = 8; sz = 8; l = a;
      } else {
        nb = 7; sx = 8; sy = 8; sz = 8; l = 0;
      }
      const int q = __shfl_sync(0xffffffffu, nbq, nb);
      if (h < kHalo) {
        const int i = sx + kSide * sy + kSide * kSide * sz;
        bool ok;
        sd[i] = staged_voxel(m, q, l, min_weight, ok);
        sok[i] = ok ? 1 : 0;
      }
    }
    __syncwarp();
    // cases of the lane's cubes: lines (y, z) = (lane & 7, lane >> 3) and
    // (lane & 7, 4 + (lane >> 3)), cubes x = 0 .. 7 along each; a column of
    // four corners at x gives the even case bits (0, 2, 4, 6) of cube x and
    // the odd ones of cube x - 1
    uint32_t cw[4];  // case of cube x of line j in byte x & 3 of cw[2 j + (x >> 2)]
    int mine = 0, busy = 0;  // the lane's triangles and cubes with triangles
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int y = lane & 7, z = (lane >> 3) + 4 * j;
      const int r = kSide * y + kSide * kSide * z;
      uint32_t prev_in = 0;
      bool prev_ok = false;
      cw[2 * j] = cw[2 * j + 1] = 0u;
#pragma unroll
      for (int x = 0; x <= 8; ++x) {
        const int i0 = r + x, i1 = i0 + kSide, i2 = i0 + kSide * kSide, i3 = i2 + kSide;
        const uint32_t in = (sd[i0] < 0.0f ? 1u : 0u) | (sd[i1] < 0.0f ? 4u : 0u) | (sd[i2] < 0.0f ? 16u : 0u) |
                            (sd[i3] < 0.0f ? 64u : 0u);
        const bool ok = (sok[i0] & sok[i1] & sok[i2] & sok[i3]) != 0;
        if (x > 0) {
          const uint32_t ci = (prev_ok && ok) ? (prev_in | (in << 1)) : 0u;
          cw[2 * j + ((x - 1) >> 2)] |= ci << (8 * ((x - 1) & 3));
          const int nt = s_count[ci];
          mine += nt;
          busy += nt ? 1 : 0;
        }
        prev_in = in;
        prev_ok = ok;
      }
    }
    // one output reservation per block: inclusive scans of the lanes'
    // triangle and cube counts
    int incl = mine, bincl = busy;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      const int yb = __shfl_up_sync(0xffffffffu, bincl, o);
      if (lane >= o) {
        incl += y;
        bincl += yb;
      }
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int ncubes = __shfl_sync(0xffffffffu, bincl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(md.cnt + 1, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    // list the cubes with triangles: cube index (9 bits), case (8 bits),
    // first triangle within the block (15 bits)
    {
      int slot = bincl - busy, tri = incl - mine;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int ci = (int)((cw[c >> 2] >> (8 * (c & 3))) & 255u);
        const int nt = s_count[ci];
        if (nt) {
          const int cube = (c & 7) + 8 * (lane & 7) + 64 * ((lane >> 3) + 4 * (c >> 3));
          list[slot++] = (uint32_t)cube | ((uint32_t)ci << 9) | ((uint32_t)tri << 17);
          tri += nt;
        }
      }
    }
    __syncwarp();
    // emit: the listed cubes dealt out across the lanes
    for (int e = lane; e < ncubes; e += 32) {
      const uint32_t ent = list[e];
      const int cube = (int)(ent & 511u), ci = (int)((ent >> 9) & 255u);
      const int x = cube & 7, y = (cube >> 3) & 7, z = cube >> 6;
      const int nt = s_count[ci];
      const float* corner = sd + x + kSide * y + kSide * kSide * z;  // corner 0
      const int gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
      unsigned long long o = base + (ent >> 17);
      for (int tr = 0; tr < nt; ++tr, ++o) {
        if (o >= (unsigned long long)cap) continue;
        if (out_cube) {
          out_cube[3 * o] = gx;
          out_cube[3 * o + 1] = gy;
          out_cube[3 * o + 2] = gz;
        }
        for (int vtx = 0; vtx < 3; ++vtx) {
          const int ed = s_edges[15 * ci + 3 * tr + vtx];
          const int axis = ed >> 2, u = ed & 1, w = (ed >> 1) & 1;
          // lower corner of edge ed: bit `axis` clear, the other two axes u, w
          const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
          const int lo = (u << o1) | (w << o2), hi = lo | (1 << axis);
          const float dlo = corner[(lo & 1) + kSide * ((lo >> 1) & 1) + kSide * kSide * (lo >> 2)];
          const float dhi = corner[(hi & 1) + kSide * ((hi >> 1) & 1) + kSide * kSide * (hi >> 2)];
          const float tt = __fdiv_rn(dlo, __fsub_rn(dlo, dhi));
          const int g[3] = {gx + (lo & 1), gy + ((lo >> 1) & 1), gz + (lo >> 2)};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float cf = __fadd_rn((float)g[a], 0.5f);
            if (a == axis) cf = __fadd_rn(cf, tt);
            out_pos[9 * o + 3 * vtx + a] = __fmul_rn(cf, m.v);
            if (out_keys) out_keys[12 * o + 4 * vtx + a] = g[a];
          }
          if (out_keys) out_keys[12 * o + 4 * vtx + 3] = axis;
        }
      }
    }
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

cudaError_t launch_mesh(const MapDev& m, const MeshDev& md, const MeshTable& table, int changed_only,
                        uint32_t gen, float min_weight, float* pos, int32_t* keys, int32_t* cubes,
                        int64_t cap, cudaStream_t s) {
  const int sms = sm_count();
  mesh_list_kernel<<<sms * 2, 256, 0, s>>>(m, md, changed_only, gen);
  mesh_kernel<<<sms * 8, kMeshWarps * 32, 0, s>>>(m, md, table, min_weight, pos, keys, cubes, cap);
  return cudaGetLastError();
}

}  // namespace gbt
