// Marching-cubes meshing of TSDF blocks (Sec. IV-B: updated blocks are
// meshed with a parallel Marching Cubes), sm_103a.
//
//  mesh_list_kernel  the blocks to mesh: every block, or every block changed
//                    since the last extraction together with the seven
//                    blocks whose cubes reach into it (-x, -y, -z sides)
//  mesh_kernel       one CTA per listed block: the block's 8^3 voxels and
//                    the +x / +y / +z faces, edges and corner of its
//                    neighbours (9^3 values) are staged in shared memory;
//                    each thread meshes four cubes with the case table; the
//                    block reserves its output with one atomic (a scan of
//                    the threads' triangle counts)
//
// A cube joins voxel centres g .. g + (1, 1, 1) and belongs to the block
// holding g; it is meshed only if its eight corners exist and are observed.
// Vertices are interpolated in FP32 on the edge from its lower corner.
#include "tsdf_internal.cuh"

namespace gbt {
namespace {

constexpr int kMeshThreads = 128;  // 4 cubes per thread
constexpr int kSide = 9;           // staged values per axis

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

__global__ void __launch_bounds__(kMeshThreads)
    mesh_kernel(const MapDev m, const MeshDev md, const __grid_constant__ MeshTable tab, float min_weight,
                float* __restrict__ out_pos, int32_t* __restrict__ out_keys,
                int32_t* __restrict__ out_cube, int64_t cap) {
  __shared__ float s_d[kSide * kSide * kSide];
  __shared__ uint8_t s_ok[kSide * kSide * kSide];
  __shared__ int s_pool[8];
  __shared__ int s_warp[kMeshThreads / 32];
  __shared__ unsigned long long s_base;
  const uint32_t n = (uint32_t)__ldcg(md.cnt);
  const int t = threadIdx.x;
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    const uint32_t p = md.list[k];
    const unsigned long long key = m.block_keys[p];
    const int bx = key_coord(key, 0), by = key_coord(key, 1), bz = key_coord(key, 2);
    __syncthreads();
    if (t < 8)
      s_pool[t] = t == 0 ? (int)p : pool_at(m, bx + (t & 1), by + ((t >> 1) & 1), bz + ((t >> 2) & 1));
    __syncthreads();
    for (int i = t; i < kSide * kSide * kSide; i += kMeshThreads) {
      const int x = i % kSide, y = (i / kSide) % kSide, z = i / (kSide * kSide);
      const int nb = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
      const int q = s_pool[nb];
      float d = 0.0f;
      bool ok = false;
      if (q >= 0) {
        const int l = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
        float w;
        if (m.storage == kStorageF16) {
          const __half2 h = reinterpret_cast<const __half2*>(m.pool)[(size_t)q * 512 + l];
          d = __low2float(h) * m.tau;
          w = __high2float(h);
        } else {
          const float2 v = reinterpret_cast<const float2*>(m.pool)[(size_t)q * 512 + l];
          d = v.x;
          w = v.y;
        }
        ok = w >= min_weight;
      }
      s_d[i] = d;
      s_ok[i] = ok ? 1 : 0;
    }
    __syncthreads();
    // case of each of this thread's four cubes (0 = nothing to mesh)
    int cases[4];
    int mine = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = 4 * t + j;
      const int x = l & 7, y = (l >> 3) & 7, z = l >> 6;
      int ci = 0;
      bool all = true;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = (x + (c & 1)) + kSide * (y + ((c >> 1) & 1)) + kSide * kSide * (z + (c >> 2));
        all = all && s_ok[i];
        if (s_d[i] < 0.0f) ci |= 1 << c;
      }
      cases[j] = all ? ci : 0;
      mine += tab.count[cases[j]];
    }
    // one output reservation per block: exclusive scan of the threads' counts
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((t & 31) >= o) incl += y;
    }
    if ((t & 31) == 31) s_warp[t >> 5] = incl;
    __syncthreads();
    if (t == 0) {
      int acc = 0;
      for (int w = 0; w < kMeshThreads / 32; ++w) {
        const int c = s_warp[w];
        s_warp[w] = acc;
        acc += c;
      }
      s_base = acc ? atomicAdd(md.cnt + 1, (unsigned long long)acc) : 0ull;
    }
    __syncthreads();
    unsigned long long o = s_base + (unsigned long long)(s_warp[t >> 5] + incl - mine);
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      const int ci = cases[j];
      const int nt = tab.count[ci];
      if (nt == 0) continue;
      const int l = 4 * t + j;
      const int x = l & 7, y = (l >> 3) & 7, z = l >> 6;
      float dc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        dc[c] = s_d[(x + (c & 1)) + kSide * (y + ((c >> 1) & 1)) + kSide * kSide * (z + (c >> 2))];
      const int gx = 8 * bx + x, gy = 8 * by + y, gz = 8 * bz + z;
      for (int tr = 0; tr < nt; ++tr, ++o) {
        if (o >= (unsigned long long)cap) continue;
        if (out_cube) {
          out_cube[3 * o] = gx;
          out_cube[3 * o + 1] = gy;
          out_cube[3 * o + 2] = gz;
        }
        for (int vtx = 0; vtx < 3; ++vtx) {
          const int e = tab.edges[ci][3 * tr + vtx];
          const int axis = e >> 2, u = e & 1, w = (e >> 1) & 1;
          // lower corner of edge e: bit `axis` clear, the other two axes u, w
          const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
          const int lo = (u << o1) | (w << o2), hi = lo | (1 << axis);
          const float tt = __fdiv_rn(dc[lo], __fsub_rn(dc[lo], dc[hi]));
          const int g[3] = {gx + (lo & 1), gy + ((lo >> 1) & 1), gz + (lo >> 2)};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float c = __fadd_rn((float)g[a], 0.5f);
            if (a == axis) c = __fadd_rn(c, tt);
            out_pos[9 * o + 3 * vtx + a] = __fmul_rn(c, m.v);
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
  mesh_kernel<<<sms * 8, kMeshThreads, 0, s>>>(m, md, table, min_weight, pos, keys, cubes, cap);
  return cudaGetLastError();
}

}  // namespace gbt
