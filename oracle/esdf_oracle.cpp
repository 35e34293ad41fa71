/*
 * CPU oracle for the incremental ESDF of nvblox (Sec. IV-C) — TEST
 * INFRASTRUCTURE ONLY.  It is loaded by the test suite through ctypes and
 * shares no code with the CUDA library.
 *
 * What it computes.  An ESDF layer sits on the blocks of a TSDF layer.  Each
 * ESDF voxel is unknown, or observed; an observed voxel may be a site (a
 * surface voxel: TSDF distance within site_eps of zero) and may hold a
 * parent, the offset from the voxel to the site it is closest to as far as
 * the propagation has found; its distance is the length of that offset.  One
 * update call takes the current TSDF blocks and the set of blocks changed
 * since the previous call and runs the stages of Sec. IV-C in order:
 *
 *   1. Allocate blocks: every changed TSDF block gets an ESDF block (all
 *      voxels unknown) if it has none.
 *   2. Mark sites, in the changed blocks.  Observed = W >= min_weight;
 *      site = observed and |D| <= site_eps; inside = observed and D < 0
 *      (every test on the FP32 TSDF values).  A new site takes itself as
 *      parent.  A voxel that stops being a site, becomes observed, or
 *      changes sides (inside <-> outside) loses its parent.  Blocks where a
 *      site disappeared are "to clear"; blocks with any change are "to
 *      update".
 *   3. Clear invalid: every ESDF block within ceil(max_dist / 8) + 1 blocks
 *      (Chebyshev distance in block coordinates) of a block to clear is
 *      checked voxel by voxel; a voxel whose parent voxel is no longer a site
 *      loses its parent and its block joins "to update".
 *   4. Lower, until no block changes: (a) sweep every block of the update
 *      set in +x, -x, +y, -y, +z, -z order, each voxel along a line trying
 *      the parent of the voxel before it; (b) every block of the update set
 *      and its six face neighbours tries, for each voxel on its faces, the
 *      parent of the adjacent voxel across the face (faces in -x, +x, -y,
 *      +y, -z, +z order), reading the neighbours as they were before this
 *      step; the blocks that changed form the next update set.
 *
 * Occupancy layers (Sec. IV-C: an occupancy voxel is a site if it is
 * adjacent to free voxels).  With set_occupancy the D input holds log-odds
 * l (W is ignored): a voxel is occupied if l > 0, free if l < 0 and unknown
 * if l == 0 (probability 1/2, never observed or decayed back); observed =
 * occupied or free; inside = occupied; site = occupied with a free voxel
 * among its six face neighbours (a neighbour in a block absent from the
 * input is unknown).  A voxel's site status then depends on the next block,
 * so stage 2 marks the changed blocks and their face neighbours.
 *
 * A voxel p "tries" the parent of a neighbour q when p is observed and not a
 * site and q has a parent: the candidate offset is (q + parent_q) - p; it is
 * taken if its squared length is at most max_dist^2 and strictly smaller
 * than p's current one (or p has none).  All of this is integer arithmetic,
 * so the result is exact and order-defined.
 *
 * State word of a voxel (uint32): bits 0-8, 9-17, 18-26 hold the parent
 * offset's x, y, z as 9-bit two's complement; bit 27 observed, bit 28 site,
 * bit 29 has a parent, bit 30 inside.  max_dist is at most 255 voxels.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

constexpr uint32_t kObs = 1u << 27, kSite = 1u << 28, kPar = 1u << 29, kInside = 1u << 30;
constexpr uint32_t kOffMask = (1u << 27) - 1u;

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
    return (size_t)(k.x * 73856093LL) ^ (size_t)(k.y * 19349663LL) ^ (size_t)(k.z * 83492791LL);
  }
};

struct Block {
  uint32_t s[512];
};

struct Esdf {
  float v = 0.0f, site_eps = 0.0f, min_weight = 0.0f;
  int32_t max_dist = 0;
  bool occupancy = false;  // sites by the occupancy rule instead of |D| <= site_eps
  std::unordered_map<Key, std::unique_ptr<Block>, KeyHash> blocks;
  int64_t iterations = 0, swept = 0, pulled = 0, cleared = 0;
};

int off_comp(uint32_t s, int axis) {
  const int32_t raw = (int32_t)((s >> (9 * axis)) & 511u);
  return raw >= 256 ? raw - 512 : raw;
}
uint32_t pack_off(int ox, int oy, int oz) {
  return ((uint32_t)ox & 511u) | (((uint32_t)oy & 511u) << 9) | (((uint32_t)oz & 511u) << 18);
}
int64_t dist2(uint32_t s) {
  const int64_t x = off_comp(s, 0), y = off_comp(s, 1), z = off_comp(s, 2);
  return x * x + y * y + z * z;
}

// p tries the parent of its neighbour q, which lies at p + (dx, dy, dz).
bool relax(uint32_t& p, uint32_t q, int dx, int dy, int dz, int64_t max2) {
  if (!(p & kObs) || (p & kSite) || !(q & kPar)) return false;
  const int cx = off_comp(q, 0) + dx, cy = off_comp(q, 1) + dy, cz = off_comp(q, 2) + dz;
  const int64_t c2 = (int64_t)cx * cx + (int64_t)cy * cy + (int64_t)cz * cz;
  if (c2 > max2) return false;
  if ((p & kPar) && c2 >= dist2(p)) return false;
  p = (p & ~kOffMask) | kPar | pack_off(cx, cy, cz);
  return true;
}

inline int lin(int x, int y, int z) { return x + 8 * y + 64 * z; }

// The six in-block sweeps of one block (stage 4a).
bool sweep_block(Block& b, int64_t max2) {
  bool changed = false;
  for (int axis = 0; axis < 3; ++axis)
    for (int dir = 0; dir < 2; ++dir)  // +axis first, then -axis
      for (int a = 0; a < 8; ++a)
        for (int c = 0; c < 8; ++c)
          for (int k = 1; k < 8; ++k) {
            const int i = dir == 0 ? k : 7 - k;       // position along the axis
            const int j = dir == 0 ? i - 1 : i + 1;  // the voxel before it in this sweep
            int pi[3], pj[3];
            // the two other axes take the coordinates (a, c) in increasing axis order
            const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
            pi[axis] = i;
            pj[axis] = j;
            pi[o1] = pj[o1] = a;
            pi[o2] = pj[o2] = c;
            int d[3] = {0, 0, 0};
            d[axis] = j - i;
            changed |= relax(b.s[lin(pi[0], pi[1], pi[2])], b.s[lin(pj[0], pj[1], pj[2])], d[0], d[1],
                             d[2], max2);
          }
  return changed;
}

Block* find(Esdf& e, const Key& k) {
  auto it = e.blocks.find(k);
  return it == e.blocks.end() ? nullptr : it->second.get();
}

// Voxel state at global voxel index g, or nullptr if its block does not exist.
const uint32_t* voxel_at(Esdf& e, int64_t gx, int64_t gy, int64_t gz) {
  auto fl = [](int64_t a) { return a >= 0 ? a / 8 : -((-a + 7) / 8); };
  const Key k{fl(gx), fl(gy), fl(gz)};
  Block* b = find(e, k);
  if (!b) return nullptr;
  return &b->s[lin((int)(gx - 8 * k.x), (int)(gy - 8 * k.y), (int)(gz - 8 * k.z))];
}

}  // namespace

extern "C" {

void* esdf_orc_create(float voxel_size, float site_eps, float min_weight, int32_t max_dist_vox) {
  if (!(voxel_size > 0.0f) || !(site_eps >= 0.0f) || max_dist_vox < 1 || max_dist_vox > 255) return nullptr;
  auto* e = new Esdf();
  e->v = voxel_size;
  e->site_eps = site_eps;
  e->min_weight = min_weight;
  e->max_dist = max_dist_vox;
  return e;
}

void esdf_orc_destroy(void* h) { delete static_cast<Esdf*>(h); }

/* Switch to the occupancy site rule (before the first update). */
void esdf_orc_set_occupancy(void* h) { static_cast<Esdf*>(h)->occupancy = true; }

/*
 * One update.  keys int32 [n][3], D and W float32 [n][512] (voxel x + 8 y +
 * 64 z): the TSDF blocks (or occupancy log-odds in D); changed uint8 [n]:
 * blocks changed since the last update (only their values, and for an
 * occupancy layer their face neighbours' values, are read).  Returns the
 * number of lowering iterations.
 */
int64_t esdf_orc_update(void* h, const int32_t* keys, const float* D, const float* W, int64_t n,
                        const uint8_t* changed) {
  Esdf& e = *static_cast<Esdf*>(h);
  const int64_t max2 = (int64_t)e.max_dist * e.max_dist;
  std::vector<Key> upd_list, clr_list;
  std::unordered_set<Key, KeyHash> upd, clr;
  static const int kFace[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  // blocks to mark: the changed ones, and for an occupancy layer their face
  // neighbours too (a site test reads across the faces)
  std::vector<uint8_t> mark(changed, changed + n);
  std::unordered_map<Key, int64_t, KeyHash> index;
  if (e.occupancy) {
    for (int64_t i = 0; i < n; ++i) index[Key{keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]}] = i;
    for (int64_t i = 0; i < n; ++i) {
      if (!changed[i]) continue;
      for (const auto& f : kFace) {
        auto it = index.find(Key{keys[3 * i] + f[0], keys[3 * i + 1] + f[1], keys[3 * i + 2] + f[2]});
        if (it != index.end()) mark[it->second] = 1;
      }
    }
  }
  // log-odds of the voxel at global index g (0 = unknown when its block is absent)
  auto occ_at = [&](int64_t gx, int64_t gy, int64_t gz) -> float {
    auto fl = [](int64_t a) { return a >= 0 ? a / 8 : -((-a + 7) / 8); };
    const Key k{fl(gx), fl(gy), fl(gz)};
    auto it = index.find(k);
    if (it == index.end()) return 0.0f;
    return D[512 * it->second + lin((int)(gx - 8 * k.x), (int)(gy - 8 * k.y), (int)(gz - 8 * k.z))];
  };
  // 1-2. allocate and mark sites in the changed blocks
  for (int64_t i = 0; i < n; ++i) {
    if (!mark[i]) continue;
    const Key k{keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]};
    auto& slot = e.blocks[k];
    if (!slot) {
      slot.reset(new Block());
      std::memset(slot->s, 0, sizeof(slot->s));
    }
    Block& b = *slot;
    bool any = false, lost_site = false;
    for (int l = 0; l < 512; ++l) {
      const float d = D[512 * i + l];
      bool obs, site, inside;
      if (e.occupancy) {
        obs = d != 0.0f;
        inside = d > 0.0f;
        bool free_nbr = false;
        const int64_t gx = 8 * k.x + (l & 7), gy = 8 * k.y + ((l >> 3) & 7), gz = 8 * k.z + (l >> 6);
        for (const auto& f : kFace) free_nbr = free_nbr || occ_at(gx + f[0], gy + f[1], gz + f[2]) < 0.0f;
        site = inside && free_nbr;
      } else {
        const float w = W[512 * i + l];
        obs = w >= e.min_weight;
        site = obs && std::fabs(d) <= e.site_eps;
        inside = obs && d < 0.0f;
      }
      const uint32_t old = b.s[l];
      uint32_t s = old;
      if (site) {
        s = kObs | kSite | kPar | (inside ? kInside : 0u);
      } else if (old & kSite) {
        s = obs ? (kObs | (inside ? kInside : 0u)) : 0u;
        lost_site = true;
      } else if (!obs) {
        s = 0u;
      } else if (!(old & kObs) || ((old & kInside) != 0) != inside) {
        s = kObs | (inside ? kInside : 0u);
      }
      if (s != old) any = true;
      b.s[l] = s;
    }
    if (any && upd.insert(k).second) upd_list.push_back(k);
    if (lost_site && clr.insert(k).second) clr_list.push_back(k);
  }
  // 3. clear invalid: voxels near the cleared blocks whose parent is no longer a site
  if (!clr_list.empty()) {
    const int64_t R = (e.max_dist + 7) / 8 + 1;
    for (auto& kv : e.blocks) {
      const Key& k = kv.first;
      bool near = false;
      for (const Key& c : clr_list)
        if (std::llabs(k.x - c.x) <= R && std::llabs(k.y - c.y) <= R && std::llabs(k.z - c.z) <= R) {
          near = true;
          break;
        }
      if (!near) continue;
      Block& b = *kv.second;
      bool any = false;
      for (int l = 0; l < 512; ++l) {
        const uint32_t s = b.s[l];
        if (!(s & kPar) || (s & kSite)) continue;
        const int64_t gx = 8 * k.x + (l & 7) + off_comp(s, 0);
        const int64_t gy = 8 * k.y + ((l >> 3) & 7) + off_comp(s, 1);
        const int64_t gz = 8 * k.z + (l >> 6) + off_comp(s, 2);
        const uint32_t* par = voxel_at(e, gx, gy, gz);
        if (!par || !(*par & kSite)) {
          b.s[l] = s & ~(kPar | kOffMask);
          ++e.cleared;
          any = true;
        }
      }
      if (any && upd.insert(k).second) upd_list.push_back(k);
    }
  }
  // 4. lower until no block changes
  int64_t iters = 0;
  std::vector<Key> S = upd_list;
  while (!S.empty()) {
    ++iters;
    for (const Key& k : S) sweep_block(*find(e, k), max2);
    e.swept += (int64_t)S.size();
    // T = S and its existing face neighbours
    std::vector<Key> T;
    std::unordered_set<Key, KeyHash> inT;
    for (const Key& k : S) {
      if (inT.insert(k).second) T.push_back(k);
      for (const auto& f : kFace) {
        const Key nk{k.x + f[0], k.y + f[1], k.z + f[2]};
        if (find(e, nk) && inT.insert(nk).second) T.push_back(nk);
      }
    }
    e.pulled += (int64_t)T.size();
    // pull across faces from the neighbours as they are now (Jacobi)
    std::vector<std::pair<Key, Block>> staged;
    for (const Key& k : T) {
      Block nb = *find(e, k);
      bool any = false;
      for (int fi = 0; fi < 6; ++fi) {
        const int* f = kFace[fi];
        const Block* other = find(e, Key{k.x + f[0], k.y + f[1], k.z + f[2]});
        if (!other) continue;
        const int axis = f[0] ? 0 : (f[1] ? 1 : 2);
        const int mine = f[axis] < 0 ? 0 : 7, theirs = 7 - mine;
        for (int a = 0; a < 8; ++a)
          for (int c = 0; c < 8; ++c) {
            int p[3], q[3];
            const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
            p[axis] = mine;
            q[axis] = theirs;
            p[o1] = q[o1] = a;
            p[o2] = q[o2] = c;
            any |= relax(nb.s[lin(p[0], p[1], p[2])], other->s[lin(q[0], q[1], q[2])], f[0], f[1],
                         f[2], max2);
          }
      }
      if (any) staged.emplace_back(k, nb);
    }
    S.clear();
    for (auto& kb : staged) {
      *find(e, kb.first) = kb.second;
      S.push_back(kb.first);
    }
  }
  e.iterations += iters;
  return iters;
}

int64_t esdf_orc_num_blocks(void* h) { return (int64_t)static_cast<Esdf*>(h)->blocks.size(); }

/* Blocks sorted by (x, y, z): keys int32 [n][3], states uint32 [n][512]. */
int64_t esdf_orc_export(void* h, int32_t* keys, uint32_t* states, int64_t cap) {
  Esdf& e = *static_cast<Esdf*>(h);
  std::vector<Key> ks;
  for (auto& kv : e.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  if ((int64_t)ks.size() > cap) return -1;
  for (size_t i = 0; i < ks.size(); ++i) {
    keys[3 * i] = (int32_t)ks[i].x;
    keys[3 * i + 1] = (int32_t)ks[i].y;
    keys[3 * i + 2] = (int32_t)ks[i].z;
    std::memcpy(states + 512 * i, e.blocks[ks[i]]->s, sizeof(uint32_t) * 512);
  }
  return (int64_t)ks.size();
}

/* out[0] lowering iterations, [1] blocks swept, [2] blocks pulled, [3] voxels cleared (totals). */
void esdf_orc_counters(void* h, int64_t* out) {
  Esdf& e = *static_cast<Esdf*>(h);
  out[0] = e.iterations;
  out[1] = e.swept;
  out[2] = e.pulled;
  out[3] = e.cleared;
}

}  // extern "C"
