/*
 * CPU oracle for meshing a TSDF layer with marching cubes (nvblox Sec. IV-B:
 * updated blocks are meshed with a parallel Marching Cubes, after Lorensen
 * and Cline) — TEST INFRASTRUCTURE ONLY.  Loaded by the tests through
 * ctypes; shares no code with the CUDA library.
 *
 * A cube joins the voxel centres g .. g + (1, 1, 1) (global voxel
 * indices); it belongs to the block holding g and is meshed only if all
 * eight corners exist and are observed (W >= min_weight).  Corner c has the
 * offset (c & 1, (c >> 1) & 1, (c >> 2) & 1) and is inside if D < 0.  Every
 * cube edge whose ends differ in inside-ness carries one vertex: on the
 * edge from its lower corner (coordinate 0 along the edge's axis) to its
 * upper corner at t = D_lower / (D_lower - D_upper).
 *
 * The polygons are built face by face, with no case table: on each of the
 * six faces the intersected edges are joined by segments, one segment if the
 * face has two, and for a face with four (two diagonal corners inside) one
 * segment around each inside corner, so that inside corners stay apart.  A
 * segment P -> Q is directed so that an inside corner I of the face it
 * bounds satisfies ((I - P) x (Q - P)) . n > 0, n the face's outward
 * normal (positions of the unit cube, edge midpoints for P and Q).  Every
 * intersected edge then has one outgoing segment; loops start at the
 * smallest unvisited edge number and follow the segments; each loop
 * (e0, e1, ..., ek-1) gives the triangles (e0, ei, ei+1), i = 1 .. k-2,
 * which face the outside (increasing D).  Edge number: 4 * axis + u + 2 w,
 * with u and w the cube coordinates of the edge on the other two axes in
 * increasing axis order.
 *
 * Output per triangle: its cube (global voxel index of corner 0), for each
 * vertex the global index of the edge's lower corner and the edge axis
 * (int32 x 4), and its position in metres (FP64, from the FP32 TSDF values).
 * A loop that crosses a face with four cuts twice can get a fan diagonal
 * lying in that face; the cube across the face may have the same diagonal,
 * so such an edge can have four triangles (the surface touches itself along
 * it) while the loops themselves meet without gaps.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

struct Key {
  int64_t x, y, z;
  bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    return (size_t)(k.x * 73856093LL) ^ (size_t)(k.y * 19349663LL) ^ (size_t)(k.z * 83492791LL);
  }
};

int64_t floordiv8(int64_t a) { return a >= 0 ? a / 8 : -((-a + 7) / 8); }

struct Layer {
  std::unordered_map<Key, int64_t, KeyHash> index;
  const float* D;
  const float* W;
  float min_weight;
  // value at global voxel g; false if its block is absent or it is unobserved
  bool at(int64_t gx, int64_t gy, int64_t gz, float& d) const {
    const Key k{floordiv8(gx), floordiv8(gy), floordiv8(gz)};
    auto it = index.find(k);
    if (it == index.end()) return false;
    const int l = (int)(gx - 8 * k.x) + 8 * (int)(gy - 8 * k.y) + 64 * (int)(gz - 8 * k.z);
    const size_t i = (size_t)it->second * 512 + l;
    if (!(W[i] >= min_weight)) return false;
    d = D[i];
    return true;
  }
};

int corner_bit(int c, int axis) { return (c >> axis) & 1; }

// Edge number of the edge along `axis` whose other coordinates are those of corner c.
int edge_of(int axis, int c) {
  const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
  return 4 * axis + corner_bit(c, o1) + 2 * corner_bit(c, o2);
}

// Lower corner of edge e.
int edge_lower(int e) {
  const int axis = e / 4, u = e & 1, w = (e >> 1) & 1;
  const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
  return (u << o1) | (w << o2);
}

void edge_mid(int e, double p[3]) {
  const int lo = edge_lower(e), axis = e / 4;
  for (int k = 0; k < 3; ++k) p[k] = corner_bit(lo, k);
  p[axis] = 0.5;
}

// Triangles (edge numbers) of one cube with inside mask `in`.
void cube_polygons(int in, std::vector<int>& tris) {
  int next[12];
  for (int& x : next) x = -1;
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) {
      // the face's corners in cyclic order: vary the two other axes
      const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
      int cyc[4];
      const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
      for (int i = 0; i < 4; ++i) cyc[i] = (side << axis) | (uv[i][0] << o1) | (uv[i][1] << o2);
      // face edges between consecutive corners
      int fe[4];
      bool cut[4];
      int ncut = 0;
      for (int i = 0; i < 4; ++i) {
        const int a = cyc[i], b = cyc[(i + 1) & 3];
        const int ax = (a ^ b) == 1 ? 0 : ((a ^ b) == 2 ? 1 : 2);
        fe[i] = edge_of(ax, a);
        cut[i] = ((in >> a) & 1) != ((in >> b) & 1);
        ncut += cut[i];
      }
      if (ncut == 0) continue;
      std::vector<std::pair<std::pair<int, int>, int>> segs;  // (edge, edge), inside corner
      if (ncut == 2) {
        int e[2], k = 0, inside = -1;
        for (int i = 0; i < 4; ++i) {
          if (cut[i]) e[k++] = fe[i];
          if ((in >> cyc[i]) & 1) inside = cyc[i];
        }
        segs.push_back({{e[0], e[1]}, inside});
      } else {  // four cuts: one segment around each inside corner
        for (int i = 0; i < 4; ++i)
          if ((in >> cyc[i]) & 1) segs.push_back({{fe[(i + 3) & 3], fe[i]}, cyc[i]});
      }
      double n[3] = {0, 0, 0};
      n[axis] = side ? 1.0 : -1.0;
      for (auto& sg : segs) {
        int p = sg.first.first, q = sg.first.second;
        double P[3], Q[3], I[3];
        edge_mid(p, P);
        edge_mid(q, Q);
        for (int k = 0; k < 3; ++k) I[k] = corner_bit(sg.second, k);
        const double a[3] = {I[0] - P[0], I[1] - P[1], I[2] - P[2]};
        const double b[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
        const double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        if (cr[0] * n[0] + cr[1] * n[1] + cr[2] * n[2] < 0) std::swap(p, q);
        next[p] = q;
      }
    }
  bool seen[12] = {false};
  for (int s = 0; s < 12; ++s) {
    if (next[s] < 0 || seen[s]) continue;
    std::vector<int> loop;
    for (int e = s; !seen[e]; e = next[e]) {
      seen[e] = true;
      loop.push_back(e);
    }
    for (size_t i = 1; i + 1 < loop.size(); ++i) {
      tris.push_back(loop[0]);
      tris.push_back(loop[i]);
      tris.push_back(loop[i + 1]);
    }
  }
}

}  // namespace

extern "C" {

/*
 * Mesh every cube of the blocks with mesh_it[i] != 0.  keys int32 [n][3],
 * D and W float32 [n][512].  Writes up to cap triangles: tri_cube int32
 * [cap][3], tri_keys int32 [cap][3][4], tri_pos double [cap][3][3]; returns
 * the number of triangles (more than cap means the output was cut).
 */
int64_t mesh_orc_extract(const int32_t* keys, const float* D, const float* W, int64_t n,
                         const uint8_t* mesh_it, float voxel_size, float min_weight,
                         int32_t* tri_cube, int32_t* tri_keys, double* tri_pos, int64_t cap) {
  Layer L;
  L.D = D;
  L.W = W;
  L.min_weight = min_weight;
  for (int64_t i = 0; i < n; ++i) L.index[Key{keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]}] = i;
  const double v = (double)voxel_size;
  std::vector<int> tris;
  int64_t count = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!mesh_it[i]) continue;
    for (int l = 0; l < 512; ++l) {
      const int64_t g[3] = {8 * (int64_t)keys[3 * i] + (l & 7), 8 * (int64_t)keys[3 * i + 1] + ((l >> 3) & 7),
                            8 * (int64_t)keys[3 * i + 2] + (l >> 6)};
      float d[8];
      bool ok = true;
      int in = 0;
      for (int c = 0; c < 8 && ok; ++c) {
        ok = L.at(g[0] + corner_bit(c, 0), g[1] + corner_bit(c, 1), g[2] + corner_bit(c, 2), d[c]);
        if (ok && d[c] < 0.0f) in |= 1 << c;
      }
      if (!ok || in == 0 || in == 255) continue;
      tris.clear();
      cube_polygons(in, tris);
      for (size_t t = 0; t + 2 < tris.size(); t += 3, ++count) {
        if (count >= cap) continue;
        for (int a = 0; a < 3; ++a) tri_cube[3 * count + a] = (int32_t)g[a];
        for (int k = 0; k < 3; ++k) {
          const int e = tris[t + k], axis = e / 4, lo = edge_lower(e), hi = lo | (1 << axis);
          const double dl = d[lo], dh = d[hi];
          const double tt = dl / (dl - dh);
          int32_t* kk = tri_keys + 12 * count + 4 * k;
          double* pp = tri_pos + 9 * count + 3 * k;
          for (int a = 0; a < 3; ++a) {
            kk[a] = (int32_t)(g[a] + corner_bit(lo, a));
            pp[a] = ((double)kk[a] + 0.5 + (a == axis ? tt : 0.0)) * v;
          }
          kk[3] = axis;
        }
      }
    }
  }
  return count;
}

/* The triangles (edge numbers, up to 12 per cube) of inside mask `in`, for
 * tests of the case construction; returns the triangle count. */
int32_t mesh_orc_case(int32_t in, int32_t* edges) {
  std::vector<int> tris;
  if (in > 0 && in < 255) cube_polygons(in, tris);
  for (size_t i = 0; i < tris.size(); ++i) edges[i] = tris[i];
  return (int32_t)(tris.size() / 3);
}

}  // extern "C"
