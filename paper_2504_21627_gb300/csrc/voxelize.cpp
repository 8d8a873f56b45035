// Host-side object geometry: the AABB of the mesh and its surface-only
// binary voxelization (Sec. 3.1), plus per-voxel triangle lists used by the
// training-label ray caster.
//
// Occupancy is decided by the separating-axis triangle/box test of
// Akenine-Moller ("Fast 3D Triangle-Box Overlap Testing", JGT 2001) in FP64,
// against the CLOSED voxel box: a triangle that only touches a box face, edge
// or corner still occupies it. Grid coordinates are
//   g = ((v - bmin) * V) / (bmax - bmin)
// so voxel (i,j,k) spans [i,i+1] x [j,j+1] x [k,k+1].
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace lsnif {

void mesh_bbox(const float *verts, int64_t nv, float bmin[3], float bmax[3]) {
  double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
  for (int64_t v = 0; v < nv; ++v) {
    for (int a = 0; a < 3; ++a) {
      const double x = verts[3 * v + a];
      lo[a] = std::min(lo[a], x);
      hi[a] = std::max(hi[a], x);
    }
  }
  double d2 = 0;
  for (int a = 0; a < 3; ++a) d2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  // An axis thinner than 1/8 of the diagonal is widened to that: the unit-cube
  // map scales an axis by 1/extent, so a thinner axis would magnify the FP32
  // rounding of ray origins along it into a large part of a voxel.
  double thin = std::sqrt(d2) / 8.0;
  if (thin == 0.0) thin = 1e-6;
  for (int a = 0; a < 3; ++a) {
    if (hi[a] - lo[a] < thin) {  // widen a flat or thin axis symmetrically
      const double mid = 0.5 * (lo[a] + hi[a]);
      lo[a] = mid - 0.5 * thin;
      hi[a] = mid + 0.5 * thin;
    }
    float l = (float)lo[a], h = (float)hi[a];  // round outward to FP32
    if ((double)l > lo[a]) l = std::nextafter(l, -HUGE_VALF);
    if ((double)h < hi[a]) h = std::nextafter(h, HUGE_VALF);
    bmin[a] = l;
    bmax[a] = h;
  }
}

namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double el(V3 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

// Triangle (a,b,c) relative to the box centre vs the closed cube of
// half-extent h. Axes: the 3 box normals, the triangle normal, and the 9
// cross products of box axes with triangle edges.
bool overlaps(V3 a, V3 b, V3 c, double h) {
  // box normals: compare the triangle's extent per axis with [-h, h]
  for (int i = 0; i < 3; ++i) {
    const double lo = std::min(el(a, i), std::min(el(b, i), el(c, i)));
    const double hi = std::max(el(a, i), std::max(el(b, i), el(c, i)));
    if (lo > h || hi < -h) return false;
  }
  const V3 edges[3] = {sub(b, a), sub(c, b), sub(a, c)};
  const V3 unit[3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (const V3 &e : edges) {
    for (const V3 &u : unit) {
      const V3 ax = cross(u, e);
      const double pa = dot(ax, a), pb = dot(ax, b), pc = dot(ax, c);
      const double r = h * (std::fabs(ax.x) + std::fabs(ax.y) + std::fabs(ax.z));
      if (std::min(pa, std::min(pb, pc)) > r) return false;
      if (std::max(pa, std::max(pb, pc)) < -r) return false;
    }
  }
  // triangle plane n.x = n.a against the box: the box's extent along n is
  // [-h*sum|n_i|, h*sum|n_i|]
  const V3 n = cross(edges[0], edges[1]);
  const double d = dot(n, a);
  const double r = h * (std::fabs(n.x) + std::fabs(n.y) + std::fabs(n.z));
  return !(d > r || d < -r);
}

}  // namespace

// occ: ceil(V^3/32) words, bit i of word i>>5 = voxel i = (z*V + y)*V + x.
// When pairs != nullptr, every (voxel, triangle) overlap is appended.
void voxelize_mesh(const float *verts, const int32_t *tris, int64_t nt, const float bmin[3], const float bmax[3],
                   int V, uint32_t *occ, std::vector<std::pair<int32_t, int32_t>> *pairs) {
  const size_t nvox = (size_t)V * V * V;
  std::memset(occ, 0, sizeof(uint32_t) * ((nvox + 31) / 32));
  for (int64_t t = 0; t < nt; ++t) {
    V3 g[3];
    for (int c = 0; c < 3; ++c) {
      const float *p = verts + 3 * (int64_t)tris[3 * t + c];
      double q[3];
      for (int a = 0; a < 3; ++a)
        q[a] = (((double)p[a] - (double)bmin[a]) * (double)V) / ((double)bmax[a] - (double)bmin[a]);
      g[c] = {q[0], q[1], q[2]};
    }
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      const double mn = std::min(el(g[0], a), std::min(el(g[1], a), el(g[2], a)));
      const double mx = std::max(el(g[0], a), std::max(el(g[1], a), el(g[2], a)));
      lo[a] = std::max(0, (int)std::ceil(mn) - 1);
      hi[a] = std::min(V - 1, (int)std::floor(mx));
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const V3 ctr = {x + 0.5, y + 0.5, z + 0.5};
          if (!overlaps(sub(g[0], ctr), sub(g[1], ctr), sub(g[2], ctr), 0.5)) continue;
          const size_t id = ((size_t)z * V + y) * V + x;
          occ[id >> 5] |= 1u << (id & 31);
          if (pairs) pairs->push_back({(int32_t)id, (int32_t)t});
        }
  }
}

// Geometric progression of lattice resolutions from N_min to N_max (Sec.
// 3.2, as in instant-NGP), rounded half up.
void level_resolutions(int N_min, int N_max, int L, int32_t *out) {
  if (L == 1) {
    out[0] = N_min;
    return;
  }
  const double growth = std::exp((std::log((double)N_max) - std::log((double)N_min)) / (double)(L - 1));
  for (int l = 0; l < L; ++l) out[l] = (int32_t)std::floor((double)N_min * std::pow(growth, (double)l) + 0.5);
}

}  // namespace lsnif
