// Bounding volume hierarchy of a triangle mesh, built on the host at load
// time for objects that keep their triangles instead of becoming LSNIF
// objects (the hybrid pipeline of Sec. 4 traces non-LSNIF objects through a
// two-level BVH: the instances' boxes on top, one of these per mesh below).
//
// Binary BVH, binned surface-area heuristic (Wald, "On fast construction of
// SAH-based bounding volume hierarchies", 2007): at each node the triangles'
// centroids are binned along the widest centroid axis and the split with the
// lowest cost C = C_t + (A_l N_l + A_r N_r) / A is taken, against making a
// leaf (cost N). Children are stored next to each other, so an internal node
// needs one child index. Leaves hold at most kMaxLeaf triangles.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "bvh.h"

namespace lsnif {

namespace {

constexpr int kBins = 16;
constexpr int kMaxLeaf = 4;
constexpr float kTraversalCost = 1.0f;  // relative to one triangle test

struct Box {
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  void grow(const float *p) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p[a]);
      hi[a] = std::max(hi[a], p[a]);
    }
  }
  void grow(const Box &b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  float area() const {
    const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    if (!(dx >= 0.f)) return 0.f;
    return 2.f * (dx * dy + dy * dz + dz * dx);
  }
};

}  // namespace

int bvh_build(const float *verts, const int32_t *tris, int64_t nt, std::vector<BvhNode> &nodes,
              std::vector<int32_t> &order) {
  nodes.clear();
  order.resize((size_t)nt);
  if (nt <= 0) return 0;
  std::vector<Box> tbox((size_t)nt);
  std::vector<float> cen(3 * (size_t)nt);
  for (int64_t i = 0; i < nt; ++i) {
    for (int k = 0; k < 3; ++k) tbox[i].grow(verts + 3 * (int64_t)tris[3 * i + k]);
    for (int a = 0; a < 3; ++a) cen[3 * i + a] = 0.5f * (tbox[i].lo[a] + tbox[i].hi[a]);
    order[i] = (int32_t)i;
  }
  struct Task {
    int32_t node, first, count, depth;
  };
  nodes.reserve(2 * (size_t)nt);
  nodes.push_back(BvhNode{});
  std::vector<Task> stack{{0, 0, (int32_t)nt, 0}};
  int max_depth = 0;
  while (!stack.empty()) {
    const Task t = stack.back();
    stack.pop_back();
    max_depth = std::max(max_depth, t.depth);
    Box box, cbox;
    for (int32_t i = t.first; i < t.first + t.count; ++i) {
      box.grow(tbox[order[i]]);
      cbox.grow(&cen[3 * (size_t)order[i]]);
    }
    BvhNode &nd = nodes[t.node];
    for (int a = 0; a < 3; ++a) {
      nd.lo[a] = box.lo[a];
      nd.hi[a] = box.hi[a];
    }
    auto make_leaf = [&]() {
      nodes[t.node].a = t.first;
      nodes[t.node].n = t.count;
    };
    if (t.count <= 1 || t.depth >= kBvhMaxDepth - 1) {
      make_leaf();
      continue;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (cbox.hi[a] - cbox.lo[a] > cbox.hi[axis] - cbox.lo[axis]) axis = a;
    const float clo = cbox.lo[axis], ext = cbox.hi[axis] - cbox.lo[axis];
    int split = -1;  // bins [0, split] go left
    float best = FLT_MAX;
    if (ext > 0.f) {
      Box bb[kBins];
      int cnt[kBins] = {0};
      const float scale = kBins / ext;
      for (int32_t i = t.first; i < t.first + t.count; ++i) {
        int b = (int)((cen[3 * (size_t)order[i] + axis] - clo) * scale);
        b = std::min(std::max(b, 0), kBins - 1);
        cnt[b]++;
        bb[b].grow(tbox[order[i]]);
      }
      float right_area[kBins];
      int right_cnt[kBins];
      Box acc;
      int c = 0;
      for (int b = kBins - 1; b > 0; --b) {
        acc.grow(bb[b]);
        c += cnt[b];
        right_area[b] = acc.area();
        right_cnt[b] = c;
      }
      Box lacc;
      int lc = 0;
      const float inv_area = 1.f / std::max(box.area(), 1e-30f);
      for (int b = 0; b < kBins - 1; ++b) {
        lacc.grow(bb[b]);
        lc += cnt[b];
        if (lc == 0 || right_cnt[b + 1] == 0) continue;
        const float cost = kTraversalCost + (lacc.area() * lc + right_area[b + 1] * right_cnt[b + 1]) * inv_area;
        if (cost < best) {
          best = cost;
          split = b;
        }
      }
    }
    int32_t mid;
    if (split >= 0 && (best < (float)t.count || t.count > kMaxLeaf)) {
      const float scale = kBins / ext;
      int32_t *beg = order.data() + t.first, *end = beg + t.count;
      int32_t *m = std::partition(beg, end, [&](int32_t tri) {
        int b = (int)((cen[3 * (size_t)tri + axis] - clo) * scale);
        b = std::min(std::max(b, 0), kBins - 1);
        return b <= split;
      });
      mid = (int32_t)(m - order.data());
    } else if (t.count > kMaxLeaf) {
      // all centroids coincide along every axis (or no useful split): halve
      // the range in index order
      mid = t.first + t.count / 2;
    } else {
      make_leaf();
      continue;
    }
    const int32_t left = (int32_t)nodes.size();
    nodes.push_back(BvhNode{});
    nodes.push_back(BvhNode{});
    nodes[t.node].a = left;
    nodes[t.node].n = 0;
    stack.push_back({left + 1, mid, t.first + t.count - mid, t.depth + 1});
    stack.push_back({left, t.first, mid - t.first, t.depth + 1});
  }
  return max_depth;
}

}  // namespace lsnif

// Host-only entry point of the builder (no GPU): lets tests check the
// structure's invariants. nodes_out: room for 2 nt - 1 nodes of 8 floats
// (lo xyz, a, hi xyz, n; a and n as int32 bit patterns); order_out: nt.
extern "C" LSNIF_API int lsnif_bvh_build_host(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                              void *nodes_out, int64_t *n_nodes, int32_t *order_out,
                                              int32_t *depth) {
  if (!verts || !tris || !nodes_out || !n_nodes || !order_out || nv <= 0 || nt <= 0) return LSNIF_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (tris[i] < 0 || tris[i] >= nv) return LSNIF_ERR_INVALID_ARG;
  std::vector<lsnif::BvhNode> nodes;
  std::vector<int32_t> order;
  const int d = lsnif::bvh_build(verts, tris, nt, nodes, order);
  memcpy(nodes_out, nodes.data(), nodes.size() * sizeof(lsnif::BvhNode));
  memcpy(order_out, order.data(), order.size() * 4);
  *n_nodes = (int64_t)nodes.size();
  if (depth) *depth = d;
  return LSNIF_OK;
}
