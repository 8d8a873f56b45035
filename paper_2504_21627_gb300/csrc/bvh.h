// BVH of a triangle mesh (objects that keep their triangles, Sec. 4): node
// layout shared by the host builder and the device traversal.
#pragma once

#include <cstdint>
#include <vector>

#include "lsnif.h"

namespace lsnif {

constexpr int kBvhMaxDepth = 64;  // traversal stack size

// 32 bytes: box, then a = left child (its sibling is a + 1) and n = 0 for an
// internal node, or a = first entry of the triangle order and n = count for
// a leaf
struct BvhNode {
  float lo[3];
  int32_t a;
  float hi[3];
  int32_t n;
};
static_assert(sizeof(BvhNode) == 32, "BvhNode is two float4");

// Build over nt triangles; order[i] = mesh triangle stored at position i.
// Returns the depth of the deepest leaf (root = 0, below kBvhMaxDepth).
int bvh_build(const float *verts, const int32_t *tris, int64_t nt, std::vector<BvhNode> &nodes,
              std::vector<int32_t> &order);

}  // namespace lsnif
