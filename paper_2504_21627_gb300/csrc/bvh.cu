// Exact ray queries of mesh objects through their BVH (the hybrid pipeline of
// Sec. 4: objects that are not replaced by LSNIF keep their triangles and
// are intersected through a BVH; the instances' boxes are the top level).
//
// One thread per ray: ordered depth-first traversal with a short stack (the
// nearer child first, the farther pushed with its entry distance and skipped
// on pop once a closer hit exists), Moller-Trumbore on the stored (v0, e1,
// e2) in FP32, closed triangles, tmin <= t <= tmax. Equal distances keep the
// lowest mesh triangle index, as a brute-force loop in index order does.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "bvh.h"
#include "device.cuh"
#include "lsnif_impl.h"

#include <algorithm>

namespace lsnif {

namespace {

struct MeshHit {
  float t, u, v;
  int32_t tri;
};

__device__ __forceinline__ bool box_enter(const float4 &lo, const float4 &hi, const float o[3], const float id[3],
                                          float tmin, float tmax, float &tnear) {
  const float x0 = (lo.x - o[0]) * id[0], x1 = (hi.x - o[0]) * id[0];
  const float y0 = (lo.y - o[1]) * id[1], y1 = (hi.y - o[1]) * id[1];
  const float z0 = (lo.z - o[2]) * id[2], z1 = (hi.z - o[2]) * id[2];
  const float tn = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
  const float tf = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), tmax));
  tnear = tn;
  // the far distance widened by 2 gamma_3 (Ize, "Robust BVH ray traversal",
  // 2013) so that FP32 rounding of the slab distances cannot drop a box
  // that the ray touches
  return tn <= tf * 1.0000004f;
}

__device__ __forceinline__ bool mt(const float4 &v0, const float4 &e1, const float4 &e2, const float o[3],
                                   const float d[3], float &t, float &u, float &v) {
  const float p0 = d[1] * e2.z - d[2] * e2.y, p1 = d[2] * e2.x - d[0] * e2.z, p2 = d[0] * e2.y - d[1] * e2.x;
  const float det = e1.x * p0 + e1.y * p1 + e1.z * p2;
  if (det == 0.f) return false;
  const float inv = 1.f / det;
  const float s0 = o[0] - v0.x, s1 = o[1] - v0.y, s2 = o[2] - v0.z;
  u = (s0 * p0 + s1 * p1 + s2 * p2) * inv;
  if (u < 0.f || u > 1.f) return false;
  const float q0 = s1 * e1.z - s2 * e1.y, q1 = s2 * e1.x - s0 * e1.z, q2 = s0 * e1.y - s1 * e1.x;
  v = (d[0] * q0 + d[1] * q1 + d[2] * q2) * inv;
  if (v < 0.f || u + v > 1.f) return false;
  t = (e2.x * q0 + e2.y * q1 + e2.z * q2) * inv;
  return true;
}

__device__ MeshHit bvh_closest(const DevObject &ob, const float o[3], const float d[3], float tmin, float tmax) {
  MeshHit best{CUDART_INF_F, 0.f, 0.f, -1};
  const float id[3] = {1.f / d[0], 1.f / d[1], 1.f / d[2]};
  float limit = tmax;
  int32_t stack[kBvhMaxDepth];
  float stack_t[kBvhMaxDepth];
  int sp = 0;
  float tn;
  if (!box_enter(ob.bvh_nodes[0], ob.bvh_nodes[1], o, id, tmin, limit, tn)) return best;
  int32_t node = 0;
  while (true) {
    const float4 lo = ob.bvh_nodes[2 * node], hi = ob.bvh_nodes[2 * node + 1];
    const int32_t a = __float_as_int(lo.w), n = __float_as_int(hi.w);
    bool descend = false;
    if (n == 0) {
      float t0, t1;
      const bool h0 = box_enter(ob.bvh_nodes[2 * a], ob.bvh_nodes[2 * a + 1], o, id, tmin, limit, t0);
      const bool h1 = box_enter(ob.bvh_nodes[2 * a + 2], ob.bvh_nodes[2 * a + 3], o, id, tmin, limit, t1);
      if (h0 && h1) {
        const bool first0 = t0 <= t1;
        if (sp < kBvhMaxDepth) {
          stack[sp] = first0 ? a + 1 : a;
          stack_t[sp] = first0 ? t1 : t0;
          ++sp;
        }
        node = first0 ? a : a + 1;
        descend = true;
      } else if (h0 || h1) {
        node = h0 ? a : a + 1;
        descend = true;
      }
    } else {
      for (int32_t i = a; i < a + n; ++i) {
        float t, u, v;
        if (mt(ob.bvh_tris[3 * i], ob.bvh_tris[3 * i + 1], ob.bvh_tris[3 * i + 2], o, d, t, u, v) && t >= tmin &&
            t <= limit) {
          const int32_t tri = ob.bvh_order[i];
          if (t < best.t || tri < best.tri) {  // t <= limit = best.t once a hit exists
            best = MeshHit{t, u, v, tri};
            limit = t;
          }
        }
      }
    }
    if (descend) continue;
    // pop the next subtree that can still hold a hit at or before `limit`
    bool found = false;
    while (sp > 0) {
      --sp;
      if (stack_t[sp] <= limit) {
        node = stack[sp];
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  return best;
}

__global__ void mesh_query_kernel(QueryLaunch q) {
  const int64_t n = q.rays.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = q.rays.obj ? q.rays.obj[i] : q.rays.single_handle;
    const int s = slot_of(q.objs, q.n_slots, h);
    if (s < 0) continue;  // reported and answered as a miss by the traversal
    const DevObject &ob = q.objs[s];
    if (ob.kind != 1) continue;
    const float o[3] = {q.rays.ox[i], q.rays.oy[i], q.rays.oz[i]};
    const float d[3] = {q.rays.dx[i], q.rays.dy[i], q.rays.dz[i]};
    const MeshHit m = bvh_closest(ob, o, d, q.rays.tmin[i], q.rays.tmax[i]);
    if (m.tri < 0) {
      miss_store(q.hits, i, 0);
      continue;
    }
    const HitsArg &H = q.hits;
    if (H.hit) H.hit[i] = 1;
    if (H.t) H.t[i] = m.t;
    const int32_t *ix = ob.tris + 3 * (int64_t)m.tri;
    const float w0 = 1.f - m.u - m.v;
    float nn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      nn[c] = w0 * ob.vnormals[3 * (int64_t)ix[0] + c] + m.u * ob.vnormals[3 * (int64_t)ix[1] + c] +
              m.v * ob.vnormals[3 * (int64_t)ix[2] + c];
    const float ln = sqrtf(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    const float inv = ln > 0.f ? 1.f / ln : 0.f;
    if (H.nx) {
      H.nx[i] = nn[0] * inv;
      H.ny[i] = nn[1] * inv;
      H.nz[i] = nn[2] * inv;
    }
    const int32_t mat = ob.tri_mat[m.tri];
    if (H.mat) H.mat[i] = mat;
    if (H.ar) {
      H.ar[i] = ob.albedo[3 * mat];
      H.ag[i] = ob.albedo[3 * mat + 1];
      H.ab[i] = ob.albedo[3 * mat + 2];
    }
  }
}

}  // namespace

cudaError_t launch_mesh_query(const QueryLaunch &q, int *launches) {
  if (q.rays.n == 0) return cudaSuccess;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>((q.rays.n + 127) / 128, (int64_t)sms * 16);
  mesh_query_kernel<<<grid, 128, 0, q.stream>>>(q);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace lsnif
