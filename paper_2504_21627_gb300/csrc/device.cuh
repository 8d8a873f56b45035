// Device helpers shared by the query, fused and training kernels:
// unit-cube mapping, AABB slab test, 3D-DDA over the occupancy grid and the
// hash-grid corner lookup.
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <math_constants.h>

#include "lsnif_impl.h"

namespace lsnif {

struct Ray3 {
  float ox, oy, oz, dx, dy, dz;
};

__device__ __forceinline__ float comp(const float3 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Object space -> unit cube of the AABB: o' = (o - bmin) * inv_ext,
// d' = d * inv_ext; t is unchanged. Returns false for a NaN/inf component or
// an all-zero direction (reported as a miss).
__device__ __forceinline__ bool to_unit(const DevObject &ob, float ox, float oy, float oz, float dx, float dy,
                                        float dz, float3 &o, float3 &d) {
  o = make_float3((ox - ob.bmin[0]) * ob.inv_ext[0], (oy - ob.bmin[1]) * ob.inv_ext[1],
                  (oz - ob.bmin[2]) * ob.inv_ext[2]);
  d = make_float3(dx * ob.inv_ext[0], dy * ob.inv_ext[1], dz * ob.inv_ext[2]);
  bool fin = isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) && isfinite(d.z);
  return fin && !(d.x == 0.f && d.y == 0.f && d.z == 0.f);
}

// Slab test against the unit cube (Fig. 2, first step). On success
// t0 = max(t_near, tmin), t1 = t_far with t1 > t0; entry_axis is the axis of
// t_near when the ray enters through a face at t0, -1 when t0 = tmin lies
// inside the cube.
__device__ __forceinline__ bool unit_slab(const float3 &o, const float3 &d, float tmin, float &t0, float &t1,
                                          int &entry_axis) {
  float tn = -CUDART_INF_F, tf = CUDART_INF_F;
  int an = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float oa = comp(o, a), da = comp(d, a);
    if (da == 0.f) {
      if (oa < 0.f || oa > 1.f) return false;
      continue;
    }
    float ta = (0.f - oa) / da, tb = (1.f - oa) / da;
    float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
    if (lo > tn) { tn = lo; an = a; }
    tf = fminf(tf, hi);
  }
  if (!(tmin == tmin)) return false;  // NaN tmin
  if (tn >= tmin) { t0 = tn; entry_axis = an; } else { t0 = tmin; entry_axis = -1; }
  t1 = tf;
  return t1 > t0;
}

__device__ __forceinline__ bool occupied(const uint32_t *occ, uint32_t vid) {
  return (__ldg(occ + (vid >> 5)) >> (vid & 31)) & 1u;
}

// One occupied-voxel segment found by the DDA.
struct Seg {
  float tin, tout;
  int ain, aout;        // crossed axis at entry (-1: interior start) and exit
  float fin, fout;      // face coordinate (unit cube) on that axis
  uint32_t vid;
};

// Amanatides-Woo 3D-DDA (the traversal Sec. 3.1 cites) over [t0, t1] of a
// unit-cube ray. Calls visit(seg) for every voxel with positive-length
// overlap for which `want(vid)` is true, in increasing t, until visit returns
// false. Crossing times are computed from the plane each step (no
// accumulated increments). Ties between axes step the lowest axis first.
template <class Want, class Visit>
__device__ __forceinline__ void dda_walk(const DevObject &ob, const float3 &o, const float3 &d, float t0, float t1,
                                         int entry_axis, Want want, Visit visit) {
  const int V = ob.V;
  const float invV = ob.invV;
  float3 p = make_float3(fmaf(t0, d.x, o.x), fmaf(t0, d.y, o.y), fmaf(t0, d.z, o.z));
  int ix[3], st[3];
  float inv[3], tn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float da = comp(d, a);
    int c = (int)floorf(comp(p, a) * (float)V);
    c = min(max(c, 0), V - 1);
    if (a == entry_axis) c = da > 0.f ? 0 : V - 1;
    ix[a] = c;
    st[a] = da > 0.f ? 1 : (da < 0.f ? -1 : 0);
    inv[a] = da != 0.f ? 1.f / da : 0.f;
    tn[a] = da != 0.f ? ((float)(c + (st[a] > 0)) * invV - comp(o, a)) * inv[a] : CUDART_INF_F;
  }
  float tcur = t0;
  int ain = entry_axis;
  float fin = entry_axis >= 0 ? (comp(d, entry_axis) > 0.f ? 0.f : 1.f) : 0.f;
  const int max_steps = 3 * V + 3;
  for (int it = 0; it < max_steps; ++it) {
    int a = (tn[0] <= tn[1]) ? (tn[0] <= tn[2] ? 0 : 2) : (tn[1] <= tn[2] ? 1 : 2);
    float tx = fminf(tn[a], t1);
    uint32_t vid = ((uint32_t)ix[2] * V + ix[1]) * V + ix[0];
    if (tx > tcur && want(vid)) {
      Seg s;
      s.tin = tcur;
      s.tout = tx;
      s.ain = ain;
      s.fin = fin;
      s.aout = a;
      s.fout = (float)(ix[a] + (st[a] > 0)) * invV;
      s.vid = vid;
      if (!visit(s)) return;
    }
    if (tn[a] >= t1) return;
    ix[a] += st[a];
    if (ix[a] < 0 || ix[a] >= V) return;
    tcur = tn[a];
    ain = a;
    fin = (float)(ix[a] + (st[a] < 0)) * invV;
    tn[a] = ((float)(ix[a] + (st[a] > 0)) * invV - comp(o, a)) * inv[a];
  }
}

// Boundary point of a segment end: o + t d, with the crossed coordinate set
// to exactly its face value (points lie on voxel faces, Sec. 3.1-3.2).
__device__ __forceinline__ float3 seg_point(const float3 &o, const float3 &d, float t, int axis, float face) {
  float3 p = make_float3(fmaf(t, d.x, o.x), fmaf(t, d.y, o.y), fmaf(t, d.z, o.z));
  if (axis == 0) p.x = face;
  else if (axis == 1) p.y = face;
  else if (axis == 2) p.z = face;
  return p;
}

__device__ __forceinline__ uint32_t hash3(uint32_t x, uint32_t y, uint32_t z) {
  return x ^ (y * kPi2) ^ (z * kPi3);
}

__device__ __forceinline__ float act_fn(float x, int act) {
  return act == 0 ? fmaxf(x, 0.f) : (x > 0.f ? x : 0.01f * x);
}

__device__ __forceinline__ float act_grad(float pre, int act) {
  return act == 0 ? (pre > 0.f ? 1.f : 0.f) : (pre > 0.f ? 1.f : 0.01f);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Read-only 16-byte and 4/8-byte loads through the non-coherent path.
__device__ __forceinline__ uint4 ldg16(const void *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ uint32_t ldg4(const void *p) { return __ldg(reinterpret_cast<const uint32_t *>(p)); }
__device__ __forceinline__ uint2 ldg8(const void *p) { return __ldg(reinterpret_cast<const uint2 *>(p)); }

__device__ __forceinline__ uint32_t pick4(const uint4 &g, uint32_t j) {
  return j == 0 ? g.x : (j == 1 ? g.y : (j == 2 ? g.z : g.w));
}

// Decode of the network outputs (Sec. 5.1, 5.3) for one ray and its stores.
__device__ __forceinline__ void decode_store(const HitsArg &h, int64_t ray, const float *z, int n_out, int n_mat,
                                             float t0, float t1, float tmin, float tmax) {
  bool occ = z[0] > 0.f;
  float t = t0 + sigmoidf_(z[1]) * (t1 - t0);
  float nx = z[2], ny = z[3], nz = z[4];
  float nn = sqrtf(nx * nx + ny * ny + nz * nz);
  if (nn > 0.f) { float r = 1.f / nn; nx *= r; ny *= r; nz *= r; } else { nx = ny = nz = 0.f; }
  int best = 0;
  float bv = z[8];
  for (int m = 1; m < n_mat; ++m)
    if (z[8 + m] > bv) { bv = z[8 + m]; best = m; }
  bool hit = occ && t >= tmin && t <= tmax;
  if (h.hit) h.hit[ray] = hit ? 1 : 0;
  if (h.t) h.t[ray] = t;
  if (h.nx) h.nx[ray] = nx;
  if (h.ny) h.ny[ray] = ny;
  if (h.nz) h.nz[ray] = nz;
  if (h.mat) h.mat[ray] = best;
  if (h.ar) h.ar[ray] = sigmoidf_(z[5]);
  if (h.ag) h.ag[ray] = sigmoidf_(z[6]);
  if (h.ab) h.ab[ray] = sigmoidf_(z[7]);
  if (h.logits)
    for (int j = 0; j < n_out; ++j) h.logits[ray * n_out + j] = z[j];
}

__device__ __forceinline__ void miss_store(const HitsArg &h, int64_t ray, int n_out) {
  if (h.hit) h.hit[ray] = 0;
  if (h.t) h.t[ray] = CUDART_INF_F;
  if (h.nx) h.nx[ray] = 0.f;
  if (h.ny) h.ny[ray] = 0.f;
  if (h.nz) h.nz[ray] = 0.f;
  if (h.mat) h.mat[ray] = -1;
  if (h.ar) h.ar[ray] = 0.f;
  if (h.ag) h.ag[ray] = 0.f;
  if (h.ab) h.ab[ray] = 0.f;
  if (h.logits)
    for (int j = 0; j < n_out; ++j) h.logits[ray * n_out + j] = CUDART_NAN_F;
}

// Resolve a ray's object slot from its handle (-1 when invalid).
__device__ __forceinline__ int slot_of(const DevObject *objs, int n_slots, uint32_t handle) {
  int s = (int)(handle & 0xFFFFu) - 1;
  if (s < 0 || s >= n_slots) return -1;
  if (objs[s].handle != handle || !objs[s].valid) return -1;
  return s;
}

}  // namespace lsnif
