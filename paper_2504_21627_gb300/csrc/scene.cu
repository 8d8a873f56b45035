// Instanced scenes (the wavefront integration of Sec. 4 over the instancing
// of Sec. 6) and next-bounce rays.
//
// lsnif_query_scene: every (ray, instance) pair whose ray, mapped into the
// instance's object frame, crosses the object's box becomes one ray of an
// ordinary multi-object query (so the pairs of all instances are grouped by
// object and share one launch sequence); a per-ray pass then keeps the
// nearest hit. Pair generation: count per ray, exclusive scan, emit; the
// pairs of a ray are contiguous and in instance order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device.cuh"
#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

namespace {

struct DevInstance {
  int32_t slot;
  uint32_t handle;
  float A[9];  // world -> object, row-major
  float b[3];
};

__device__ __forceinline__ void to_object(const DevInstance &in, float ox, float oy, float oz, float dx, float dy,
                                          float dz, float *o, float *d) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    o[r] = fmaf(in.A[3 * r], ox, fmaf(in.A[3 * r + 1], oy, fmaf(in.A[3 * r + 2], oz, in.b[r])));
    d[r] = fmaf(in.A[3 * r], dx, fmaf(in.A[3 * r + 1], dy, in.A[3 * r + 2] * dz));
  }
}

// the query's own box test (a1-a2) on the mapped ray
__device__ __forceinline__ bool crosses_box(const DevObject &ob, const float *o, const float *d, float tmin) {
  float3 uo, ud;
  float t0, t1;
  int ea;
  return to_unit(ob, o[0], o[1], o[2], d[0], d[1], d[2], uo, ud) && unit_slab(uo, ud, tmin, t0, t1, ea);
}

__global__ void scene_count_kernel(RaysArg r, const DevInstance *inst, int n_inst, const DevObject *objs,
                                   int32_t *count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r.n) return;
  const float ox = r.ox[i], oy = r.oy[i], oz = r.oz[i], dx = r.dx[i], dy = r.dy[i], dz = r.dz[i], tmin = r.tmin[i];
  int c = 0;
  for (int k = 0; k < n_inst; ++k) {
    float o[3], d[3];
    to_object(inst[k], ox, oy, oz, dx, dy, dz, o, d);
    c += crosses_box(objs[inst[k].slot], o, d, tmin);
  }
  count[i] = c;
}

struct PairOut {
  float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
  uint32_t *obj;
  int32_t *ray, *inst;
};

__global__ void scene_emit_kernel(RaysArg r, const DevInstance *inst, int n_inst, const DevObject *objs,
                                  const int32_t *offset, PairOut p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r.n) return;
  const float ox = r.ox[i], oy = r.oy[i], oz = r.oz[i], dx = r.dx[i], dy = r.dy[i], dz = r.dz[i];
  const float tmin = r.tmin[i], tmax = r.tmax[i];
  int64_t q = offset[i];
  for (int k = 0; k < n_inst; ++k) {
    float o[3], d[3];
    to_object(inst[k], ox, oy, oz, dx, dy, dz, o, d);
    if (!crosses_box(objs[inst[k].slot], o, d, tmin)) continue;
    p.ox[q] = o[0]; p.oy[q] = o[1]; p.oz[q] = o[2];
    p.dx[q] = d[0]; p.dy[q] = d[1]; p.dz[q] = d[2];
    p.tmin[q] = tmin; p.tmax[q] = tmax;
    p.obj[q] = inst[k].handle;
    p.ray[q] = (int32_t)i;
    p.inst[q] = k;
    ++q;
  }
}

// nearest hit over a ray's pairs; world normal A^T n
__global__ void scene_resolve_kernel(int64_t n, const int32_t *offset, const int32_t *count, const int32_t *pinst,
                                     const DevInstance *inst, HitsArg ph, HitsArg h, int32_t *inst_hit) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = offset[i], e = b + count[i];
  int64_t best = -1;
  float bt = CUDART_INF_F;
  for (int64_t q = b; q < e; ++q)
    if (ph.hit[q] && ph.t[q] < bt) {
      bt = ph.t[q];
      best = q;
    }
  if (best < 0) {
    miss_store(h, i, 0);
    if (inst_hit) inst_hit[i] = -1;
    return;
  }
  const DevInstance &in = inst[pinst[best]];
  const float nl[3] = {ph.nx[best], ph.ny[best], ph.nz[best]};
  float nw[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) nw[c] = fmaf(in.A[c], nl[0], fmaf(in.A[3 + c], nl[1], in.A[6 + c] * nl[2]));
  const float ln = sqrtf(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
  const float s = ln > 0.f ? 1.f / ln : 0.f;
  if (h.hit) h.hit[i] = 1;
  if (h.t) h.t[i] = bt;
  if (h.nx) h.nx[i] = nw[0] * s;
  if (h.ny) h.ny[i] = nw[1] * s;
  if (h.nz) h.nz[i] = nw[2] * s;
  if (h.mat) h.mat[i] = ph.mat[best];
  if (h.ar) h.ar[i] = ph.ar[best];
  if (h.ag) h.ag[i] = ph.ag[best];
  if (h.ab) h.ab[i] = ph.ab[best];
  if (inst_hit) inst_hit[i] = pinst[best];
}

// orthonormal basis about unit n (Duff et al. 2017, "Building an Orthonormal
// Basis, Revisited")
__device__ __forceinline__ void onb(const float *n, float *t, float *b) {
  const float s = n[2] >= 0.f ? 1.f : -1.f;
  const float a = -1.f / (s + n[2]);
  const float bb = n[0] * n[1] * a;
  t[0] = 1.f + s * n[0] * n[0] * a;
  t[1] = s * bb;
  t[2] = -s * n[0];
  b[0] = bb;
  b[1] = s + n[1] * n[1] * a;
  b[2] = -n[1];
}

__global__ void bounce_kernel(RaysArg r, const uint8_t *hit, const float *t, const float *nx, const float *ny,
                              const float *nz, const float *u, float eps, float *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = r.n;
  if (i >= n) return;
  float nn[3] = {nx[i], ny[i], nz[i]};
  const float ln = sqrtf(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
  float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
  if (hit[i] && ln > 0.f) {
    const float inv = 1.f / ln;
    const float rd[3] = {r.dx[i], r.dy[i], r.dz[i]};
#pragma unroll
    for (int c = 0; c < 3; ++c) nn[c] *= inv;
    const float facing = (nn[0] * rd[0] + nn[1] * rd[1] + nn[2] * rd[2]) > 0.f ? -1.f : 1.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) nn[c] *= facing;
    const float th = t[i];
    o[0] = fmaf(th, rd[0], r.ox[i]) + eps * nn[0];
    o[1] = fmaf(th, rd[1], r.oy[i]) + eps * nn[1];
    o[2] = fmaf(th, rd[2], r.oz[i]) + eps * nn[2];
    const float u0 = u[2 * i], u1 = u[2 * i + 1];
    const float rr = sqrtf(u0), ph = 6.283185307179586f * u1;
    float sp, cp;
    sincosf(ph, &sp, &cp);
    const float x = rr * cp, y = rr * sp, z = sqrtf(fmaxf(0.f, 1.f - u0));
    float tb[3], bb[3];
    onb(nn, tb, bb);
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = x * tb[c] + y * bb[c] + z * nn[c];
  }
  out[i] = o[0];
  out[n + i] = o[1];
  out[2 * n + i] = o[2];
  out[3 * n + i] = d[0];
  out[4 * n + i] = d[1];
  out[5 * n + i] = d[2];
  out[6 * n + i] = 0.f;
  out[7 * n + i] = CUDART_INF_F;
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int lsnif_query_scene(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_instance *inst, int n_inst,
                                 lsnif_hits *hits, int32_t *inst_hit, int precision, void *stream) {
  if (!ctx || !rays || !inst || !hits) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: NULL argument");
  if (n_inst < 1) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: n_inst < 1");
  if (hits->logits) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: logits are not supported");
  if (rays->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: n < 0");
  if (!valid_precision(precision)) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: unknown precision %d", precision);
  if (rays->n == 0) return LSNIF_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz || !rays->tmin || !rays->tmax)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: every ray array must be given");
  std::vector<DevInstance> hin(n_inst);
  for (int k = 0; k < n_inst; ++k) {
    Object *o = find_object(ctx, inst[k].obj);
    if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_query_scene: instance %d names unknown object %u", k, inst[k].obj);
    const float *m = inst[k].world_to_obj;
    const double det = (double)m[0] * ((double)m[5] * m[10] - (double)m[6] * m[9]) -
                       (double)m[1] * ((double)m[4] * m[10] - (double)m[6] * m[8]) +
                       (double)m[2] * ((double)m[4] * m[9] - (double)m[5] * m[8]);
    if (!(std::fabs(det) > 1e-30) || !std::isfinite(det))
      return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_scene: instance %d has a singular transform", k);
    hin[k].slot = o->slot;
    hin[k].handle = o->handle;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) hin[k].A[3 * r + c] = m[4 * r + c];
      hin[k].b[r] = m[4 * r + 3];
    }
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = rays->n;
  const int64_t nb = (n + 1023) / 1024;
  // scene scratch: instances, per-ray counts and offsets, block sums
  const size_t head = al(sizeof(DevInstance) * n_inst) + 2 * al((size_t)n * 4) + al((size_t)(nb + 1) * 4);
  if (ctx->scene_bytes < head) {
    if (ctx->scene_buf) {
      cudaDeviceSynchronize();
      dev_free(ctx, ctx->scene_buf);
      ctx->scene_buf = nullptr;
      ctx->scene_bytes = 0;
    }
    int rc = dev_alloc(ctx, head, &ctx->scene_buf, "scene scratch");
    if (rc) return rc;
    ctx->scene_bytes = head;
  }
  uint8_t *p = reinterpret_cast<uint8_t *>(ctx->scene_buf);
  DevInstance *dinst = reinterpret_cast<DevInstance *>(p);
  p += al(sizeof(DevInstance) * n_inst);
  int32_t *count = reinterpret_cast<int32_t *>(p);
  p += al((size_t)n * 4);
  int32_t *offset = reinterpret_cast<int32_t *>(p);
  p += al((size_t)n * 4);
  int32_t *sums = reinterpret_cast<int32_t *>(p);

  cudaError_t e = cudaMemcpyAsync(dinst, hin.data(), sizeof(DevInstance) * n_inst, cudaMemcpyHostToDevice, st);
  RaysArg ra{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax, nullptr, 0, n};
  const int grid = (int)((n + 255) / 256);
  if (e == cudaSuccess) {
    scene_count_kernel<<<grid, 256, 0, st>>>(ra, dinst, n_inst, ctx->d_objs, count);
    e = cudaMemcpyAsync(offset, count, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) {
    e = launch_exclusive_scan(offset, n, sums, st);
  }
  int32_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, sums + nb, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_query_scene: pair count");

  // pair rays and their results
  const int64_t np = std::max<int64_t>(total, 1);
  const size_t pair_bytes = 11 * al((size_t)np * 4) + al((size_t)np) + 8 * al((size_t)np * 4);
  if (ctx->pair_bytes < pair_bytes) {
    if (ctx->pair_buf) {
      cudaDeviceSynchronize();
      dev_free(ctx, ctx->pair_buf);
      ctx->pair_buf = nullptr;
      ctx->pair_bytes = 0;
    }
    int rc = dev_alloc(ctx, pair_bytes, &ctx->pair_buf, "scene pairs");
    if (rc) return rc;
    ctx->pair_bytes = pair_bytes;
  }
  uint8_t *q = reinterpret_cast<uint8_t *>(ctx->pair_buf);
  auto take = [&](size_t bytes) {
    uint8_t *r = q;
    q += al(bytes);
    return r;
  };
  PairOut po;
  float **pf[8] = {&po.ox, &po.oy, &po.oz, &po.dx, &po.dy, &po.dz, &po.tmin, &po.tmax};
  for (auto f : pf) *f = reinterpret_cast<float *>(take((size_t)np * 4));
  po.obj = reinterpret_cast<uint32_t *>(take((size_t)np * 4));
  po.ray = reinterpret_cast<int32_t *>(take((size_t)np * 4));
  po.inst = reinterpret_cast<int32_t *>(take((size_t)np * 4));
  lsnif_hits ph{};
  ph.hit = take((size_t)np);
  ph.t = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.nx = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.ny = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.nz = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.mat = reinterpret_cast<int32_t *>(take((size_t)np * 4));
  ph.ar = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.ag = reinterpret_cast<float *>(take((size_t)np * 4));
  ph.ab = reinterpret_cast<float *>(take((size_t)np * 4));
  if (total > 0) {
    scene_emit_kernel<<<grid, 256, 0, st>>>(ra, dinst, n_inst, ctx->d_objs, offset, po);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "lsnif_query_scene: emit");
    lsnif_rays pr{};
    pr.ox = po.ox; pr.oy = po.oy; pr.oz = po.oz;
    pr.dx = po.dx; pr.dy = po.dy; pr.dz = po.dz;
    pr.tmin = po.tmin; pr.tmax = po.tmax;
    pr.obj = po.obj;
    pr.n = total;
    int rc = run_query(ctx, &ctx->ws, &pr, &ph, precision, st, false);
    if (rc) return rc;
  }
  HitsArg hp{ph.hit, ph.t, ph.nx, ph.ny, ph.nz, ph.mat, ph.ar, ph.ag, ph.ab, nullptr};
  HitsArg hh{hits->hit, hits->t, hits->nx, hits->ny, hits->nz, hits->mat, hits->ar, hits->ag, hits->ab, nullptr};
  scene_resolve_kernel<<<grid, 256, 0, st>>>(n, offset, count, po.inst, dinst, hp, hh, inst_hit);
  e = cudaGetLastError();
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_query_scene: resolve");
}

extern "C" int lsnif_bounce_rays(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_hits *hits, const float *u,
                                 float eps, float *out, void *stream) {
  if (!ctx || !rays || !hits || !u || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_bounce_rays: NULL argument");
  if (rays->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_bounce_rays: n < 0");
  if (rays->n == 0) return LSNIF_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_bounce_rays: every ray origin and direction array must be given");
  if (!hits->hit || !hits->t || !hits->nx || !hits->ny || !hits->nz)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_bounce_rays: hits need hit, t and the normal");
  cudaSetDevice(ctx->device);
  RaysArg ra{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax, nullptr, 0, rays->n};
  bounce_kernel<<<(unsigned)((rays->n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      ra, hits->hit, hits->t, hits->nx, hits->ny, hits->nz, u, eps, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_bounce_rays");
}
