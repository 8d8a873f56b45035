// Primary-ray G-buffer by software rasterisation (the hybrid pipeline of
// Sec. 4, Fig. 4a: primary visibility comes from rasterising the meshes,
// LSNIF answers the later rays). Per pixel: the nearest triangle that the
// ray through the pixel centre hits -- instance, triangle, barycentric (u, v)
// and camera distance.
//
// One thread per (instance, triangle): the triangle goes to world space, is
// projected to find the pixel centres its screen box holds, and each of
// those pixels' rays is tested against it (Moller-Trumbore on the world
// triangle; the parts that do not depend on the pixel are computed once per
// triangle). A hit is merged with a 64-bit atomicMin of (distance bits,
// linear triangle id): non-negative FP32 values order like their bit
// patterns, so the minimum is the nearest hit, and equal distances keep the
// lowest instance, then the lowest triangle. Triangles whose box holds more
// than a few pixel centres, or that cross the camera plane, are queued for a
// second kernel where a whole warp sweeps their pixels. A resolve pass
// re-tests the winning triangle to recover (u, v) and writes the buffers.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

namespace {

constexpr int kSmallPixels = 64;        // larger boxes go to the warp-per-triangle queue
constexpr unsigned long long kEmpty = ~0ull;

struct RInstance {
  int32_t slot;
  uint32_t first;  // linear id of the instance's triangle 0
  uint32_t nt;
  float M[9];      // object -> world linear part (A^-1), row-major
  float c[3];      // object -> world translation (-A^-1 b)
  float A[9];      // world -> object, for normals (A^T n)
};

struct RCam {
  float e[3], f[3], r[3], u[3];
  float tx, ty;  // tan(half fov) * aspect, tan(half fov)
  float rw, rh;  // 2 / width, 2 / height
  int w, h;
};

struct WorldTri {
  float a[3], e1[3], e2[3];
  float s[3];  // eye - a
  float q[3];  // s x e1
  float tq;    // e2 . q
};

__device__ __forceinline__ void pixel_dir(const RCam &cam, int px, int py, float d[3]) {
  const float x = fmaf((float)px + 0.5f, cam.rw, -1.f) * cam.tx;
  const float y = fmaf(-((float)py + 0.5f), cam.rh, 1.f) * cam.ty;
  float n2 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d[k] = cam.f[k] + x * cam.r[k] + y * cam.u[k];
    n2 += d[k] * d[k];
  }
  const float inv = rsqrtf(n2);
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] *= inv;
}

__device__ __forceinline__ void world_vertex(const RInstance &in, const float *v, float out[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) out[r] = fmaf(in.M[3 * r], v[0], fmaf(in.M[3 * r + 1], v[1], fmaf(in.M[3 * r + 2], v[2], in.c[r])));
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

__device__ __forceinline__ void make_tri(const RCam &cam, const float a[3], const float b[3], const float c[3],
                                         WorldTri &T) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T.a[k] = a[k];
    T.e1[k] = b[k] - a[k];
    T.e2[k] = c[k] - a[k];
    T.s[k] = cam.e[k] - a[k];
  }
  cross3(T.s, T.e1, T.q);
  T.tq = dot3(T.e2, T.q);
}

// Moller-Trumbore against the ray eye + t d (closed triangle, t >= 0)
__device__ __forceinline__ bool tri_hit(const WorldTri &T, const float d[3], float &t, float &u, float &v) {
  float p[3];
  cross3(d, T.e2, p);
  const float det = dot3(T.e1, p);
  if (det == 0.f) return false;
  const float inv = 1.f / det;
  u = dot3(T.s, p) * inv;
  if (u < 0.f || u > 1.f) return false;
  v = dot3(d, T.q) * inv;
  if (v < 0.f || u + v > 1.f) return false;
  t = T.tq * inv;
  return t >= 0.f;
}

__device__ __forceinline__ int find_instance(const RInstance *inst, int n_inst, uint32_t gid) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].first <= gid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the same search over a copy of the instances' first ids
__device__ __forceinline__ int find_first(const uint32_t *first, int n_inst, uint32_t gid) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= gid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void load_world_tri(const RInstance &in, const DevObject &ob, uint32_t tri, const RCam &cam,
                                               WorldTri &T, float zc[3], float sx[3], float sy[3]) {
  const int32_t *ix = ob.tris + 3 * (int64_t)tri;
  float w[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float *v = ob.verts + 3 * (int64_t)__ldg(ix + k);
    const float vo[3] = {__ldg(v), __ldg(v + 1), __ldg(v + 2)};
    world_vertex(in, vo, w[k]);
    const float q[3] = {w[k][0] - cam.e[0], w[k][1] - cam.e[1], w[k][2] - cam.e[2]};
    zc[k] = dot3(q, cam.f);
    const float xc = dot3(q, cam.r), yc = dot3(q, cam.u);
    // approximate division: the box is widened and the ray test decides
    sx[k] = (__fdividef(xc, zc[k] * cam.tx) + 1.f) * 0.5f * (float)cam.w;
    sy[k] = (1.f - __fdividef(yc, zc[k] * cam.ty)) * 0.5f * (float)cam.h;
  }
  make_tri(cam, w[0], w[1], w[2], T);
}

// pixel-centre range of a projected box, widened by a little so that the
// exact ray test, not the projection's rounding, decides the edges
__device__ __forceinline__ bool pixel_box(const RCam &cam, const float sx[3], const float sy[3], int &x0, int &x1,
                                          int &y0, int &y1) {
  float lx = fminf(sx[0], fminf(sx[1], sx[2])), hx = fmaxf(sx[0], fmaxf(sx[1], sx[2]));
  float ly = fminf(sy[0], fminf(sy[1], sy[2])), hy = fmaxf(sy[0], fmaxf(sy[1], sy[2]));
  const float slack = 5e-2f;
  if (!(hx >= -1.f && lx <= (float)cam.w + 1.f && hy >= -1.f && ly <= (float)cam.h + 1.f)) return false;
  // clamp before the integer conversions (vertices near the camera plane
  // project far outside the image)
  lx = fmaxf(lx, -2.f);
  hx = fminf(hx, (float)cam.w + 2.f);
  ly = fmaxf(ly, -2.f);
  hy = fminf(hy, (float)cam.h + 2.f);
  x0 = max(0, (int)ceilf(lx - 0.5f - slack));
  x1 = min(cam.w - 1, (int)floorf(hx - 0.5f + slack));
  y0 = max(0, (int)ceilf(ly - 0.5f - slack));
  y1 = min(cam.h - 1, (int)floorf(hy - 0.5f + slack));
  return x0 <= x1 && y0 <= y1;
}

__device__ __forceinline__ void test_pixel(const RCam &cam, const WorldTri &T, uint32_t gid, int px, int py,
                                           unsigned long long *keys) {
  float d[3], t, u, v;
  pixel_dir(cam, px, py, d);
  if (tri_hit(T, d, t, u, v)) {
    const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | gid;
    atomicMin(keys + (int64_t)py * cam.w + px, key);
  }
}

// Setup: one thread per (instance, triangle). A warp then tests the pixel
// centres of its 32 triangles' boxes together: the lanes' pixel counts are
// scanned, and the warp walks the concatenated (triangle, pixel) list 32
// items at a time, each item finding its triangle in the warp's shared
// memory -- so one triangle with a large box does not idle the other lanes.
constexpr int kSetupThreads = 256;
constexpr int kMaxSharedInstances = 2048;

__global__ void __launch_bounds__(kSetupThreads) raster_setup_kernel(RCam cam, const RInstance *inst, int n_inst,
                                                                     const DevObject *objs, uint32_t total,
                                                                     unsigned long long *keys, uint32_t *large,
                                                                     uint32_t *n_large) {
  __shared__ WorldTri s_tri[kSetupThreads];
  __shared__ int s_box[kSetupThreads][2];  // x0 | y0 << 16, width
  __shared__ uint32_t s_gid[kSetupThreads];
  __shared__ int s_end[kSetupThreads];     // inclusive prefix of the pixel counts, per warp
  __shared__ uint32_t s_first[kMaxSharedInstances];
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  const bool shared_first = n_inst <= kMaxSharedInstances;
  if (shared_first)
    for (int k = threadIdx.x; k < n_inst; k += blockDim.x) s_first[k] = inst[k].first;
  __syncthreads();
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < total; base += stride) {
    const uint32_t gid = base + threadIdx.x;
    int count = 0;
    if (gid < total) {
      const int k = shared_first ? find_first(s_first, n_inst, gid) : find_instance(inst, n_inst, gid);
      const RInstance &in = inst[k];
      WorldTri T;
      float zc[3], sx[3], sy[3];
      load_world_tri(in, objs[in.slot], gid - in.first, cam, T, zc, sx, sy);
      const bool behind = zc[0] <= 0.f && zc[1] <= 0.f && zc[2] <= 0.f;
      const bool straddles = zc[0] <= 0.f || zc[1] <= 0.f || zc[2] <= 0.f || !isfinite(sx[0]) ||
                             !isfinite(sx[1]) || !isfinite(sx[2]) || !isfinite(sy[0]) || !isfinite(sy[1]) ||
                             !isfinite(sy[2]);
      int x0, x1, y0, y1;
      if (behind) {
      } else if (straddles) {  // crosses the camera plane: the whole screen, in the queue
        large[atomicAdd(n_large, 1u)] = gid;
      } else if (pixel_box(cam, sx, sy, x0, x1, y0, y1)) {
        const int bw = x1 - x0 + 1, n = bw * (y1 - y0 + 1);
        if (n > kSmallPixels) {
          large[atomicAdd(n_large, 1u)] = gid;
        } else {
          count = n;
          s_tri[threadIdx.x] = T;
          s_box[threadIdx.x][0] = x0 | (y0 << 16);
          s_box[threadIdx.x][1] = bw;
          s_gid[threadIdx.x] = gid;
        }
      }
    }
    int incl = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    s_end[threadIdx.x] = incl;
    const int n_items = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    for (int j = lane; j < n_items; j += 32) {
      // owner: the first lane whose inclusive prefix exceeds j
      int lo = 0, hi = 31;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[wbase + mid] > j) hi = mid;
        else lo = mid + 1;
      }
      const int t = wbase + lo;
      const int first = lo ? s_end[t - 1] : 0;
      const int idx = j - first;
      const int bw = s_box[t][1];
      const int px = (s_box[t][0] & 0xffff) + idx % bw, py = (s_box[t][0] >> 16) + idx / bw;
      test_pixel(cam, s_tri[t], s_gid[t], px, py, keys);
    }
    __syncwarp();
  }
}

// one warp per queued triangle at a time: every lane forms the triangle
// (the loads are shared through L1), then the lanes sweep its box
__global__ void raster_large_kernel(RCam cam, const RInstance *inst, int n_inst, const DevObject *objs,
                                    unsigned long long *keys, const uint32_t *large, const uint32_t *n_large,
                                    uint32_t *next) {
  const int lane = threadIdx.x & 31;
  const uint32_t n = *n_large;
  while (true) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(next, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n) break;
    const uint32_t gid = large[item];
    const int k = find_instance(inst, n_inst, gid);
    const RInstance &in = inst[k];
    WorldTri T;
    float zc[3], sx[3], sy[3];
    load_world_tri(in, objs[in.slot], gid - in.first, cam, T, zc, sx, sy);
    int x0 = 0, x1 = cam.w - 1, y0 = 0, y1 = cam.h - 1;
    const bool straddles = zc[0] <= 0.f || zc[1] <= 0.f || zc[2] <= 0.f || !isfinite(sx[0]) || !isfinite(sx[1]) ||
                           !isfinite(sx[2]) || !isfinite(sy[0]) || !isfinite(sy[1]) || !isfinite(sy[2]);
    if (!straddles && !pixel_box(cam, sx, sy, x0, x1, y0, y1)) continue;
    const int bw = x1 - x0 + 1, bh = y1 - y0 + 1;
    for (int64_t j = lane; j < (int64_t)bw * bh; j += 32)
      test_pixel(cam, T, gid, x0 + (int)(j % bw), y0 + (int)(j / bw), keys);
  }
}

__global__ void raster_resolve_kernel(RCam cam, const RInstance *inst, int n_inst, const DevObject *objs,
                                      const unsigned long long *keys, lsnif_gbuffer g) {
  const int64_t npix = (int64_t)cam.w * cam.h;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[i];
    int32_t shape = -1, prim = -1;
    float u = 0.f, v = 0.f, t = CUDART_INF_F, n[3] = {0.f, 0.f, 0.f};
    if (key != kEmpty) {
      const uint32_t gid = (uint32_t)(key & 0xffffffffu);
      const int k = find_instance(inst, n_inst, gid);
      const RInstance &in = inst[k];
      const DevObject &ob = objs[in.slot];
      const uint32_t tri = gid - in.first;
      WorldTri T;
      float zc[3], sx[3], sy[3];
      load_world_tri(in, ob, tri, cam, T, zc, sx, sy);
      float d[3], tt;
      pixel_dir(cam, (int)(i % cam.w), (int)(i / cam.w), d);
      tri_hit(T, d, tt, u, v);  // the same test that produced the key: a hit
      t = __uint_as_float((uint32_t)(key >> 32));
      shape = k;
      prim = (int32_t)tri;
      if (g.nx) {
        const int32_t *ix = ob.tris + 3 * (int64_t)tri;
        const float w0 = 1.f - u - v;
        float no[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          no[c] = w0 * ob.vnormals[3 * (int64_t)ix[0] + c] + u * ob.vnormals[3 * (int64_t)ix[1] + c] +
                  v * ob.vnormals[3 * (int64_t)ix[2] + c];
        // normals map with the inverse transpose of the object -> world map: A^T
#pragma unroll
        for (int c = 0; c < 3; ++c) n[c] = in.A[c] * no[0] + in.A[3 + c] * no[1] + in.A[6 + c] * no[2];
        const float ln = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (ln > 0.f)
#pragma unroll
          for (int c = 0; c < 3; ++c) n[c] /= ln;
      }
    }
    if (g.hit) g.hit[i] = shape >= 0 ? 1 : 0;
    if (g.shape) g.shape[i] = shape;
    if (g.prim) g.prim[i] = prim;
    if (g.u) g.u[i] = u;
    if (g.v) g.v[i] = v;
    if (g.dist) g.dist[i] = t;
    if (g.nx) {
      g.nx[i] = n[0];
      g.ny[i] = n[1];
      g.nz[i] = n[2];
    }
  }
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int lsnif_raster_gbuffer(lsnif_ctx *ctx, const lsnif_camera *cam, const lsnif_instance *inst, int n_inst,
                                    lsnif_gbuffer *out, void *stream) {
  if (!ctx || !cam || !inst || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: NULL argument");
  if (n_inst < 1) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: n_inst < 1");
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: image %d x %d outside 1..16384", cam->width,
                cam->height);
  if (!(cam->tan_half_fov > 0.f) || !std::isfinite(cam->tan_half_fov))
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: tan_half_fov must be positive");
  if ((out->nx || out->ny || out->nz) && !(out->nx && out->ny && out->nz))
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: give all three normal arrays or none");
  {
    const float *v[3] = {cam->forward, cam->right, cam->up};
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        const double dd = (double)v[i][0] * v[j][0] + (double)v[i][1] * v[j][1] + (double)v[i][2] * v[j][2];
        if (std::fabs(dd - (i == j ? 1.0 : 0.0)) > 1e-4)
          return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: forward, right, up must be orthonormal");
      }
  }
  std::vector<RInstance> hin(n_inst);
  uint64_t total = 0;
  for (int k = 0; k < n_inst; ++k) {
    Object *o = find_object(ctx, inst[k].obj);
    if (!o)
      return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_raster_gbuffer: instance %d names unknown object %u", k, inst[k].obj);
    if (!o->d.verts || !o->d.tris || !o->d.vnormals)
      return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_raster_gbuffer: object %u was loaded without its mesh (keep_mesh)",
                  inst[k].obj);
    const float *m = inst[k].world_to_obj;
    double A[9], b[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) A[3 * r + c] = m[4 * r + c];
      b[r] = m[4 * r + 3];
    }
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 1e-30) || !std::isfinite(det))
      return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: instance %d has a singular transform", k);
    double M[9];  // inverse by cofactors
    M[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    M[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    M[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    M[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    M[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    M[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    M[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    M[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    M[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    RInstance &ri = hin[k];
    ri.slot = o->slot;
    ri.first = (uint32_t)total;
    ri.nt = (uint32_t)o->d.nt;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) {
        ri.M[3 * r + c] = (float)M[3 * r + c];
        ri.A[3 * r + c] = (float)A[3 * r + c];
      }
      ri.c[r] = (float)-(M[3 * r] * b[0] + M[3 * r + 1] * b[1] + M[3 * r + 2] * b[2]);
    }
    total += (uint64_t)o->d.nt;
  }
  if (total >= (1ull << 31))
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_raster_gbuffer: 2^31 or more triangles over the instances");
  RCam rc{};
  for (int k = 0; k < 3; ++k) {
    rc.e[k] = cam->eye[k];
    rc.f[k] = cam->forward[k];
    rc.r[k] = cam->right[k];
    rc.u[k] = cam->up[k];
  }
  rc.ty = cam->tan_half_fov;
  rc.tx = (float)((double)cam->tan_half_fov * cam->width / cam->height);
  rc.rw = 2.f / (float)cam->width;
  rc.rh = 2.f / (float)cam->height;
  rc.w = cam->width;
  rc.h = cam->height;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t npix = (int64_t)cam->width * cam->height;
  const size_t bytes = al(sizeof(RInstance) * n_inst) + al((size_t)npix * 8) + al((size_t)total * 4) + al(16);
  if (ctx->raster_bytes < bytes) {
    if (ctx->raster_buf) {
      cudaDeviceSynchronize();
      dev_free(ctx, ctx->raster_buf);
      ctx->raster_buf = nullptr;
      ctx->raster_bytes = 0;
    }
    int r = dev_alloc(ctx, bytes, &ctx->raster_buf, "raster scratch");
    if (r) return r;
    ctx->raster_bytes = bytes;
  }
  uint8_t *p = reinterpret_cast<uint8_t *>(ctx->raster_buf);
  RInstance *dinst = reinterpret_cast<RInstance *>(p);
  p += al(sizeof(RInstance) * n_inst);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(p);
  p += al((size_t)npix * 8);
  uint32_t *large = reinterpret_cast<uint32_t *>(p);
  p += al((size_t)total * 4);
  uint32_t *counters = reinterpret_cast<uint32_t *>(p);  // [0] queued, [1] next

  cudaError_t e = cudaMemcpyAsync(dinst, hin.data(), sizeof(RInstance) * n_inst, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, (size_t)npix * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 8, st);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess && total > 0) {
    const uint32_t t32 = (uint32_t)total;
    const int grid = (int)std::min<uint64_t>((total + 255) / 256, (uint64_t)sms * 16);
    raster_setup_kernel<<<grid, 256, 0, st>>>(rc, dinst, n_inst, ctx->d_objs, t32, keys, large, counters);
    raster_large_kernel<<<sms * 8, 256, 0, st>>>(rc, dinst, n_inst, ctx->d_objs, keys, large, counters,
                                                 counters + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int grid = (int)std::min<int64_t>((npix + 255) / 256, (int64_t)sms * 16);
    raster_resolve_kernel<<<grid, 256, 0, st>>>(rc, dinst, n_inst, ctx->d_objs, keys, *out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_raster_gbuffer");
  return LSNIF_OK;
}
