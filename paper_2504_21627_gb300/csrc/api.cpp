// C ABI of the LSNIF library: contexts, objects, the query orchestration,
// stage entry points, profiling and host-side fault injection.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bvh.h"
#include "lsnif_impl.h"
#include "runtime.h"

namespace lsnif {
void mesh_bbox(const float *verts, int64_t nv, float bmin[3], float bmax[3]);
void voxelize_mesh(const float *verts, const int32_t *tris, int64_t nt, const float bmin[3], const float bmax[3],
                   int V, uint32_t *occ, std::vector<std::pair<int32_t, int32_t>> *pairs);
void level_resolutions(int N_min, int N_max, int L, int32_t *out);
}  // namespace lsnif

using namespace lsnif;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

int lsnif::fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int lsnif::cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) return fail(LSNIF_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorNotSupported) return fail(LSNIF_ERR_UNSUPPORTED, "%s: configuration not supported", what);
  return fail(LSNIF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *lsnif_last_error(void) { return g_err.c_str(); }
// format version of serialized objects (lsnif_save_object), independent of the API's
constexpr uint64_t kBlobVersion = 1;

extern "C" int lsnif_version(void) { return LSNIF_API_VERSION; }

// ---------------------------------------------------------------------------
// device memory accounting
// ---------------------------------------------------------------------------
int lsnif::dev_alloc(lsnif_ctx *ctx, size_t bytes, void **out, const char *what) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->fail_alloc_after >= 0) {
    if (ctx->fail_alloc_after == 0) {
      ctx->fail_alloc_after = -1;
      return fail(LSNIF_ERR_OUT_OF_MEMORY, "%s: injected allocation failure (%zu bytes)", what, bytes);
    }
    --ctx->fail_alloc_after;
  }
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(LSNIF_ERR_OVER_BUDGET, "%s: %zu bytes would exceed the budget (%zu of %zu used)", what, bytes,
                ctx->used, ctx->budget);
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return cuda_fail(e, what);
  }
  ctx->used += bytes;
  ctx->sizes[*out] = bytes;
  return LSNIF_OK;
}

void lsnif::dev_free(lsnif_ctx *ctx, void *p) {
  if (!p) return;
  auto it = ctx->sizes.find(p);
  if (it != ctx->sizes.end()) {
    ctx->used -= it->second;
    ctx->sizes.erase(it);
  }
  cudaFree(p);
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int lsnif_create(lsnif_ctx **out, int device, size_t budget) {
  if (!out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "lsnif_create: no CUDA device");
  }
  if (device < 0 || device >= ndev) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_create: device %d of %d", device, ndev);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "lsnif_create: cudaSetDevice");
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  if (prop.major < 10) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_create: device is sm_%d%d, need sm_103a", prop.major, prop.minor);
  lsnif_ctx *c = new lsnif_ctx();
  c->device = device;
  c->budget = budget;
  c->sms = prop.multiProcessorCount;
  c->slots.assign(kMaxSlots, nullptr);
  c->gen.assign(kMaxSlots, 0);
  int rc = dev_alloc(c, sizeof(DevObject) * kMaxSlots, (void **)&c->d_objs, "lsnif_create: object table");
  if (rc) { delete c; return rc; }
  cudaMemset(c->d_objs, 0, sizeof(DevObject) * kMaxSlots);
  rc = dev_alloc(c, 64, (void **)&c->d_err, "lsnif_create: error word");
  if (rc) { dev_free(c, c->d_objs); delete c; return rc; }
  cudaMemset(c->d_err, 0, 64);
  rc = dev_alloc(c, 64, (void **)&c->d_prof_meta, "lsnif_create: profile");
  if (rc) { dev_free(c, c->d_objs); dev_free(c, c->d_err); delete c; return rc; }
  for (auto &ev : c->ev) cudaEventCreate(&ev);
  *out = c;
  return LSNIF_OK;
}

extern "C" int lsnif_destroy(lsnif_ctx *ctx) {
  if (!ctx) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  server_shutdown(ctx);
  cudaDeviceSynchronize();
  clear_graphs(ctx);
  for (int s = 0; s < kMaxSlots; ++s)
    if (ctx->slots[s]) free_object(ctx, ctx->slots[s]);
  free_workspace(ctx, &ctx->ws);
  if (ctx->scene_buf) dev_free(ctx, ctx->scene_buf);
  if (ctx->pair_buf) dev_free(ctx, ctx->pair_buf);
  if (ctx->raster_buf) dev_free(ctx, ctx->raster_buf);
  dev_free(ctx, ctx->d_objs);
  dev_free(ctx, ctx->d_err);
  dev_free(ctx, ctx->d_prof_meta);
  for (auto &ev : ctx->ev) cudaEventDestroy(ev);
  for (auto &ev : ctx->hev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
  if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
  delete ctx;
  return LSNIF_OK;
}

extern "C" size_t lsnif_device_bytes(lsnif_ctx *ctx) { return ctx ? ctx->used : 0; }

extern "C" int lsnif_debug_fail_alloc_after(lsnif_ctx *ctx, int64_t n) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_debug_fail_alloc_after: ctx is NULL");
  ctx->fail_alloc_after = n;
  return LSNIF_OK;
}

int lsnif::check_device(lsnif_ctx *ctx, cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int h = 0;
  e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read device error word");
  if (h) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (h & kErrBadHandle) return fail(LSNIF_ERR_DEVICE_CHECK, "a ray named an unknown object handle");
    if (h & kErrWaitTimeout) return fail(LSNIF_ERR_DEVICE_CHECK, "a kernel gave up a bounded wait");
    return fail(LSNIF_ERR_DEVICE_CHECK, "a kernel reported a failed internal check (0x%x)", h);
  }
  return LSNIF_OK;
}

extern "C" int lsnif_check(lsnif_ctx *ctx, void *stream) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_check: ctx is NULL");
  return check_device(ctx, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
namespace {

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
float unif(uint64_t &s) { return (float)((splitmix64(s) >> 40) * (1.0 / 16777216.0)); }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate_config(const lsnif_config &c) {
  if (!is_pow2(c.V) || c.V < 2 || c.V > 1024) return fail(LSNIF_ERR_INVALID_ARG, "V=%d must be a power of two in [2,1024]", c.V);
  if (c.H < 2 || c.H > 2 * kMaxCap || (c.H & 1)) return fail(LSNIF_ERR_INVALID_ARG, "H=%d must be even in [2,64]", c.H);
  if (c.L < 1 || c.L > LSNIF_MAX_LEVELS) return fail(LSNIF_ERR_INVALID_ARG, "L=%d out of [1,%d]", c.L, LSNIF_MAX_LEVELS);
  if (!(c.F == 1 || c.F == 2 || c.F == 4)) return fail(LSNIF_ERR_INVALID_ARG, "F=%d must be 1, 2 or 4", c.F);
  if (c.log2_T < 4 || c.log2_T > 24) return fail(LSNIF_ERR_INVALID_ARG, "log2_T=%d out of [4,24]", c.log2_T);
  if (c.N_min < 1 || c.N_max < c.N_min || c.N_max > (1 << 20)) return fail(LSNIF_ERR_INVALID_ARG, "bad N_min/N_max");
  if (c.n_hidden < 1 || c.n_hidden > LSNIF_MAX_HIDDEN) return fail(LSNIF_ERR_INVALID_ARG, "n_hidden=%d", c.n_hidden);
  if (c.width < 16 || c.width > 256 || c.width % 16) return fail(LSNIF_ERR_INVALID_ARG, "width=%d", c.width);
  if (c.n_mat < 1 || c.n_mat > 56) return fail(LSNIF_ERR_INVALID_ARG, "n_mat=%d out of [1,56]", c.n_mat);
  if (c.activation != LSNIF_RELU && c.activation != LSNIF_LEAKY_RELU) return fail(LSNIF_ERR_INVALID_ARG, "activation");
  if ((int64_t)c.H * c.L * c.F % 16) return fail(LSNIF_ERR_INVALID_ARG, "H*L*F must be a multiple of 16");
  if (!(c.table_init >= 0.f)) return fail(LSNIF_ERR_INVALID_ARG, "table_init");
  return LSNIF_OK;
}

int64_t mlp_param_count(const lsnif_config &c) {
  int64_t n_in = (int64_t)c.H * c.L * c.F, n = 0, fi = n_in;
  for (int l = 0; l < c.n_hidden; ++l) { n += fi * c.width + c.width; fi = c.width; }
  n += fi * (8 + c.n_mat) + (8 + c.n_mat);
  return n;
}

// Blob layout: [header][config][bbox 6f][res L i32][occ words][tables f32][mlp f32][fnv64]
constexpr char kMagic[8] = {'L', 'S', 'N', 'I', 'F', 'B', 'L', '1'};
uint64_t fnv1a(const uint8_t *p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
  return h;
}

}  // namespace

size_t lsnif::blob_size(const Object *o) {
  const lsnif_config &c = o->cfg;
  size_t occ_words = ((size_t)c.V * c.V * c.V + 31) / 32;
  return 8 + 8 + sizeof(lsnif_config) + 24 + 4 * (size_t)c.L + 4 * occ_words +
         4 * ((size_t)c.L << c.log2_T) * c.F + 4 * (size_t)mlp_param_count(c) + 8;
}

void lsnif::free_object(lsnif_ctx *ctx, Object *o) {
  for (void *p : o->allocs) dev_free(ctx, p);
  free_train_state(ctx, o);
  ctx->slots[o->slot] = nullptr;
  DevObject z{};
  cudaMemcpy(ctx->d_objs + o->slot, &z, sizeof z, cudaMemcpyHostToDevice);
  delete o;
}

static int obj_alloc(lsnif_ctx *ctx, Object *o, size_t bytes, void **p, const char *what) {
  int rc = dev_alloc(ctx, bytes, p, what);
  if (rc == LSNIF_OK) {
    o->allocs.push_back(*p);
    o->device_bytes += ctx->sizes[*p];
  }
  return rc;
}

// Upload tables + MLP (host FP32) and rebuild the reduced-precision copies.
int lsnif::upload_params(lsnif_ctx *ctx, Object *o, const float *tables, const float *mlp) {
  const lsnif_config &c = o->cfg;
  size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  cudaError_t e;
  if (tables && (e = cudaMemcpy((void *)o->d.tab32, tables, 4 * nt, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload tables");
  if (mlp && (e = cudaMemcpy((void *)o->d.mlp32, mlp, 4 * o->n_params_mlp, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload network");
  return refresh_copies(ctx, o, 0);
}

int lsnif::refresh_copies(lsnif_ctx *, Object *o, cudaStream_t st) {
  o->fp8_stale = true;
  const lsnif_config &c = o->cfg;
  size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  cudaError_t e = launch_tables_to_half(o->d.tab32, const_cast<uint16_t *>(o->d.tab16), (int64_t)nt, st);
  if (e == cudaSuccess) e = launch_build_umma(o->d, st);
  if (e != cudaSuccess) return cuda_fail(e, "refresh reduced-precision copies");
  return LSNIF_OK;
}

// ---- FP8 network (LSNIF_FP8_FUSED) -------------------------------------------

// The power of two s with 448/2 < s m <= 448 (1 when m is 0).
static double e4m3_scale(double m) {
  if (!(m > 0)) return 1.0;
  int e = 0;
  std::frexp(448.0 / m, &e);
  return std::ldexp(1.0, e - 1);
}

// Nearest FP8 E4M3 code (1 sign, 4 exponent bits with bias 7, 3 mantissa
// bits; normals from 2^-6, subnormals in steps of 2^-9, largest finite 448),
// ties to even, saturating.
static uint8_t to_e4m3(double x) {
  const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
  double a = std::fabs(x);
  if (!(a == a)) return 0x7F;
  if (a >= 448.0) return sign | 0x7E;
  int e = 0;
  std::frexp(a, &e);  // a = f 2^e, 0.5 <= f < 1
  const int E = std::max(e - 1, -6);
  const double q = std::ldexp(1.0, E - 3);
  double k = std::nearbyint(a / q);  // default rounding: to nearest, ties to even
  double r = k * q;
  if (r >= 448.0) return sign | 0x7E;
  if (r == 0.0) return sign;
  int er = 0;
  std::frexp(r, &er);
  const int Er = er - 1;
  if (Er < -6) return sign | (uint8_t)(r / std::ldexp(1.0, -9));           // subnormal: m 2^-9
  const int m = (int)(r / std::ldexp(1.0, Er - 3)) - 8;                      // 1.m x 2^Er
  return sign | (uint8_t)(((Er + 7) << 3) | m);
}

// offset of (row n, column k) in a K-major core-matrix tile of E4M3 bytes
// with K columns
static size_t core8(int n, int k, int K) {
  return ((size_t)(n >> 3) * (K / 16) + (k >> 4)) * 128 + (n & 7) * 16 + (k & 15);
}

int lsnif::ensure_fp8(lsnif_ctx *ctx, Object *o, cudaStream_t st) {
  DevObject &d = o->d;
  if (!fused8_supported(d))
    return fail(LSNIF_ERR_UNSUPPORTED, "FP8 query: object %u has no FP8 kernel shape (F in {2,4}, width 64/128, "
                                       "L*F a multiple of 16, L <= 16)", o->handle);
  if (!o->fp8_stale && d.w0_8) return LSNIF_OK;
  const lsnif_config &c = o->cfg;
  const int W = c.width, n_in = d.n_in, nh = c.n_hidden, nop = d.n_out_pad, n_out = d.n_out;
  const int CHK = 2 * c.L * c.F, chunks = c.H / 2;
  const size_t hid_bytes = (size_t)(nh - 1) * W * W, out_bytes = (size_t)nop * W;
  const size_t bias_off = (hid_bytes + out_bytes + 15) & ~size_t(15);
  const size_t n_bias = (size_t)nh * W + nop;
  const size_t scale_off = bias_off + 4 * n_bias;
  const size_t blob_bytes = (scale_off + 4 * 2 * (nh + 1) + 15) & ~size_t(15);
  int rc;
  if (!d.w0_8) {
    void *p = nullptr;
    if ((rc = obj_alloc(ctx, o, (size_t)W * n_in, &p, "FP8 first layer"))) return rc;
    d.w0_8 = (const uint8_t *)p;
    if ((rc = obj_alloc(ctx, o, blob_bytes, &p, "FP8 network"))) return rc;
    d.blob8 = (const uint8_t *)p;
  }
  // the parameters as they are now (training may have changed them)
  std::vector<float> mlp(o->n_params_mlp);
  uint32_t *dmax = nullptr;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMalloc(&dmax, 4);
  if (e == cudaSuccess)
    e = launch_max_abs_half(d.tab16, ((int64_t)c.L << c.log2_T) * c.F, dmax, st);
  uint32_t mbits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mbits, dmax, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mlp.data(), d.mlp32, 4 * mlp.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dmax) cudaFree(dmax);
  if (e != cudaSuccess) return cuda_fail(e, "FP8 network: read parameters");
  float tmax;
  memcpy(&tmax, &mbits, 4);
  // layers: (fan_in, fan_out) = n_in -> W (x nh) -> n_out
  std::vector<int> fi(nh + 1), fo(nh + 1);
  for (int l = 0; l <= nh; ++l) {
    fi[l] = l == 0 ? n_in : W;
    fo[l] = l == nh ? n_out : W;
  }
  std::vector<size_t> woff(nh + 1);
  size_t off = 0;
  for (int l = 0; l <= nh; ++l) {
    woff[l] = off;
    off += (size_t)fi[l] * fo[l] + fo[l];
  }
  std::vector<double> s_in(nh + 1), w_sc(nh + 1);
  double M = tmax;
  for (int l = 0; l <= nh; ++l) {
    const float *Wl = mlp.data() + woff[l], *bl = Wl + (size_t)fi[l] * fo[l];
    double wmax = 0.0, next = 0.0;
    for (int j = 0; j < fo[l]; ++j) {
      double ss = 0.0;
      for (int i = 0; i < fi[l]; ++i) {
        const double w = Wl[(size_t)j * fi[l] + i];
        wmax = std::max(wmax, std::fabs(w));
        ss += w * w;
      }
      next = std::max(next, std::sqrt(ss) * M + std::fabs((double)bl[j]));
    }
    s_in[l] = e4m3_scale(M);
    w_sc[l] = e4m3_scale(wmax);
    M = next;
  }
  // first layer, chunk-major: chunk s holds columns [s CHK, (s+1) CHK)
  std::vector<uint8_t> w0((size_t)W * n_in, 0);
  for (int s2 = 0; s2 < chunks; ++s2)
    for (int n = 0; n < W; ++n)
      for (int k = 0; k < CHK; ++k)
        w0[(size_t)s2 * W * CHK + core8(n, k, CHK)] =
            to_e4m3((double)mlp[woff[0] + (size_t)n * n_in + (size_t)s2 * CHK + k] * w_sc[0]);
  // hidden layers 1.., then the output layer (rows beyond n_out zero), then FP32
  std::vector<uint8_t> blob(blob_bytes, 0);
  size_t p8 = 0;
  for (int l = 1; l <= nh; ++l) {
    const int rows = l == nh ? nop : W;
    for (int n = 0; n < rows; ++n)
      for (int k = 0; k < W; ++k)
        blob[p8 + core8(n, k, W)] =
            n < fo[l] ? to_e4m3((double)mlp[woff[l] + (size_t)n * W + k] * w_sc[l]) : (uint8_t)0;
    p8 += (size_t)rows * W;
  }
  float *fb = reinterpret_cast<float *>(blob.data() + bias_off);
  for (int l = 0; l <= nh; ++l)
    for (int j = 0; j < (l == nh ? nop : W); ++j)
      fb[(size_t)l * W + j] = j < fo[l] ? mlp[woff[l] + (size_t)fi[l] * fo[l] + j] : 0.f;
  float *fs = reinterpret_cast<float *>(blob.data() + scale_off);
  for (int l = 0; l <= nh; ++l) {
    fs[l] = (float)(1.0 / (s_in[l] * w_sc[l]));
    fs[nh + 1 + l] = (float)s_in[l];
  }
  e = cudaMemcpy((void *)d.w0_8, w0.data(), w0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void *)d.blob8, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  d.blob8_bytes = (uint32_t)blob_bytes;
  d.blob8_bias_off = (uint32_t)bias_off;
  d.blob8_scale_off = (uint32_t)scale_off;
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_objs + o->slot, &d, sizeof d, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "FP8 network: upload");
  o->fp8_stale = false;
  return LSNIF_OK;
}

// Chebyshev (L-infinity) distance, in voxels, from every voxel to the
// nearest occupied one, capped at `cap` -- separable: the distance along x
// within each row, then D(x,y,z) = min over |j| <= cap of max(|j|,
// D_x(x,y+j,z)), then the same along z (the maximum norm splits into
// per-axis maxima, so the minimum over all occupied voxels can be taken one
// axis at a time).
static std::vector<uint8_t> occupancy_distance(const std::vector<uint32_t> &occ, int V, int cap) {
  const size_t n = (size_t)V * V * V;
  std::vector<uint8_t> a(n), b(n);
  for (size_t row = 0; row < (size_t)V * V; ++row) {
    uint8_t *r = a.data() + row * V;
    int last = -1000000;
    for (int x = 0; x < V; ++x) {
      const size_t id = row * V + x;
      if ((occ[id >> 5] >> (id & 31)) & 1u) last = x;
      r[x] = (uint8_t)std::min(cap, x - last);
    }
    last = 1000000;
    for (int x = V - 1; x >= 0; --x) {
      const size_t id = row * V + x;
      if ((occ[id >> 5] >> (id & 31)) & 1u) last = x;
      r[x] = (uint8_t)std::min<int>(r[x], std::min(cap, last - x));
    }
  }
  auto pass = [&](const std::vector<uint8_t> &src, std::vector<uint8_t> &dst, size_t stride) {
    for (size_t id = 0; id < n; ++id) {
      const int c = (int)((id / stride) % (size_t)V);
      int best = src[id];
      for (int j = 1; j < best && j <= cap; ++j) {
        if (c - j >= 0) best = std::min(best, std::max(j, (int)src[id - j * stride]));
        if (c + j < V) best = std::min(best, std::max(j, (int)src[id + j * stride]));
      }
      dst[id] = (uint8_t)best;
    }
  };
  pass(a, b, (size_t)V);
  pass(b, a, (size_t)V * V);
  return a;
}

// Host-only entry point of the distance transform (no GPU), for tests.
extern "C" int lsnif_occupancy_distance_host(const uint32_t *occ, int32_t V, int32_t cap, uint8_t *out) {
  if (!occ || !out || V < 1 || V > 1024 || cap < 1 || cap > 255) return LSNIF_ERR_INVALID_ARG;
  const size_t words = ((size_t)V * V * V + 31) / 32;
  std::vector<uint32_t> o(occ, occ + words);
  const std::vector<uint8_t> d = occupancy_distance(o, V, cap);
  memcpy(out, d.data(), d.size());
  return LSNIF_OK;
}

// A mesh object: the triangles, shading normals, materials and a BVH built
// on the host; no voxels, tables or network.
static int load_mesh_object(lsnif_ctx *ctx, const lsnif_object_desc *desc, lsnif_obj *out) {
  const lsnif_mesh &m = desc->mesh;
  const int n_mat = desc->cfg.n_mat;
  if (n_mat < 1 || n_mat > 64) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: n_mat = %d", n_mat);
  if (!m.verts || !m.tris || m.nv <= 0 || m.nt <= 0)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: mesh needs vertices and triangles");
  if (m.nt >= ((int64_t)1 << 30)) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: too many triangles");
  for (int64_t i = 0; i < 3 * m.nt; ++i)
    if (m.tris[i] < 0 || m.tris[i] >= m.nv) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: triangle index out of range");
  for (int64_t i = 0; i < 3 * m.nv; ++i)
    if (!std::isfinite(m.verts[i])) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: non-finite vertex");
  if (m.tri_mat)
    for (int64_t i = 0; i < m.nt; ++i)
      if (m.tri_mat[i] < 0 || m.tri_mat[i] >= n_mat) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: material index out of range");
  float bmin[3], bmax[3];
  mesh_bbox(m.verts, m.nv, bmin, bmax);
  std::vector<BvhNode> nodes;
  std::vector<int32_t> order;
  bvh_build(m.verts, m.tris, m.nt, nodes, order);
  std::vector<float> tdata(12 * (size_t)m.nt, 0.f);  // v0, e1, e2 as float4
  for (int64_t i = 0; i < m.nt; ++i) {
    const int32_t *ix = m.tris + 3 * (int64_t)order[i];
    const float *a = m.verts + 3 * (int64_t)ix[0], *b = m.verts + 3 * (int64_t)ix[1], *c = m.verts + 3 * (int64_t)ix[2];
    float *w = tdata.data() + 12 * i;
    for (int k = 0; k < 3; ++k) {
      w[k] = a[k];
      w[4 + k] = b[k] - a[k];
      w[8 + k] = c[k] - a[k];
    }
  }
  int slot = -1;
  for (int s = 0; s < kMaxSlots; ++s)
    if (!ctx->slots[s]) { slot = s; break; }
  if (slot < 0) return fail(LSNIF_ERR_OUT_OF_MEMORY, "lsnif_load_object: object table full (%d)", kMaxSlots);
  Object *o = new Object();
  o->cfg = lsnif_config{};
  o->cfg.n_mat = n_mat;
  o->slot = slot;
  ctx->gen[slot] = (uint16_t)(ctx->gen[slot] + 1);
  if (ctx->gen[slot] == 0) ctx->gen[slot] = 1;
  o->handle = ((uint32_t)ctx->gen[slot] << 16) | (uint32_t)(slot + 1);
  memcpy(o->bmin, bmin, 12);
  memcpy(o->bmax, bmax, 12);
  o->bvh_nodes = (int64_t)nodes.size();
  ctx->slots[slot] = o;
  DevObject &d = o->d;
  memset(&d, 0, sizeof d);
  for (int a = 0; a < 3; ++a) {
    d.bmin[a] = bmin[a];
    d.inv_ext[a] = 1.0f / (bmax[a] - bmin[a]);
  }
  d.kind = 1;
  d.n_mat = n_mat;
  d.nt = m.nt;
  std::vector<float> vn(3 * m.nv, 0.f), alb(3 * n_mat, 0.5f);
  std::vector<int32_t> tm(m.nt, 0);
  if (m.vnormals) memcpy(vn.data(), m.vnormals, 12 * m.nv);
  if (m.tri_mat) memcpy(tm.data(), m.tri_mat, 4 * m.nt);
  if (m.mat_albedo) memcpy(alb.data(), m.mat_albedo, 12 * n_mat);
  int rc;
  void *p;
  cudaError_t e = cudaSuccess;
  auto put = [&](const void **field, const void *src, size_t bytes, const char *what) -> bool {
    if ((rc = obj_alloc(ctx, o, bytes, &p, what)) != LSNIF_OK) return false;
    *field = p;
    if (e == cudaSuccess) e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
    return true;
  };
  if (!put((const void **)&d.verts, m.verts, 12 * m.nv, "mesh vertices") ||
      !put((const void **)&d.tris, m.tris, 12 * m.nt, "mesh triangles") ||
      !put((const void **)&d.vnormals, vn.data(), 12 * m.nv, "mesh normals") ||
      !put((const void **)&d.tri_mat, tm.data(), 4 * m.nt, "mesh materials") ||
      !put((const void **)&d.albedo, alb.data(), 12 * n_mat, "material albedo") ||
      !put((const void **)&d.bvh_nodes, nodes.data(), sizeof(BvhNode) * nodes.size(), "BVH nodes") ||
      !put((const void **)&d.bvh_tris, tdata.data(), 4 * tdata.size(), "BVH triangles") ||
      !put((const void **)&d.bvh_order, order.data(), 4 * order.size(), "BVH order")) {
    free_object(ctx, o);
    return rc;
  }
  d.handle = o->handle;
  d.valid = 1;
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_objs + slot, &d, sizeof d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_object(ctx, o); return cuda_fail(e, "lsnif_load_object: upload mesh object"); }
  ctx->n_slots_used = std::max(ctx->n_slots_used, slot + 1);
  *out = o->handle;
  return LSNIF_OK;
}

extern "C" int lsnif_load_object(lsnif_ctx *ctx, const lsnif_object_desc *desc, lsnif_obj *out) {
  if (!ctx || !desc || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: NULL argument");
  *out = 0;
  cudaSetDevice(ctx->device);
  if (!desc->blob && desc->bvh_below_faces > 0 && desc->mesh.nt < desc->bvh_below_faces)
    return load_mesh_object(ctx, desc, out);
  lsnif_config cfg;
  float bmin[3], bmax[3];
  std::vector<int32_t> res;
  std::vector<uint32_t> occ;
  std::vector<float> tables, mlp;
  const float *tab_src = desc->tables, *mlp_src = desc->mlp;
  std::vector<std::pair<int32_t, int32_t>> pairs;

  if (desc->blob) {
    const uint8_t *b = (const uint8_t *)desc->blob;
    size_t n = desc->blob_len;
    if (n < 16 + sizeof(lsnif_config) + 24 + 8 || memcmp(b, kMagic, 8) != 0)
      return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: not an LSNIF blob");
    uint64_t ver;
    memcpy(&ver, b + 8, 8);
    if (ver != kBlobVersion) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: blob version %llu", (unsigned long long)ver);
    uint64_t stored;
    memcpy(&stored, b + n - 8, 8);
    if (fnv1a(b, n - 8) != stored) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: checksum mismatch");
    memcpy(&cfg, b + 16, sizeof cfg);
    int rc = validate_config(cfg);
    if (rc) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: blob config invalid (%s)", g_err.c_str());
    Object tmp;
    tmp.cfg = cfg;
    if (blob_size(&tmp) != n) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: blob size %zu, expected %zu", n, blob_size(&tmp));
    const uint8_t *p = b + 16 + sizeof cfg;
    memcpy(bmin, p, 12);
    memcpy(bmax, p + 12, 12);
    p += 24;
    res.resize(cfg.L);
    memcpy(res.data(), p, 4 * cfg.L);
    p += 4 * cfg.L;
    occ.resize(((size_t)cfg.V * cfg.V * cfg.V + 31) / 32);
    memcpy(occ.data(), p, 4 * occ.size());
    p += 4 * occ.size();
    tables.resize(((size_t)cfg.L << cfg.log2_T) * cfg.F);
    memcpy(tables.data(), p, 4 * tables.size());
    p += 4 * tables.size();
    mlp.resize(mlp_param_count(cfg));
    memcpy(mlp.data(), p, 4 * mlp.size());
    tab_src = tables.data();
    mlp_src = mlp.data();
    for (int a = 0; a < 3; ++a)
      if (!(bmax[a] > bmin[a])) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: blob AABB is empty");
  } else {
    cfg = desc->cfg;
    int rc = validate_config(cfg);
    if (rc) return rc;
    const lsnif_mesh &m = desc->mesh;
    if (!m.verts || !m.tris || m.nv <= 0 || m.nt <= 0)
      return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: mesh needs vertices and triangles");
    for (int64_t i = 0; i < 3 * m.nt; ++i)
      if (m.tris[i] < 0 || m.tris[i] >= m.nv) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: triangle index out of range");
    for (int64_t i = 0; i < 3 * m.nv; ++i)
      if (!std::isfinite(m.verts[i])) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: non-finite vertex");
    if (m.tri_mat)
      for (int64_t i = 0; i < m.nt; ++i)
        if (m.tri_mat[i] < 0 || m.tri_mat[i] >= cfg.n_mat) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_load_object: material index out of range");
    mesh_bbox(m.verts, m.nv, bmin, bmax);
    occ.resize(((size_t)cfg.V * cfg.V * cfg.V + 31) / 32);
    voxelize_mesh(m.verts, m.tris, m.nt, bmin, bmax, cfg.V, occ.data(), desc->keep_mesh ? &pairs : nullptr);
    res.resize(cfg.L);
    level_resolutions(cfg.N_min, cfg.N_max, cfg.L, res.data());
    uint64_t s = cfg.seed * 0x9E3779B97F4A7C15ull + 0x1234567ull;
    if (!tab_src) {
      tables.resize(((size_t)cfg.L << cfg.log2_T) * cfg.F);
      for (float &v : tables) v = (2.f * unif(s) - 1.f) * cfg.table_init;
      tab_src = tables.data();
    }
    if (!mlp_src) {
      mlp.resize(mlp_param_count(cfg));
      size_t o = 0;
      int fi = cfg.H * cfg.L * cfg.F;
      for (int l = 0; l <= cfg.n_hidden; ++l) {
        int fo = l < cfg.n_hidden ? cfg.width : 8 + cfg.n_mat;
        float a = std::sqrt(6.f / (float)(fi + fo));  // Xavier-uniform
        for (int64_t i = 0; i < (int64_t)fi * fo; ++i) mlp[o++] = (2.f * unif(s) - 1.f) * a;
        for (int i = 0; i < fo; ++i) mlp[o++] = 0.f;
        fi = fo;
      }
      mlp_src = mlp.data();
    }
  }
  for (int l = 0; l < cfg.L; ++l)
    if (res[l] < 1) return fail(LSNIF_ERR_CORRUPT, "lsnif_load_object: level resolution < 1");

  // slot + handle
  int slot = -1;
  for (int s = 0; s < kMaxSlots; ++s)
    if (!ctx->slots[s]) { slot = s; break; }
  if (slot < 0) return fail(LSNIF_ERR_OUT_OF_MEMORY, "lsnif_load_object: object table full (%d)", kMaxSlots);
  Object *o = new Object();
  o->cfg = cfg;
  o->slot = slot;
  ctx->gen[slot] = (uint16_t)(ctx->gen[slot] + 1);
  if (ctx->gen[slot] == 0) ctx->gen[slot] = 1;
  o->handle = ((uint32_t)ctx->gen[slot] << 16) | (uint32_t)(slot + 1);
  o->n_params_mlp = mlp_param_count(cfg);
  o->occ_host = occ;
  o->res.assign(res.begin(), res.end());
  memcpy(o->bmin, bmin, 12);
  memcpy(o->bmax, bmax, 12);
  ctx->slots[slot] = o;  // freed through free_object on any failure below

  DevObject &d = o->d;
  memset(&d, 0, sizeof d);
  for (int a = 0; a < 3; ++a) {
    d.bmin[a] = bmin[a];
    d.inv_ext[a] = 1.0f / (bmax[a] - bmin[a]);
  }
  d.V = cfg.V;
  d.log2V = 0;
  while ((1 << d.log2V) < cfg.V) ++d.log2V;
  d.invV = 1.0f / (float)cfg.V;
  d.L = cfg.L;
  d.F = cfg.F;
  d.log2T = cfg.log2_T;
  d.mask = (1u << cfg.log2_T) - 1u;
  for (int l = 0; l < cfg.L; ++l) d.res[l] = res[l];
  d.H = cfg.H;
  d.n_in = cfg.H * cfg.L * cfg.F;
  d.n_hidden = cfg.n_hidden;
  d.width = cfg.width;
  d.n_out = 8 + cfg.n_mat;
  d.n_out_pad = (d.n_out + 15) / 16 * 16;
  d.n_mat = cfg.n_mat;
  d.act = cfg.activation;
  size_t nt = ((size_t)cfg.L << cfg.log2_T) * cfg.F;
  int rc;
  void *p;
#define OALLOC(field, type, bytes, what)                                   \
  if ((rc = obj_alloc(ctx, o, (bytes), &p, what)) != LSNIF_OK) {          \
    free_object(ctx, o);                                                   \
    return rc;                                                             \
  }                                                                        \
  d.field = (type)p;
  OALLOC(occ, const uint32_t *, 4 * occ.size(), "occupancy");
  // occupancy distance field for empty-space skipping in the traversal
  const std::vector<uint8_t> dist = occupancy_distance(occ, cfg.V, kDistCap);
  OALLOC(dist, const uint8_t *, dist.size(), "occupancy distance");
  OALLOC(tab32, const float *, 4 * nt, "tables");
  OALLOC(tab16, const uint16_t *, 2 * nt, "FP16 tables");
  OALLOC(mlp32, const float *, 4 * (size_t)o->n_params_mlp, "network");
  // tcgen05 weight blobs (BF16 and FP16 copies): layers (output padded to n_out_pad rows) + FP32 biases
  size_t wbytes = (size_t)cfg.width * d.n_in * 2 + (size_t)(cfg.n_hidden - 1) * cfg.width * cfg.width * 2 +
                  (size_t)d.n_out_pad * cfg.width * 2;
  d.umma_bias_off = (uint32_t)((wbytes + 15) & ~size_t(15));
  d.umma_bytes = (uint32_t)(d.umma_bias_off + 4 * ((size_t)cfg.n_hidden * cfg.width + d.n_out_pad));
  d.umma_bytes = (d.umma_bytes + 15) & ~15u;
  OALLOC(umma, const uint8_t *, d.umma_bytes, "tensor-core weights");
  OALLOC(umma_h, const uint8_t *, d.umma_bytes, "FP16 tensor-core weights");
  d.umma_lo_bytes = (uint32_t)(((wbytes - (size_t)cfg.width * d.n_in * 2) + 15) & ~size_t(15));
  OALLOC(umma_lo, const uint8_t *, d.umma_lo_bytes, "BF16 residual weights");
  OALLOC(w0_16c, const uint8_t *, (size_t)cfg.width * d.n_in * 2, "chunk-major FP16 first layer");
  OALLOC(plain_out, const float *, 4 * ((size_t)d.n_out_pad * cfg.width + d.n_out_pad), "padded output layer");
  cudaError_t e = cudaMemcpy((void *)d.occ, occ.data(), 4 * occ.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void *)d.dist, dist.data(), dist.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { free_object(ctx, o); return cuda_fail(e, "upload occupancy"); }
  cudaMemset((void *)d.umma, 0, d.umma_bytes);
  cudaMemset((void *)d.umma_h, 0, d.umma_bytes);
  cudaMemset((void *)d.umma_lo, 0, d.umma_lo_bytes);
  if ((rc = upload_params(ctx, o, tab_src, mlp_src)) != LSNIF_OK) { free_object(ctx, o); return rc; }
  // kept mesh for training labels
  if (!desc->blob && desc->keep_mesh) {
    const lsnif_mesh &m = desc->mesh;
    std::vector<float> vn(3 * m.nv), alb(3 * cfg.n_mat, 0.5f);
    std::vector<int32_t> tm(m.nt, 0);
    if (m.vnormals) memcpy(vn.data(), m.vnormals, 12 * m.nv);
    if (m.tri_mat) memcpy(tm.data(), m.tri_mat, 4 * m.nt);
    if (m.mat_albedo) memcpy(alb.data(), m.mat_albedo, 12 * cfg.n_mat);
    size_t nvox = (size_t)cfg.V * cfg.V * cfg.V;
    std::vector<int32_t> start(nvox + 1, 0), list(pairs.size());
    for (auto &pr : pairs) start[pr.first + 1]++;
    for (size_t i = 0; i < nvox; ++i) start[i + 1] += start[i];
    {
      std::vector<int32_t> cur(start.begin(), start.end() - 1);
      for (auto &pr : pairs) list[cur[pr.first]++] = pr.second;
    }
    OALLOC(verts, const float *, 12 * m.nv, "mesh vertices");
    OALLOC(tris, const int32_t *, 12 * m.nt, "mesh triangles");
    OALLOC(vnormals, const float *, 12 * m.nv, "mesh normals");
    OALLOC(tri_mat, const int32_t *, 4 * m.nt, "mesh materials");
    OALLOC(albedo, const float *, 12 * cfg.n_mat, "material albedo");
    OALLOC(vox_start, const int32_t *, 4 * start.size(), "voxel triangle lists");
    OALLOC(vox_tris, const int32_t *, 4 * std::max<size_t>(list.size(), 1), "voxel triangle lists");
    cudaMemcpy((void *)d.verts, m.verts, 12 * m.nv, cudaMemcpyHostToDevice);
    cudaMemcpy((void *)d.tris, m.tris, 12 * m.nt, cudaMemcpyHostToDevice);
    cudaMemcpy((void *)d.vnormals, vn.data(), 12 * m.nv, cudaMemcpyHostToDevice);
    cudaMemcpy((void *)d.tri_mat, tm.data(), 4 * m.nt, cudaMemcpyHostToDevice);
    cudaMemcpy((void *)d.albedo, alb.data(), 12 * cfg.n_mat, cudaMemcpyHostToDevice);
    cudaMemcpy((void *)d.vox_start, start.data(), 4 * start.size(), cudaMemcpyHostToDevice);
    if (!list.empty()) cudaMemcpy((void *)d.vox_tris, list.data(), 4 * list.size(), cudaMemcpyHostToDevice);
    d.nt = m.nt;
  }
#undef OALLOC
  d.handle = o->handle;
  d.valid = 1;
  e = cudaMemcpy(ctx->d_objs + slot, &d, sizeof d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_object(ctx, o); return cuda_fail(e, "lsnif_load_object: upload"); }
  ctx->n_slots_used = std::max(ctx->n_slots_used, slot + 1);
  *out = o->handle;
  return LSNIF_OK;
}

Object *lsnif::find_object(lsnif_ctx *ctx, lsnif_obj h) {
  int s = (int)(h & 0xFFFFu) - 1;
  if (!ctx || s < 0 || s >= kMaxSlots || !ctx->slots[s] || ctx->slots[s]->handle != h) return nullptr;
  return ctx->slots[s];
}

extern "C" int lsnif_unload_object(lsnif_ctx *ctx, lsnif_obj h) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_unload_object: bad handle %u", h);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  free_object(ctx, o);
  return LSNIF_OK;
}

extern "C" int lsnif_get_object_info(lsnif_ctx *ctx, lsnif_obj h, lsnif_object_info *out) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_get_object_info: bad handle %u", h);
  if (!out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_get_object_info: out is NULL");
  memset(out, 0, sizeof *out);
  out->cfg = o->cfg;
  memcpy(out->bmin, o->bmin, 12);
  memcpy(out->bmax, o->bmax, 12);
  for (int l = 0; l < o->cfg.L; ++l) out->res[l] = o->res[l];
  int64_t occn = 0;
  for (uint32_t w : o->occ_host) occn += __builtin_popcount(w);
  out->n_occupied = occn;
  out->n_params_mlp = o->n_params_mlp;
  out->device_bytes = o->device_bytes;
  const lsnif_config &c = o->cfg;
  out->footprint_fp16_bytes = ((size_t)c.V * c.V * c.V) / 8 + 2 * (((size_t)c.L << c.log2_T) * c.F) +
                              2 * (size_t)o->n_params_mlp;
  out->kind = o->d.kind;
  out->n_triangles = o->d.nt;
  out->bvh_nodes = o->bvh_nodes;
  if (o->d.kind != 0) out->footprint_fp16_bytes = 0;
  return LSNIF_OK;
}

extern "C" int lsnif_save_object(lsnif_ctx *ctx, lsnif_obj h, void *buf, size_t *inout_len) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_save_object: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_save_object: object %u is a mesh object (no LSNIF state)", o->handle);
  if (!inout_len) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_save_object: inout_len is NULL");
  size_t need = blob_size(o);
  if (!buf) { *inout_len = need; return LSNIF_OK; }
  if (*inout_len < need) {
    *inout_len = need;
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_save_object: buffer of %zu bytes, need %zu", *inout_len, need);
  }
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  const lsnif_config &c = o->cfg;
  uint8_t *b = (uint8_t *)buf;
  memcpy(b, kMagic, 8);
  uint64_t ver = kBlobVersion;
  memcpy(b + 8, &ver, 8);
  memcpy(b + 16, &c, sizeof c);
  uint8_t *p = b + 16 + sizeof c;
  memcpy(p, o->bmin, 12);
  memcpy(p + 12, o->bmax, 12);
  p += 24;
  memcpy(p, o->res.data(), 4 * c.L);
  p += 4 * c.L;
  memcpy(p, o->occ_host.data(), 4 * o->occ_host.size());
  p += 4 * o->occ_host.size();
  size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  cudaError_t e = cudaMemcpy(p, o->d.tab32, 4 * nt, cudaMemcpyDeviceToHost);
  p += 4 * nt;
  if (e == cudaSuccess) e = cudaMemcpy(p, o->d.mlp32, 4 * o->n_params_mlp, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_save_object: download");
  p += 4 * o->n_params_mlp;
  uint64_t hsum = fnv1a(b, (size_t)(p - b));
  memcpy(p, &hsum, 8);
  *inout_len = need;
  return LSNIF_OK;
}

extern "C" int lsnif_read_params(lsnif_ctx *ctx, lsnif_obj h, int which, void *dst, size_t bytes) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_read_params: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_read_params: object %u is a mesh object (no LSNIF state)", o->handle);
  if (!dst) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_read_params: dst is NULL");
  cudaSetDevice(ctx->device);
  const lsnif_config &c = o->cfg;
  size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  const void *src = nullptr;
  size_t need = 0;
  switch (which) {
    case LSNIF_PARAM_OCCUPANCY: src = o->d.occ; need = 4 * o->occ_host.size(); break;
    case LSNIF_PARAM_TABLES: src = o->d.tab32; need = 4 * nt; break;
    case LSNIF_PARAM_MLP: src = o->d.mlp32; need = 4 * o->n_params_mlp; break;
    case LSNIF_PARAM_GRAD_TABLES: src = o->tb.grad_tab; need = 4 * nt; break;
    case LSNIF_PARAM_GRAD_MLP: src = o->tb.grad_mlp; need = 4 * o->n_params_mlp; break;
    default: return fail(LSNIF_ERR_INVALID_ARG, "lsnif_read_params: unknown array %d", which);
  }
  if (!src) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_read_params: no gradients yet (run lsnif_train_step)");
  if (bytes != need) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_read_params: %zu bytes, array has %zu", bytes, need);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_read_params");
  return LSNIF_OK;
}

extern "C" int lsnif_write_params(lsnif_ctx *ctx, lsnif_obj h, int which, const void *src, size_t bytes) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_write_params: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_write_params: object %u is a mesh object (no LSNIF state)", o->handle);
  if (!src) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_write_params: src is NULL");
  cudaSetDevice(ctx->device);
  const lsnif_config &c = o->cfg;
  size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  cudaDeviceSynchronize();
  int rc;
  if (which == LSNIF_PARAM_TABLES) {
    if (bytes != 4 * nt) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_write_params: %zu bytes, tables have %zu", bytes, 4 * nt);
    rc = upload_params(ctx, o, (const float *)src, nullptr);
  } else if (which == LSNIF_PARAM_MLP) {
    if (bytes != 4 * (size_t)o->n_params_mlp) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_write_params: size mismatch");
    rc = upload_params(ctx, o, nullptr, (const float *)src);
  } else {
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_write_params: array %d is read-only", which);
  }
  if (rc) return rc;
  reset_optimizer(ctx, o);
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_write_params");
}
