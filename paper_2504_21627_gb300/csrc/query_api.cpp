// Query orchestration behind lsnif_query_rays: scratch workspaces, the
// launch sequence of either precision, host-buffer queries, the stage entry
// points used to check each kernel on its own, and profiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

namespace {

constexpr int kChunkTiles = 1024;  // FP32 path: tiles whose features are materialised at once

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

struct Carve {
  uint8_t *p;
  template <class T>
  T *take(size_t bytes) {
    T *r = reinterpret_cast<T *>(p);
    p += al(bytes);
    return r;
  }
};

int max_tiles_for(int64_t n, int n_slots) { return (int)(n / kTileM + n_slots + 1); }

}  // namespace

size_t lsnif::workspace_bytes(int64_t n, int H, int n_slots, int n_in) {
  const int mt = max_tiles_for(n, n_slots);
  size_t b = al((size_t)n * H * 12) + al((size_t)n * 8) + al((size_t)n) + al((size_t)n * 4) + al((size_t)n * 2) +
             al((size_t)n * 4) +
             3 * al((size_t)n_slots * kBuckets * 4) + al((size_t)mt * 12) + al(64 * 4) +
             al((size_t)(n / kGroupBlock + 2) * 8) + al((size_t)kBinsAlloc * 4) +
             al((size_t)kBinSumsAlloc * 4);
  if (n_in > 0) b += al((size_t)std::min(mt, kChunkTiles) * kTileM * n_in * 4);
  return b;
}

int lsnif::ensure_workspace(lsnif_ctx *ctx, Workspace *ws, int64_t n, int H, int n_slots, int n_in) {
  if (ws->base && n <= ws->cap_rays && H <= ws->cap_H && n_slots <= ws->cap_slots && n_in <= ws->cap_nin)
    return LSNIF_OK;
  const int64_t nn = std::max(n, ws->cap_rays);
  const int HH = std::max(H, ws->cap_H), SS = std::max(n_slots, ws->cap_slots), NI = std::max(n_in, ws->cap_nin);
  const size_t bytes = workspace_bytes(nn, HH, SS, NI);
  if (ws->base) {
    cudaDeviceSynchronize();  // the old scratch may still be in use by queued work
    if (ctx->graphs_ws == ws->base) clear_graphs(ctx);
    dev_free(ctx, ws->base);
    ws->base = nullptr;
  }
  int rc = dev_alloc(ctx, bytes, &ws->base, "query scratch");
  if (rc) {
    ws->cap_rays = ws->cap_H = ws->cap_slots = ws->cap_nin = 0;
    return rc;
  }
  ws->bytes = bytes;
  ws->cap_rays = nn;
  ws->cap_H = HH;
  ws->cap_slots = SS;
  ws->cap_nin = NI;
  return LSNIF_OK;
}

void lsnif::free_workspace(lsnif_ctx *ctx, Workspace *ws) {
  if (ws->base) dev_free(ctx, ws->base);
  if (ws->stage) dev_free(ctx, ws->stage);
  *ws = Workspace{};
}

static QueryScratch carve(Workspace *ws, int64_t n, int H, int n_slots, int n_in) {
  // carve with the workspace's capacity so pointers stay valid for any
  // request that fits it
  const int64_t N = ws->cap_rays;
  const int HH = ws->cap_H, SS = ws->cap_slots;
  (void)n; (void)H; (void)n_slots; (void)n_in;
  Carve c{reinterpret_cast<uint8_t *>(ws->base)};
  QueryScratch s{};
  s.pts = c.take<float>((size_t)N * HH * 12);
  s.t01 = c.take<float>((size_t)N * 8);
  s.k = c.take<uint8_t>((size_t)N);
  s.dup = c.take<uint32_t>((size_t)N * 4);
  s.slot = c.take<int16_t>((size_t)N * 2);
  s.order = c.take<int32_t>((size_t)N * 4);
  s.counts = c.take<int32_t>((size_t)SS * kBuckets * 4);
  s.offsets = c.take<int32_t>((size_t)SS * kBuckets * 4);
  s.cursor = c.take<int32_t>((size_t)SS * kBuckets * 4);
  const int mt = max_tiles_for(N, SS);
  s.tiles = c.take<int32_t>((size_t)mt * 12);
  s.meta = c.take<int32_t>(64 * 4);
  s.blk = c.take<int32_t>((size_t)(N / kGroupBlock + 2) * 8);
  s.bins = c.take<int32_t>((size_t)kBinsAlloc * 4);
  s.bin_sums = c.take<int32_t>((size_t)kBinSumsAlloc * 4);
  s.X = ws->cap_nin > 0 ? c.take<float>((size_t)std::min(mt, kChunkTiles) * kTileM * ws->cap_nin * 4) : nullptr;
  s.max_tiles = max_tiles_for(n, n_slots);
  return s;
}

// Objects a query can touch and the shape parameters its kernels need.
struct Shape {
  int H = 0, n_in = 0, wmax = 0, n_slots = 0;
  const Object *rep = nullptr;   // representative object (fused: F/width)
  uint32_t umma_max = 0, umma_lo_max = 0;
  bool mixed_fused = false;      // objects differ in F or width
  bool has_mesh = false;         // some object of the batch is a mesh object
};

static int shape_of(lsnif_ctx *ctx, const lsnif_rays *r, Shape *sh) {
  auto add = [&](const Object *o) {
    if (o->d.kind != 0) {  // mesh objects take no part in the LSNIF launches
      sh->has_mesh = true;
      return;
    }
    sh->H = std::max(sh->H, o->cfg.H);
    sh->n_in = std::max(sh->n_in, o->d.n_in);
    sh->wmax = std::max(sh->wmax, std::max(o->d.width, o->d.n_out_pad));
    sh->umma_max = std::max(sh->umma_max, o->d.umma_bytes);
    sh->umma_lo_max = std::max(sh->umma_lo_max, o->d.umma_lo_bytes);
    if (!sh->rep) sh->rep = o;
    else if (sh->rep->d.F != o->d.F || sh->rep->d.width != o->d.width || o->d.L > 16) sh->mixed_fused = true;
  };
  if (!r->obj) {
    const Object *o = find_object(ctx, r->single_obj);
    if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "query: bad object handle %u", r->single_obj);
    add(o);
  } else {
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) add(ctx->slots[s]);
    if (!sh->rep && !sh->has_mesh) return fail(LSNIF_ERR_BAD_HANDLE, "query: no objects are loaded");
  }
  sh->n_slots = std::max(ctx->n_slots_used, 1);
  return LSNIF_OK;
}

static int check_rays(const lsnif_rays *r, const lsnif_hits *h) {
  if (!r || !h) return fail(LSNIF_ERR_INVALID_ARG, "query: rays or hits is NULL");
  if (r->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "query: n = %lld", (long long)r->n);
  if (r->n > ((int64_t)1 << 31) - 1) return fail(LSNIF_ERR_INVALID_ARG, "query: n = %lld exceeds 2^31-1", (long long)r->n);
  if (r->n > 0 && (!r->ox || !r->oy || !r->oz || !r->dx || !r->dy || !r->dz || !r->tmin || !r->tmax))
    return fail(LSNIF_ERR_INVALID_ARG, "query: every ray array must be given");
  return LSNIF_OK;
}

// Build (or refresh) the FP8 networks of every object the rays may name. It
// synchronises `st` when a network is stale, so it runs before any capture.
static int ensure_fp8_for(lsnif_ctx *ctx, const lsnif_rays *r, cudaStream_t st) {
  int rc;
  if (!r->obj) {
    Object *o = find_object(ctx, r->single_obj);
    if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "query: bad object handle %u", r->single_obj);
    return o->d.kind != 0 ? LSNIF_OK : ensure_fp8(ctx, o, st);
  }
  for (int s = 0; s < ctx->n_slots_used; ++s)
    if (ctx->slots[s] && ctx->slots[s]->d.kind == 0 && (rc = ensure_fp8(ctx, ctx->slots[s], st))) return rc;
  return LSNIF_OK;
}

int lsnif::run_query(lsnif_ctx *ctx, Workspace *ws, const lsnif_rays *r, lsnif_hits *h, int precision,
                     cudaStream_t st, bool profile, int *err) {
  if (!err) err = ctx->d_err;
  int rc = check_rays(r, h);
  if (rc) return rc;
  if (!valid_precision(precision)) return fail(LSNIF_ERR_INVALID_ARG, "query: unknown precision %d", precision);
  if (r->n == 0) return LSNIF_OK;
  Shape sh;
  if ((rc = shape_of(ctx, r, &sh))) return rc;
  if (!sh.rep) {  // mesh objects only: the BVH query alone
    QueryLaunch q{};
    q.objs = ctx->d_objs;
    q.n_slots = sh.n_slots;
    q.rays = RaysArg{r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->tmin, r->tmax, r->obj, r->single_obj, r->n};
    q.hits = HitsArg{h->hit, h->t, h->nx, h->ny, h->nz, h->mat, h->ar, h->ag, h->ab, h->logits};
    q.err = err;
    q.stream = st;
    int launches = 0;
    cudaError_t e = launch_mesh_query(q, &launches);
    if (profile) {
      ctx->prof = lsnif_profile{};
      ctx->prof.n_rays = r->n;
      ctx->prof.launches = launches;
      ctx->prof_valid = false;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mesh query launch");
    return LSNIF_OK;
  }
  if (precision == LSNIF_FP8_FUSED) {
    if ((rc = ensure_fp8_for(ctx, r, st))) return rc;
    if ((rc = shape_of(ctx, r, &(sh = Shape{})))) return rc;
  }
  DevObject rep = sh.rep->d;
  if (precision == LSNIF_FP8_FUSED) {
    uint32_t b8 = 0;
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) b8 = std::max(b8, ctx->slots[s]->d.blob8_bytes);
    rep.blob8_bytes = std::max(rep.blob8_bytes, r->obj ? b8 : 0u);
    if (sh.mixed_fused || !fused8_supported(rep) || fused8_smem_bytes(rep, sh.H) > 232448)
      return fail(LSNIF_ERR_UNSUPPORTED, "query: the fused FP8 path needs F in {2,4}, width 64/128, L <= 16, "
                                         "L*F a multiple of 16 and one shape for all objects");
  }
  bool streamed = false;  // FP16 with the weights streamed (networks too large for shared memory)
  if (fused16_precision(precision)) {
    rep.umma_bytes = sh.umma_max;
    rep.umma_lo_bytes = sh.umma_lo_max;
    if (sh.mixed_fused || !fused_supported(rep) || fused_smem_bytes(rep, sh.H, precision == LSNIF_FP16_FUSED) > 232448) {
      streamed = precision == LSNIF_FP16_FUSED && !sh.mixed_fused && fused16s_supported(rep) &&
                 fused16s_smem_bytes(rep, sh.H) <= 232448;
      if (!streamed)
        return fail(LSNIF_ERR_UNSUPPORTED, "query: the fused BF16/FP16 path needs F in {2,4}, width 64/128, L <= 16 "
                                           "and one shape for all objects; BF16 also weights that fit shared memory");
    }
  }
  const int n_in = precision == LSNIF_FP32_PLAIN ? sh.n_in : 0;
  if ((rc = ensure_workspace(ctx, ws, r->n, sh.H, sh.n_slots, n_in))) return rc;
  QueryLaunch q{};
  q.objs = ctx->d_objs;
  q.n_slots = sh.n_slots;
  q.H_max = ws->cap_H;
  q.rays = RaysArg{r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->tmin, r->tmax, r->obj, r->single_obj, r->n};
  q.hits = HitsArg{h->hit, h->t, h->nx, h->ny, h->nz, h->mat, h->ar, h->ag, h->ab, h->logits};
  q.s = carve(ws, r->n, sh.H, sh.n_slots, n_in);
  q.s.wmax = sh.wmax;
  q.err = err;
  q.stream = st;
  q.trace_mode = ctx->trace_mode;
  q.group_mode = ctx->group_mode == 2 ? 3 : ctx->group_mode == 1 ? (r->obj ? 2 : 1) : 0;
  q.single_slot = r->obj ? 0 : sh.rep->slot;
  int launches = 0;
  if (profile) cudaEventRecord(ctx->ev[0], st);
  cudaError_t e = launch_trace(q, &launches);
  if (profile) cudaEventRecord(ctx->ev[1], st);
  if (e == cudaSuccess) e = launch_group(q, &launches);
  if (profile) cudaEventRecord(ctx->ev[2], st);
  if (e == cudaSuccess) {
    if (precision == LSNIF_FP32_PLAIN) e = launch_plain_tail(q, ws->cap_nin, kChunkTiles, &launches);
    else if (precision == LSNIF_FP8_FUSED) e = launch_fused8(q, rep, ctx->fp8_variant, &launches);
    else if (streamed) e = launch_fused16s(q, rep, &launches);
    else
      e = launch_fused(q, rep, precision == LSNIF_FP16_FUSED ? ctx->fused_variant16 : ctx->fused_variant,
                       precision == LSNIF_FP16_FUSED, &launches);
  }
  // rays on mesh objects were answered as misses by the traversal (no
  // voxels); their BVH query overwrites them
  if (e == cudaSuccess && sh.has_mesh) e = launch_mesh_query(q, &launches);
  if (profile) {
    cudaEventRecord(ctx->ev[3], st);
    cudaMemcpyAsync(ctx->d_prof_meta, q.s.meta, 16, cudaMemcpyDeviceToDevice, st);
    ctx->prof_stream = st;
    ctx->prof = lsnif_profile{};
    ctx->prof.n_rays = r->n;
    ctx->prof.launches = launches + 1;  // + the counts reset
    ctx->prof_valid = true;
  }
  if (e != cudaSuccess) return cuda_fail(e, "query launch");
  return LSNIF_OK;
}

void lsnif::clear_graphs(lsnif_ctx *ctx) {
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
  ctx->graphs_ws = nullptr;
}

// Replay a captured graph of this exact query, capturing it first. The key
// holds everything the launch sequence depends on; the scratch must already
// be large enough so that nothing is allocated while capturing.
static int query_graph(lsnif_ctx *ctx, const lsnif_rays *r, lsnif_hits *h, int precision, cudaStream_t st) {
  int rc = check_rays(r, h);
  if (rc) return rc;
  if (r->n == 0) return LSNIF_OK;
  if (precision == LSNIF_FP8_FUSED && (rc = ensure_fp8_for(ctx, r, st))) return rc;
  Shape sh;
  if ((rc = shape_of(ctx, r, &sh))) return rc;
  if (!sh.rep) return run_query(ctx, &ctx->ws, r, h, precision, st, false);
  const int n_in = precision == LSNIF_FP32_PLAIN ? sh.n_in : 0;
  if ((rc = ensure_workspace(ctx, &ctx->ws, r->n, sh.H, sh.n_slots, n_in))) return rc;
  if (ctx->graphs_ws != ctx->ws.base) clear_graphs(ctx);
  std::vector<uint64_t> key = {(uint64_t)r->n, (uint64_t)precision,
                               (uint64_t)(precision == LSNIF_FP8_FUSED    ? 1000 + ctx->fp8_variant
                                          : precision == LSNIF_FP16_FUSED ? 2000 + ctx->fused_variant16
                                                                          : ctx->fused_variant),
                               (uint64_t)ctx->trace_mode, (uint64_t)ctx->group_mode, (uint64_t)sh.n_slots,
                               (uint64_t)r->single_obj};
  for (const void *p : {(const void *)r->ox, (const void *)r->oy, (const void *)r->oz, (const void *)r->dx,
                        (const void *)r->dy, (const void *)r->dz, (const void *)r->tmin, (const void *)r->tmax,
                        (const void *)r->obj, (const void *)h->hit, (const void *)h->t, (const void *)h->nx,
                        (const void *)h->ny, (const void *)h->nz, (const void *)h->mat, (const void *)h->ar,
                        (const void *)h->ag, (const void *)h->ab, (const void *)h->logits})
    key.push_back((uint64_t)(uintptr_t)p);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "lsnif_query_rays: begin graph capture");
    rc = run_query(ctx, &ctx->ws, r, h, precision, st, false);
    e = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "lsnif_query_rays: end graph capture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "lsnif_query_rays: instantiate graph");
    it = ctx->graphs.emplace(key, ex).first;
    ctx->graphs_ws = ctx->ws.base;
  }
  cudaError_t e = cudaGraphLaunch(it->second, st);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_query_rays: graph launch");
}

extern "C" int lsnif_query_rays(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                                void *stream) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays: ctx is NULL");
  cudaSetDevice(ctx->device);
  if (ctx->graph_mode && !ctx->profiling && stream != nullptr)
    return query_graph(ctx, rays, hits, precision, (cudaStream_t)stream);
  return run_query(ctx, &ctx->ws, rays, hits, precision, (cudaStream_t)stream, ctx->profiling);
}

extern "C" int lsnif_set_graph_mode(lsnif_ctx *ctx, int on) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_graph_mode: ctx is NULL");
  cudaSetDevice(ctx->device);
  ctx->graph_mode = on != 0;
  if (!on) clear_graphs(ctx);
  return LSNIF_OK;
}

// Host-buffer query, pipelined: the batch is cut into up to 4 chunks of at
// least 2^20 rays; chunk c's rays are copied in on one copy stream, queried on
// the caller's stream and its results copied out on a second copy stream, so
// the copies of neighbouring chunks overlap the query of chunk c (the two
// copy directions also overlap each other). Synchronous: returns once every
// result is in host memory.
extern "C" int lsnif_set_host_mode(lsnif_ctx *ctx, int mode) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_host_mode: ctx is NULL");
  if (mode != LSNIF_HOST_STAGED && mode != LSNIF_HOST_DIRECT)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_host_mode: unknown mode %d", mode);
  ctx->host_mode = mode;
  return LSNIF_OK;
}

// The device address of a page-locked, mapped host buffer (the same address
// under unified addressing), or NULL when p is not one (pageable memory,
// device memory) or is NULL.
static void *mapped_host(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Direct host-buffer query: every given buffer is page-locked host memory
// that the kernels read and write through its mapped address (on GB300 the
// host memory is reached over the coherent NVLink-C2C link), so nothing is
// staged or copied. Returns 1 (not done) when some buffer is not
// page-locked; the caller then stages.
static int query_host_direct(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                             cudaStream_t st, int *rc) {
  lsnif_rays dr = *rays;
  lsnif_hits dh = *hits;
  const float **rin[8] = {&dr.ox, &dr.oy, &dr.oz, &dr.dx, &dr.dy, &dr.dz, &dr.tmin, &dr.tmax};
  for (auto pp : rin)
    if (!(*pp = static_cast<const float *>(mapped_host(*pp)))) return 1;
  if (rays->obj && !(dr.obj = static_cast<const uint32_t *>(mapped_host(rays->obj)))) return 1;
  float **fout[8] = {&dh.t, &dh.nx, &dh.ny, &dh.nz, &dh.ar, &dh.ag, &dh.ab, &dh.logits};
  for (auto pp : fout)
    if (*pp && !(*pp = static_cast<float *>(mapped_host(*pp)))) return 1;
  if (hits->hit && !(dh.hit = static_cast<uint8_t *>(mapped_host(hits->hit)))) return 1;
  if (hits->mat && !(dh.mat = static_cast<int32_t *>(mapped_host(hits->mat)))) return 1;
  *rc = run_query(ctx, &ctx->ws, &dr, &dh, precision, st, ctx->profiling);
  if (*rc == LSNIF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) *rc = cuda_fail(e, "lsnif_query_rays_host");
  }
  return 0;
}

extern "C" int lsnif_query_rays_host(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                                     void *stream) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_host: ctx is NULL");
  int rc = check_rays(rays, hits);
  if (rc) return rc;
  if (rays->n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (hits->logits && rays->obj)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_host: logits need a single object");
  if (ctx->host_mode == LSNIF_HOST_DIRECT && query_host_direct(ctx, rays, hits, precision, st, &rc) == 0) return rc;
  Shape sh;
  if ((rc = shape_of(ctx, rays, &sh))) return rc;
  const int64_t n = rays->n;
  int n_out_q = 0;
  if (hits->logits) {
    if (rays->obj) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_host: logits need a single object");
    n_out_q = sh.rep->d.n_out;
  }
  const size_t need = al(n * 4) * 8 + al(n * 4) + al(n) + al(n * 4) * 8 + al(n * 4) + al((size_t)n * 4 * n_out_q);
  Workspace *ws = &ctx->ws;
  if (ws->stage_bytes < need) {
    if (ws->stage) {
      cudaDeviceSynchronize();
      dev_free(ctx, ws->stage);
      ws->stage = nullptr;
      ws->stage_bytes = 0;
    }
    if ((rc = dev_alloc(ctx, need, &ws->stage, "host-query staging"))) return rc;
    ws->stage_bytes = need;
  }
  if (!ctx->copy_in) {
    if (cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(LSNIF_ERR_CUDA, "lsnif_query_rays_host: cannot create copy streams");
    }
    for (auto &ev : ctx->hev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(LSNIF_ERR_CUDA, "lsnif_query_rays_host: cannot create events");
      }
  }
  // device staging for the whole batch (each chunk uses its own slice)
  Carve c{reinterpret_cast<uint8_t *>(ws->stage)};
  const float *src[8] = {rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax};
  float *dray[8];
  for (int i = 0; i < 8; ++i) dray[i] = c.take<float>(n * 4);
  uint32_t *dobj = c.take<uint32_t>(n * 4);
  uint8_t *dhit = hits->hit ? c.take<uint8_t>(n) : nullptr;
  float *hf_src[7] = {hits->t, hits->nx, hits->ny, hits->nz, hits->ar, hits->ag, hits->ab};
  float *dhf[7];
  for (int i = 0; i < 7; ++i) dhf[i] = hf_src[i] ? c.take<float>(n * 4) : nullptr;
  int32_t *dmat = hits->mat ? c.take<int32_t>(n * 4) : nullptr;
  float *dlog = hits->logits ? c.take<float>((size_t)n * 4 * n_out_q) : nullptr;

  const int64_t kMinChunk = int64_t(1) << 20;
  const int n_chunks = (int)std::max<int64_t>(1, std::min<int64_t>(4, n / kMinChunk));
  const int64_t chunk = (n + n_chunks - 1) / n_chunks;
  // the copies start after the caller's earlier work on its stream
  cudaError_t e = cudaEventRecord(ctx->hev[15], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_in, ctx->hev[15], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_out, ctx->hev[15], 0);
  for (int k = 0; k < n_chunks && e == cudaSuccess; ++k) {
    const int64_t off = k * chunk, len = std::min(chunk, n - off);
    cudaEvent_t ev_in = ctx->hev[2 * k], ev_done = ctx->hev[2 * k + 1];
    for (int i = 0; i < 8 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(dray[i] + off, src[i] + off, len * 4, cudaMemcpyHostToDevice, ctx->copy_in);
    if (rays->obj && e == cudaSuccess)
      e = cudaMemcpyAsync(dobj + off, rays->obj + off, len * 4, cudaMemcpyHostToDevice, ctx->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, ctx->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in, 0);
    if (e != cudaSuccess) break;
    lsnif_rays dr = *rays;
    dr.ox = dray[0] + off; dr.oy = dray[1] + off; dr.oz = dray[2] + off;
    dr.dx = dray[3] + off; dr.dy = dray[4] + off; dr.dz = dray[5] + off;
    dr.tmin = dray[6] + off; dr.tmax = dray[7] + off;
    dr.obj = rays->obj ? dobj + off : nullptr;
    dr.n = len;
    lsnif_hits dh{};
    dh.hit = dhit ? dhit + off : nullptr;
    float **dhf_dst[7] = {&dh.t, &dh.nx, &dh.ny, &dh.nz, &dh.ar, &dh.ag, &dh.ab};
    for (int i = 0; i < 7; ++i) *dhf_dst[i] = dhf[i] ? dhf[i] + off : nullptr;
    dh.mat = dmat ? dmat + off : nullptr;
    dh.logits = dlog ? dlog + (size_t)off * n_out_q : nullptr;
    if ((rc = run_query(ctx, ws, &dr, &dh, precision, st, ctx->profiling))) {
      cudaStreamSynchronize(ctx->copy_in);  // no copy may outlive the call
      cudaStreamSynchronize(ctx->copy_out);
      return rc;
    }
    e = cudaEventRecord(ev_done, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_out, ev_done, 0);
    if (hits->hit && e == cudaSuccess)
      e = cudaMemcpyAsync(hits->hit + off, dhit + off, len, cudaMemcpyDeviceToHost, ctx->copy_out);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i)
      if (hf_src[i]) e = cudaMemcpyAsync(hf_src[i] + off, dhf[i] + off, len * 4, cudaMemcpyDeviceToHost, ctx->copy_out);
    if (hits->mat && e == cudaSuccess)
      e = cudaMemcpyAsync(hits->mat + off, dmat + off, len * 4, cudaMemcpyDeviceToHost, ctx->copy_out);
    if (hits->logits && e == cudaSuccess)
      e = cudaMemcpyAsync(hits->logits + (size_t)off * n_out_q, dlog + (size_t)off * n_out_q,
                          (size_t)len * 4 * n_out_q, cudaMemcpyDeviceToHost, ctx->copy_out);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->hev[14], ctx->copy_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->hev[14], 0);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(ctx->copy_in);
    cudaStreamSynchronize(ctx->copy_out);
    return cuda_fail(e, "lsnif_query_rays_host: copies");
  }
  return check_device(ctx, st);
}

// ---- stage entry points ------------------------------------------------------

extern "C" int lsnif_trace(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_trace_out *out, void *stream) {
  if (!ctx || !rays || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_trace: NULL argument");
  Object *o = find_object(ctx, rays->single_obj);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_trace: bad handle %u", rays->single_obj);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_trace: object %u is a mesh object (no LSNIF state)", o->handle);
  lsnif_hits dummy{};
  int rc = check_rays(rays, &dummy);
  if (rc) return rc;
  if (rays->n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  RaysArg ra{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax, nullptr, o->handle,
             rays->n};
  cudaError_t e = launch_trace_only(ctx->d_objs + o->slot, ra, out->k, out->t01, out->pts, out->vox, ctx->d_err,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_trace");
}

extern "C" int lsnif_encode(lsnif_ctx *ctx, lsnif_obj h, const float *pts, int64_t n, float *feats, int precision,
                            void *stream) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_encode: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_encode: object %u is a mesh object (no LSNIF state)", o->handle);
  if (n < 0 || (n > 0 && (!pts || !feats))) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_encode: bad arguments");
  if (n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_encode(ctx->d_objs + o->slot, o->d, pts, n, feats, precision, (cudaStream_t)stream);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_encode");
}

extern "C" int lsnif_corner_indices(lsnif_ctx *ctx, lsnif_obj h, const float *pts, int64_t n, uint32_t *out,
                                    void *stream) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_corner_indices: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_corner_indices: object %u is a mesh object (no LSNIF state)", o->handle);
  if (n < 0 || (n > 0 && (!pts || !out))) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_corner_indices: bad arguments");
  if (n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_corners(ctx->d_objs + o->slot, o->d, pts, n, out, (cudaStream_t)stream);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_corner_indices");
}

extern "C" int lsnif_mlp(lsnif_ctx *ctx, lsnif_obj h, const float *X, int64_t n, float *Z, int precision,
                         void *stream) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_mlp: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_mlp: object %u is a mesh object (no LSNIF state)", o->handle);
  if (n < 0 || (n > 0 && (!X || !Z))) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_mlp: bad arguments");
  if (n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e;
  if (precision == LSNIF_FP32_PLAIN) {
    e = launch_mlp_plain(ctx->d_objs + o->slot, o->d, X, n, Z, (cudaStream_t)stream);
  } else if (fused16_precision(precision)) {
    if (!fused_supported(o->d) || fused_smem_bytes(o->d, o->d.H, precision == LSNIF_FP16_FUSED) > 232448)
      return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_mlp: shape not covered by the tensor-core kernel");
    e = launch_mlp_fused(ctx->d_objs + o->slot, o->d, X, n, Z, precision == LSNIF_FP16_FUSED, ctx->d_err,
                         (cudaStream_t)stream);
  } else {
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_mlp: unknown precision %d", precision);
  }
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_mlp");
}

// ---- profiling ---------------------------------------------------------------

extern "C" int lsnif_set_profiling(lsnif_ctx *ctx, int on) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_profiling: ctx is NULL");
  ctx->profiling = on != 0;
  return LSNIF_OK;
}

extern "C" int lsnif_last_profile(lsnif_ctx *ctx, lsnif_profile *out) {
  if (!ctx || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_last_profile: NULL argument");
  if (!ctx->prof_valid) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_last_profile: no profiled query yet");
  cudaSetDevice(ctx->device);
  int rc = check_device(ctx, ctx->prof_stream);
  if (rc) return rc;
  lsnif_profile p = ctx->prof;
  cudaEventElapsedTime(&p.ms_trace, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&p.ms_group, ctx->ev[1], ctx->ev[2]);
  cudaEventElapsedTime(&p.ms_mlp, ctx->ev[2], ctx->ev[3]);
  cudaEventElapsedTime(&p.ms_total, ctx->ev[0], ctx->ev[3]);
  p.ms_encode = 0.f;
  int32_t meta[4] = {0, 0, 0, 0};
  cudaMemcpy(meta, ctx->d_prof_meta, 16, cudaMemcpyDeviceToHost);
  p.n_live = meta[0];
  p.n_points = meta[2];
  *out = p;
  return LSNIF_OK;
}

// ---- autotuning --------------------------------------------------------------

extern "C" int lsnif_variant_count(void) { return fused_variant_count(); }

extern "C" int lsnif_variant_shape(int v, int *threads, int *levels) {
  if (v < 0 || v >= fused_variant_count() || !threads || !levels)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_variant_shape: bad variant %d", v);
  fused_variant_shape(v, threads, levels);
  return LSNIF_OK;
}

extern "C" int lsnif_set_variant(lsnif_ctx *ctx, int v) {
  if (!ctx || v < 0 || v >= fused_variant_count())
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_variant: bad variant %d", v);
  ctx->fused_variant = v;
  ctx->fused_variant16 = v;
  return LSNIF_OK;
}

extern "C" int lsnif_variant8_count(void) { return fused8_variant_count(); }

extern "C" int lsnif_variant8_shape(int v, int *threads, int *levels) {
  if (v < 0 || v >= fused8_variant_count() || !threads || !levels)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_variant8_shape: bad variant %d", v);
  fused8_variant_shape(v, threads, levels);
  return LSNIF_OK;
}

extern "C" int lsnif_set_variant8(lsnif_ctx *ctx, int v) {
  if (!ctx || v < 0 || v >= fused8_variant_count())
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_variant8: bad variant %d", v);
  ctx->fp8_variant = v;
  return LSNIF_OK;
}

extern "C" int lsnif_autotune(lsnif_ctx *ctx, const lsnif_rays *rays, int reps, void *stream, int *chosen) {
  if (!ctx || !rays || reps < 1) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_autotune: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  lsnif_hits none{};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int keep_v = ctx->fused_variant, keep_v16 = ctx->fused_variant16, keep_t = ctx->trace_mode,
            keep_g = ctx->group_mode;
  auto time_it = [&](float *ms, int precision = LSNIF_BF16_FUSED) -> int {
    int rc = run_query(ctx, &ctx->ws, rays, &none, precision, st, false);
    if (rc) return rc;
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && rc == LSNIF_OK; ++r) rc = run_query(ctx, &ctx->ws, rays, &none, precision, st, false);
    cudaEventRecord(b, st);
    if (rc) return rc;
    if ((rc = check_device(ctx, st))) return rc;
    cudaEventElapsedTime(ms, a, b);
    return LSNIF_OK;
  };
  int best = -1, rc = LSNIF_OK;
  float best_ms = 0.f;
  // the fused kernel's tile shape first, then the traversal kernel
  for (int v = 0; v < fused_variant_count() && rc == LSNIF_OK; ++v) {
    ctx->fused_variant = v;
    float ms = 0.f;
    if ((rc = time_it(&ms))) break;
    if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
  }
  int best_t = ctx->trace_mode, best_g = ctx->group_mode;
  if (rc == LSNIF_OK) {
    ctx->fused_variant = best;
    for (int t = 0; t < 3 && rc == LSNIF_OK; ++t) {
      if (t == best_t) continue;
      ctx->trace_mode = t;
      float ms = 0.f;
      if ((rc = time_it(&ms))) break;
      if (ms < best_ms) { best_t = t; best_ms = ms; }
    }
    ctx->trace_mode = best_t;
    // grouping: by (object, point count), rays kept in order within their
    // object, or sorted by the cell of their first point
    if (rc == LSNIF_OK) {
      for (int g = 0; g < 3 && rc == LSNIF_OK; ++g) {
        if (g == best_g) continue;
        ctx->group_mode = g;
        float ms = 0.f;
        if ((rc = time_it(&ms))) break;
        if (ms < best_ms) { best_g = g; best_ms = ms; }
      }
    }
  }
  // the FP16 kernel's shape on its own (its shared memory, so its L1, differs)
  int best16 = -1;
  if (rc == LSNIF_OK) {
    ctx->trace_mode = best_t;
    ctx->group_mode = best_g;
    float best16_ms = 0.f;
    for (int v = 0; v < fused_variant_count() && rc == LSNIF_OK; ++v) {
      ctx->fused_variant16 = v;
      float ms = 0.f;
      if ((rc = time_it(&ms, LSNIF_FP16_FUSED))) break;
      if (best16 < 0 || ms < best16_ms) { best16 = v; best16_ms = ms; }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) {
    ctx->fused_variant = keep_v;
    ctx->fused_variant16 = keep_v16;
    ctx->trace_mode = keep_t;
    ctx->group_mode = keep_g;
    return rc;
  }
  ctx->fused_variant = best;
  ctx->fused_variant16 = best16;
  ctx->trace_mode = best_t;
  ctx->group_mode = best_g;
  if (chosen) *chosen = best;
  return LSNIF_OK;
}

extern "C" int lsnif_get_tuning(lsnif_ctx *ctx, int *variant, int *trace_mode, int *group_mode) {
  if (!ctx || !variant || !trace_mode || !group_mode) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_get_tuning: NULL argument");
  *variant = ctx->fused_variant;
  *trace_mode = ctx->trace_mode;
  *group_mode = ctx->group_mode;
  return LSNIF_OK;
}

extern "C" int lsnif_set_group_mode(lsnif_ctx *ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_group_mode: bad mode %d", mode);
  ctx->group_mode = mode;
  return LSNIF_OK;
}

extern "C" int lsnif_set_trace_mode(lsnif_ctx *ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_set_trace_mode: bad mode %d", mode);
  ctx->trace_mode = mode;
  return LSNIF_OK;
}
