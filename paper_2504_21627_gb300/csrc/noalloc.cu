// lsnif_query_rays_noalloc: the BF16 fused query with its scratch in a
// fixed, file-scope device array instead of memory the library allocates.
//
// Some callers cannot allocate device memory while they run: a renderer
// whose frame loop forbids cudaMalloc/cudaFree (both can synchronise the
// whole device and stall the frame), a plug-in inside a host engine that owns
// every allocation, or a service that fixes its memory at start-up. This
// entry point runs the same traversal, grouping and fused kernels as
// lsnif_query_rays at BF16 (with the context's traversal and grouping
// choices), but points their scratch (boundary points, ray intervals,
// grouping and tile tables) at the array below. It calls no cudaMalloc,
// cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

namespace {

// Upper bound of the static scratch. Every GPU that loads the library holds
// this much device memory until the process exits.
constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB

// The scratch itself. In host code this name is only a host-side stand-in;
// kernels need the device address that cudaGetSymbolAddress returns.
__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the scratch's device address.
int scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_noalloc: device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(LSNIF_ERR_CUDA, "lsnif_query_rays_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return LSNIF_OK;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int lsnif_query_rays_noalloc(lsnif_ctx *ctx, const lsnif_rays *r, lsnif_hits *h, void *stream) {
  if (!ctx || !r || !h) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_noalloc: NULL argument");
  if (r->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_noalloc: n < 0");
  // sizes below are computed in size_t from n; bound n first, as the regular query does
  if (r->n > ((int64_t)1 << 31) - 1)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_noalloc: n = %lld exceeds 2^31-1", (long long)r->n);
  if (r->n == 0) return LSNIF_OK;
  if (!r->ox || !r->oy || !r->oz || !r->dx || !r->dy || !r->dz || !r->tmin || !r->tmax)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_query_rays_noalloc: every ray array must be given");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(LSNIF_ERR_CUDA, "lsnif_query_rays_noalloc: device");

  // the objects the rays may name, and the shape the kernels need
  int H = 0, n_slots = std::max(ctx->n_slots_used, 1);
  const Object *rep = nullptr;
  uint32_t umma_max = 0, umma_lo_max = 0;
  bool mixed = false;
  bool mesh = false;
  auto add = [&](const Object *o) {
    if (o->d.kind != 0) {
      mesh = true;
      return;
    }
    H = std::max(H, o->cfg.H);
    umma_max = std::max(umma_max, o->d.umma_bytes);
    umma_lo_max = std::max(umma_lo_max, o->d.umma_lo_bytes);
    if (!rep) rep = o;
    else if (rep->d.F != o->d.F || rep->d.width != o->d.width || o->d.L > 16) mixed = true;
  };
  if (!r->obj) {
    const Object *o = find_object(ctx, r->single_obj);
    if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_query_rays_noalloc: bad object handle %u", r->single_obj);
    add(o);
  } else {
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) add(ctx->slots[s]);
    if (!rep && !mesh) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_query_rays_noalloc: no objects are loaded");
  }
  if (mesh || !rep)
    return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_query_rays_noalloc: mesh objects are answered by lsnif_query_rays");
  DevObject hobj = rep->d;
  hobj.umma_bytes = umma_max;
  hobj.umma_lo_bytes = umma_lo_max;
  if (mixed || !fused_supported(hobj) || fused_smem_bytes(hobj, H, false) > 232448)
    return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_query_rays_noalloc: objects outside the fused BF16 kernel's shapes");

  // carve the static scratch; reject what does not fit
  const int64_t n = r->n;
  // the counting sorts' bins take 8 MiB of the scratch
  const bool spatial = ctx->group_mode == 2 || ctx->trace_mode == 2;
  const int max_tiles = (int)(n / kTileM + n_slots + 1);
  const size_t need = al256((size_t)n * H * 12) + al256((size_t)n * 8) + al256((size_t)n) + al256((size_t)n * 4) +
                      al256((size_t)n * 2) +
                      al256((size_t)n * 4) + 3 * al256((size_t)n_slots * kBuckets * 4) +
                      al256((size_t)max_tiles * 12) + al256(64 * 4) + al256((size_t)(n / kGroupBlock + 2) * 8) +
                      (spatial ? al256((size_t)kBinsAlloc * 4) + al256((size_t)kBinSumsAlloc * 4) : 0);
  if (need > kNoAllocBytes)
    return fail(LSNIF_ERR_INVALID_ARG,
                "lsnif_query_rays_noalloc: %lld rays need %zu bytes of scratch but the static scratch holds %zu "
                "(split the batch, or use lsnif_query_rays)",
                (long long)n, need, kNoAllocBytes);
  void *base = nullptr;
  int rc = scratch_address(ctx->device, &base);
  if (rc) return rc;
  uint8_t *p = reinterpret_cast<uint8_t *>(base);
  auto take = [&](size_t bytes) {
    uint8_t *q = p;
    p += al256(bytes);
    return q;
  };
  QueryScratch s{};
  s.pts = reinterpret_cast<float *>(take((size_t)n * H * 12));
  s.t01 = reinterpret_cast<float *>(take((size_t)n * 8));
  s.k = take((size_t)n);
  s.dup = reinterpret_cast<uint32_t *>(take((size_t)n * 4));
  s.slot = reinterpret_cast<int16_t *>(take((size_t)n * 2));
  s.order = reinterpret_cast<int32_t *>(take((size_t)n * 4));
  s.counts = reinterpret_cast<int32_t *>(take((size_t)n_slots * kBuckets * 4));
  s.offsets = reinterpret_cast<int32_t *>(take((size_t)n_slots * kBuckets * 4));
  s.cursor = reinterpret_cast<int32_t *>(take((size_t)n_slots * kBuckets * 4));
  s.tiles = reinterpret_cast<int32_t *>(take((size_t)max_tiles * 12));
  s.meta = reinterpret_cast<int32_t *>(take(64 * 4));
  s.blk = reinterpret_cast<int32_t *>(take((size_t)(n / kGroupBlock + 2) * 8));
  if (spatial) {
    s.bins = reinterpret_cast<int32_t *>(take((size_t)kBinsAlloc * 4));
    s.bin_sums = reinterpret_cast<int32_t *>(take((size_t)kBinSumsAlloc * 4));
  }
  s.X = nullptr;
  s.max_tiles = max_tiles;
  s.wmax = 0;

  QueryLaunch q{};
  q.objs = ctx->d_objs;
  q.n_slots = n_slots;
  q.H_max = H;
  q.rays = RaysArg{r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->tmin, r->tmax, r->obj, r->single_obj, n};
  q.hits = HitsArg{h->hit, h->t, h->nx, h->ny, h->nz, h->mat, h->ar, h->ag, h->ab, h->logits};
  q.s = s;
  q.err = ctx->d_err;
  q.stream = (cudaStream_t)stream;
  q.trace_mode = ctx->trace_mode;
  q.group_mode = ctx->group_mode == 2 ? 3 : ctx->group_mode == 1 ? (r->obj ? 2 : 1) : 0;
  q.single_slot = r->obj ? 0 : rep->slot;
  // The bucket counts must start at zero: launch_trace clears them on the
  // stream; the grouping kernel resets the cursors and the tile counter.
  int launches = 0;
  cudaError_t e = launch_trace(q, &launches);
  if (e == cudaSuccess) e = launch_group(q, &launches);
  if (e == cudaSuccess) e = launch_fused(q, hobj, ctx->fused_variant, false, &launches);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_query_rays_noalloc");
  return LSNIF_OK;
}
