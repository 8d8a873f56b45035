// Training entry points: training-ray generation, ground-truth labels and the
// optimisation step, with the per-object optimiser state they keep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

void lsnif::free_train_state(lsnif_ctx *ctx, Object *o) {
  for (void *p : o->train_allocs) dev_free(ctx, p);
  o->train_allocs.clear();
  o->tb = TrainBuffers{};
  o->tb_batch = 0;
  o->step = 0;
}

void lsnif::reset_optimizer(lsnif_ctx *, Object *o) {
  if (!o->tb.m_mlp) return;
  const lsnif_config &c = o->cfg;
  const size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  cudaMemset(o->tb.m_mlp, 0, 4 * o->n_params_mlp);
  cudaMemset(o->tb.v_mlp, 0, 4 * o->n_params_mlp);
  cudaMemset(o->tb.m_tab, 0, 4 * nt);
  cudaMemset(o->tb.v_tab, 0, 4 * nt);
  o->step = 0;
}

static int train_alloc(lsnif_ctx *ctx, Object *o, size_t bytes, void **p, const char *what) {
  int rc = dev_alloc(ctx, bytes, p, what);
  if (rc == LSNIF_OK) o->train_allocs.push_back(*p);
  return rc;
}

// Size the batch buffers for B rays; the optimiser state survives regrowth.
static int ensure_train(lsnif_ctx *ctx, Object *o, int64_t B) {
  if (o->tb_batch >= B && o->tb.feats) return LSNIF_OK;
  cudaDeviceSynchronize();
  const lsnif_config &c = o->cfg;
  const size_t nt = ((size_t)c.L << c.log2_T) * c.F;
  TrainBuffers keep = o->tb;
  // batch-sized buffers are reallocated; optimiser state and gradients kept
  std::vector<void *> persistent;
  for (void *p : o->train_allocs) {
    if (p == keep.m_mlp || p == keep.v_mlp || p == keep.m_tab || p == keep.v_tab || p == keep.grad_mlp ||
        p == keep.grad_tab || p == keep.loss)
      persistent.push_back(p);
    else
      dev_free(ctx, p);
  }
  o->train_allocs = persistent;
  TrainBuffers &tb = o->tb;
  const int W = c.width, NI = o->d.n_in, NO = o->d.n_out;
  void *p;
  int rc;
#define TALLOC(field, type, bytes)                                                   \
  if ((rc = train_alloc(ctx, o, (bytes), &p, "training buffers")) != LSNIF_OK) return rc; \
  tb.field = (type)p;
  TALLOC(feats, float *, 4 * (size_t)B * NI);
  TALLOC(acts, float *, 4 * (size_t)B * W * c.n_hidden);
  TALLOC(pre, float *, 4 * (size_t)B * W * c.n_hidden);
  TALLOC(Z, float *, 4 * (size_t)B * NO);
  TALLOC(dZ, float *, 4 * (size_t)B * NO);
  TALLOC(dA, float *, 4 * (size_t)B * std::max(W, NI));
  TALLOC(dB, float *, 4 * (size_t)B * std::max(W, NI));
  TALLOC(pts, float *, 12 * (size_t)B * c.H);
  TALLOC(t01, float *, 8 * (size_t)B);
  TALLOC(k, int32_t *, 4 * (size_t)B);
  TALLOC(k8, uint8_t *, (size_t)B);
  TALLOC(dup, uint32_t *, 4 * (size_t)B);
  TALLOC(slot, int16_t *, 2 * (size_t)B);
  TALLOC(counts, int32_t *, 4 * (size_t)kMaxSlots * kBuckets);
  TALLOC(meta, int32_t *, 64);
  if (!keep.loss) {
    TALLOC(loss, float *, 64);
    TALLOC(grad_mlp, float *, 4 * (size_t)o->n_params_mlp);
    TALLOC(grad_tab, float *, 4 * nt);
    TALLOC(m_mlp, float *, 4 * (size_t)o->n_params_mlp);
    TALLOC(v_mlp, float *, 4 * (size_t)o->n_params_mlp);
    TALLOC(m_tab, float *, 4 * nt);
    TALLOC(v_tab, float *, 4 * nt);
    cudaMemset(tb.m_mlp, 0, 4 * o->n_params_mlp);
    cudaMemset(tb.v_mlp, 0, 4 * o->n_params_mlp);
    cudaMemset(tb.m_tab, 0, 4 * nt);
    cudaMemset(tb.v_tab, 0, 4 * nt);
    cudaMemset(tb.grad_mlp, 0, 4 * o->n_params_mlp);
    cudaMemset(tb.grad_tab, 0, 4 * nt);
  } else {
    tb.loss = keep.loss;
    tb.grad_mlp = keep.grad_mlp;
    tb.grad_tab = keep.grad_tab;
    tb.m_mlp = keep.m_mlp;
    tb.v_mlp = keep.v_mlp;
    tb.m_tab = keep.m_tab;
    tb.v_tab = keep.v_tab;
  }
#undef TALLOC
  o->tb_batch = B;
  return LSNIF_OK;
}

extern "C" int lsnif_make_training_rays(lsnif_ctx *ctx, lsnif_obj h, const float *u, int64_t n, int64_t n_outside,
                                        float *rays_out, uint8_t *surface, void *stream) {
  Object *o = find_object(ctx, h);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_make_training_rays: bad handle %u", h);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_make_training_rays: object %u is a mesh object (no LSNIF state)", o->handle);
  if (n < 0 || n_outside < 0 || n_outside > n || (n > 0 && (!u || !rays_out)))
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_make_training_rays: bad arguments");
  if (!o->d.vox_start)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_make_training_rays: load the object with keep_mesh = 1");
  if (n == 0) return LSNIF_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_make_training_rays(ctx->d_objs + o->slot, o->d, u, n, n_outside, rays_out, surface,
                                            (cudaStream_t)stream);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_make_training_rays");
}

extern "C" int lsnif_label_rays(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_labels *out, void *stream) {
  if (!ctx || !rays || !out) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_label_rays: NULL argument");
  Object *o = find_object(ctx, rays->single_obj);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_label_rays: bad handle %u", rays->single_obj);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_label_rays: object %u is a mesh object (no LSNIF state)", o->handle);
  if (!o->d.vox_start) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_label_rays: load the object with keep_mesh = 1");
  if (rays->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_label_rays: n < 0");
  if (rays->n == 0) return LSNIF_OK;
  if (!rays->ox || !rays->oy || !rays->oz || !rays->dx || !rays->dy || !rays->dz || !rays->tmin || !rays->tmax)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_label_rays: every ray array must be given");
  cudaSetDevice(ctx->device);
  RaysArg ra{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax, nullptr, o->handle,
             rays->n};
  cudaError_t e = launch_label_rays(ctx->d_objs + o->slot, o->d, ra, *out, (cudaStream_t)stream);
  return e == cudaSuccess ? LSNIF_OK : cuda_fail(e, "lsnif_label_rays");
}

extern "C" int lsnif_train_step(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_labels *labels,
                                const lsnif_train_opts *opts, lsnif_train_stats *stats, void *stream) {
  if (!ctx || !rays || !labels || !opts) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_train_step: NULL argument");
  Object *o = find_object(ctx, rays->single_obj);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_train_step: bad handle %u", rays->single_obj);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_train_step: object %u is a mesh object (no LSNIF state)", o->handle);
  if (rays->n <= 0 || rays->n > (1 << 24)) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_train_step: batch of %lld rays", (long long)rays->n);
  if (!labels->occ || !labels->t_local || !labels->normal || !labels->albedo || !labels->mat)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_train_step: labels need occ, t_local, normal, albedo and mat");
  if (!(opts->lr > 0.f) || !(opts->beta1 >= 0.f && opts->beta1 < 1.f) || !(opts->beta2 >= 0.f && opts->beta2 < 1.f) ||
      !(opts->eps > 0.f))
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_train_step: bad optimiser settings");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_train(ctx, o, rays->n);
  if (rc) return rc;
  RaysArg ra{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax, nullptr, o->handle,
             rays->n};
  const int64_t step = opts->apply_update ? o->step + 1 : o->step;
  if (opts->products != LSNIF_TRAIN_TENSOR_CORES && opts->products != LSNIF_TRAIN_FP32_SIMT)
    return fail(LSNIF_ERR_INVALID_ARG, "lsnif_train_step: unknown products %d", opts->products);
  cudaError_t e = launch_train_step(ctx->d_objs, o->slot + 1, ctx->d_objs + o->slot, o->d, ra, *labels, *opts, step,
                                    o->tb, o->n_params_mlp, ctx->d_err, st);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_train_step");
  if (opts->apply_update) {
    o->step = step;
    if ((rc = refresh_copies(ctx, o, st))) return rc;
  }
  if (stats) {
    float acc[8];
    e = cudaMemcpyAsync(acc, o->tb.loss, sizeof acc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lsnif_train_step: stats");
    stats->total = acc[0];
    stats->occ = acc[1];
    stats->t = acc[2];
    stats->normal = acc[3];
    stats->albedo = acc[4];
    stats->mat = acc[5];
    stats->step = o->step;
  }
  return LSNIF_OK;
}
