// Host-side runtime state of the library: the context, loaded objects,
// per-stream scratch workspaces and the serving queue.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "lsnif_impl.h"

namespace lsnif {

constexpr int kMaxSlots = 1024;

struct Object {
  lsnif_config cfg{};
  int slot = -1;
  uint32_t handle = 0;
  DevObject d{};
  float bmin[3]{}, bmax[3]{};
  std::vector<int32_t> res;
  std::vector<uint32_t> occ_host;
  int64_t n_params_mlp = 0;
  size_t device_bytes = 0;
  std::vector<void *> allocs;
  // training state
  TrainBuffers tb{};
  int64_t tb_batch = 0;   // rays the buffers are sized for
  int64_t step = 0;
  std::vector<void *> train_allocs;
  bool fp8_stale = true;   // the FP8 network no longer matches the parameters
  int64_t bvh_nodes = 0;   // mesh objects: nodes of the BVH
};

// Scratch of one query stream. Grows on demand; freed with the context.
struct Workspace {
  void *base = nullptr;
  size_t bytes = 0;
  int64_t cap_rays = 0;
  int cap_H = 0, cap_slots = 0, cap_nin = 0;
  // host-query staging
  void *stage = nullptr;
  size_t stage_bytes = 0;
};

struct Request;
struct Server;

}  // namespace lsnif

struct lsnif_ctx {
  int device = 0;
  int sms = 0;
  size_t budget = 0, used = 0;
  int64_t fail_alloc_after = -1;
  std::map<void *, size_t> sizes;
  std::vector<lsnif::Object *> slots;
  std::vector<uint16_t> gen;
  int n_slots_used = 0;
  lsnif::DevObject *d_objs = nullptr;
  int *d_err = nullptr;
  int32_t *d_prof_meta = nullptr;
  lsnif::Workspace ws;
  int fused_variant = 0;    // fused-kernel shape of BF16 queries (see lsnif_autotune)
  int fused_variant16 = 0;  // and of FP16 queries
  int fp8_variant = 0;    // FP8 fused-kernel shape (lsnif_set_variant8)
  int trace_mode = 1;     // traversal kernel (see lsnif_autotune)
  int group_mode = 0;     // grouping of live rays (see lsnif_set_group_mode)
  int host_mode = 0;      // host-buffer queries: 0 staged copies, 1 direct access (lsnif_set_host_mode)
  // CUDA-graph cache of queries (see lsnif_set_graph_mode)
  bool graph_mode = false;
  std::map<std::vector<uint64_t>, cudaGraphExec_t> graphs;
  void *graphs_ws = nullptr;  // workspace the cached graphs point into
  // profiling
  bool profiling = false;
  cudaEvent_t ev[6]{};
  cudaStream_t prof_stream = nullptr;
  lsnif_profile prof{};
  bool prof_valid = false;
  // serving
  lsnif::Server *server = nullptr;
  // instanced-scene queries: instances, per-ray pair counts and offsets; pairs
  void *scene_buf = nullptr, *pair_buf = nullptr, *raster_buf = nullptr;
  size_t scene_bytes = 0, pair_bytes = 0, raster_bytes = 0;
  // host-buffer queries: copy streams and per-chunk events (created on first use)
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t hev[16]{};
};

namespace lsnif {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
int dev_alloc(lsnif_ctx *ctx, size_t bytes, void **out, const char *what);
void dev_free(lsnif_ctx *ctx, void *p);
int check_device(lsnif_ctx *ctx, cudaStream_t st);

Object *find_object(lsnif_ctx *ctx, lsnif_obj h);
void free_object(lsnif_ctx *ctx, Object *o);
size_t blob_size(const Object *o);
int upload_params(lsnif_ctx *ctx, Object *o, const float *tables, const float *mlp);
int refresh_copies(lsnif_ctx *ctx, Object *o, cudaStream_t st);
int ensure_fp8(lsnif_ctx *ctx, Object *o, cudaStream_t st);

// query
size_t workspace_bytes(int64_t n, int H, int n_slots, int n_in);
int ensure_workspace(lsnif_ctx *ctx, Workspace *ws, int64_t n, int H, int n_slots, int n_in);
void free_workspace(lsnif_ctx *ctx, Workspace *ws);
// err: the device error word the kernels report to (NULL: the context's)
int run_query(lsnif_ctx *ctx, Workspace *ws, const lsnif_rays *rays, lsnif_hits *hits, int precision,
              cudaStream_t st, bool profile, int *err = nullptr);
int query_shape(lsnif_ctx *ctx, const lsnif_rays *rays, int precision, int *H, int *n_in);
void clear_graphs(lsnif_ctx *ctx);

// training
void free_train_state(lsnif_ctx *ctx, Object *o);
void reset_optimizer(lsnif_ctx *ctx, Object *o);

// serving
void server_shutdown(lsnif_ctx *ctx);

}  // namespace lsnif
