// Internal declarations of the LSNIF library: the device-side object record,
// kernel argument blocks and the launchers each .cu file exports to api.cpp.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "lsnif.h"

namespace lsnif {

// spatial-hash multipliers (instant-NGP, the encoding LSNIF's sparse grid uses)
constexpr uint32_t kPi2 = 2654435761u;
constexpr uint32_t kPi3 = 805459861u;

constexpr int kMaxCap = 32;          // H/2 <= 32
constexpr int kBuckets = kMaxCap + 1;  // per object: k = 0..32
constexpr int kTileM = 128;          // rays per tensor-core tile (tcgen05 M)
constexpr int kDistCap = 32;         // largest stored occupancy distance

inline bool valid_precision(int p) {
  return p == LSNIF_FP32_PLAIN || p == LSNIF_BF16_FUSED || p == LSNIF_FP8_FUSED || p == LSNIF_FP16_FUSED;
}
// the BF16 and FP16 paths share the fused kernel (only the operand type differs)
inline bool fused16_precision(int p) { return p == LSNIF_BF16_FUSED || p == LSNIF_FP16_FUSED; }

// error word bits written by kernels (never trap, never hang)
enum DeviceError : int {
  kErrBadHandle = 1,
  kErrWaitTimeout = 2,
  kErrCheck = 4,
};

// Everything a kernel needs to know about one object. Plain data, copied to
// a device array indexed by object slot.
struct DevObject {
  float bmin[3];
  float inv_ext[3];
  int32_t V;
  int32_t log2V;
  float invV;
  const uint32_t *occ;  // ceil(V^3/32) words
  // per voxel, the Chebyshev distance (in voxels) to the nearest occupied
  // voxel, capped at kDistCap: 0 = occupied; D >= 1 = every voxel within
  // D - 1 of this one is empty (V^3 bytes, voxel order of occ)
  const uint8_t *dist;
  // FP8 network (built on the first FP8 query after a parameter change):
  // first layer chunk-major (W x 2LF E4M3 bytes per chunk, core-matrix
  // layout); hidden and output layers (E4M3) then FP32 biases and scales
  const uint8_t *w0_8;
  const uint8_t *blob8;
  uint32_t blob8_bytes, blob8_bias_off, blob8_scale_off;

  int32_t L, F, log2T;
  uint32_t mask;
  int32_t res[LSNIF_MAX_LEVELS];
  const float *tab32;   // L x T x F
  const uint16_t *tab16;  // FP16 copy, same layout

  int32_t H, n_in, n_hidden, width, n_out, n_out_pad, n_mat, act;
  const float *mlp32;   // packed FP32 [W0 b0 W1 b1 ...]
  const uint8_t *umma;  // BF16 weights in tcgen05 core-matrix layout + FP32 biases
  const uint8_t *umma_h;  // the same blob with FP16 weights (saturated at 65504)
  uint32_t umma_bytes;  // total bytes of the umma blob (each of the two)
  uint32_t umma_bias_off;  // byte offset of the FP32 biases inside it
  // BF16 residuals W - BF16(W) of the layers after the first, in the layout of
  // those layers' part of umma (no biases): the BF16 path runs those layers
  // with two-term operands (hi.hi + hi.lo + lo.hi)
  const uint8_t *umma_lo;
  uint32_t umma_lo_bytes;
  // the first layer's FP16 weights chunk-major for the streamed FP16 kernel:
  // chunk s (network inputs [s CHK, (s+1) CHK), CHK = 2 L F: two points) is a
  // contiguous W x CHK core-matrix slice, so one bulk copy moves it
  const uint8_t *w0_16c;
  const float *plain_out;  // FP32 output layer padded to n_out_pad rows, then its bias

  // kept mesh (training labels): per-voxel triangle lists in CSR form
  const float *verts;
  const int32_t *tris;
  const float *vnormals;
  const int32_t *tri_mat;
  const float *albedo;
  const int32_t *vox_start;  // V^3 + 1
  const int32_t *vox_tris;
  int64_t nt;

  // object kind: 0 = LSNIF (voxels, hash grid, network); 1 = a triangle mesh
  // answered exactly through its BVH (the hybrid pipeline's non-LSNIF
  // objects, Sec. 4)
  int32_t kind;
  const float4 *bvh_nodes;   // 2 float4 per node (BvhNode)
  const float4 *bvh_tris;    // 3 float4 per stored triangle: v0, e1 = v1 - v0, e2 = v2 - v0
  const int32_t *bvh_order;  // stored position -> mesh triangle

  uint32_t handle;  // handle the slot currently holds (0 = free)
  int32_t valid;
};

// Rays as the kernels see them (SoA device pointers).
struct RaysArg {
  const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
  const uint32_t *obj;
  uint32_t single_handle;
  int64_t n;
};

struct HitsArg {
  uint8_t *hit;
  float *t, *nx, *ny, *nz;
  int32_t *mat;
  float *ar, *ag, *ab;
  float *logits;
};

// Scratch a query uses (device pointers into the context's workspace).
struct QueryScratch {
  float *pts;        // n x H x 3
  float *t01;        // n x 2
  uint8_t *k;        // n
  uint32_t *dup;     // n: bit s set when boundary point 2s is bit-identical to point 2s-1
  int16_t *slot;     // n object slot per ray (-1 invalid)
  int32_t *order;    // n ray indices grouped by (object, k desc)
  int32_t *counts;   // n_slots x kBuckets
  int32_t *offsets;  // n_slots x kBuckets
  int32_t *cursor;   // n_slots x kBuckets
  int32_t *tiles;    // max_tiles x 3 (slot, start, count)
  int32_t *meta;     // [0] n_live, [1] n_tiles, [2] n_points, [3] tile cursor
  float *X;          // FP32 path: chunk of tiles x kTileM rows x ldx features
  int32_t *blk;      // coherent grouping: live rays and points per block of kGroupBlock rays, then offsets
  int32_t *bins;     // counting sorts: rays per bin, then each bin's first position (kBinsAlloc)
  int32_t *bin_sums; // counting sorts: block sums of the bins' scan (kBinSumsAlloc)
  int32_t max_tiles; // upper bound on tiles (n / kTileM + n_slots)
  int32_t wmax;      // FP32 path: widest layer (hidden width or padded output)
};

struct QueryLaunch {
  const DevObject *objs;  // device array [n_slots]
  int32_t n_slots;
  int32_t H_max;
  RaysArg rays;
  HitsArg hits;
  QueryScratch s;
  int *err;               // device error word
  cudaStream_t stream;
  int trace_mode;         // traversal kernel: 0 one ray per thread, 1 persistent lanes, 2 persistent lanes
                          // over rays presorted by (object, entry cell, direction octant)
  int group_mode;         // 0: live rays grouped by (object, k desc); 1: one object, original order kept;
                          // 2: grouped by object only, warps of consecutive rays kept together;
                          // 3: by object, then by the Morton cell of the first boundary point
  int single_slot;        // object slot of a single-object query (group_mode 1)
};

constexpr int kGroupBlock = 4096;  // rays per block of the order-keeping grouping
constexpr int64_t kSpatialBins = int64_t(1) << 21;  // spatial grouping: (object, cell) bins at most
// bins and block sums the scratch holds for either counting sort (the
// presorted traversal adds one bin for the rays that miss)
constexpr int64_t kBinsAlloc = kSpatialBins + 1;
constexpr int64_t kBinSumsAlloc = (kBinsAlloc + 1023) / 1024 + 1;

// Spatial grouping: bits of a cell's Morton code, 3 m for 2^m cells per axis
// of the unit cube -- m = 6 (64 per axis) where the objects' bins fit
// kSpatialBins, fewer for many objects.
inline int spatial_cell_bits(int n_slots) {
  int m = 6;
  while (m > 1 && ((int64_t)n_slots << (3 * m)) > kSpatialBins) --m;
  return 3 * m;
}

// ---- launchers (query.cu) ----
// Traversal + histogram; returns kernels launched (adds to *launches).
cudaError_t launch_trace(const QueryLaunch &q, int *launches);
cudaError_t launch_group(const QueryLaunch &q, int *launches);
// exclusive scan of v[0..n) in place; sums needs (n + 1023) / 1024 + 1
// entries and receives the total at sums[(n + 1023) / 1024]
cudaError_t launch_exclusive_scan(int32_t *v, int64_t n, int32_t *sums, cudaStream_t st);
cudaError_t launch_plain_tail(const QueryLaunch &q, int ldx, int chunk_tiles, int *launches);
cudaError_t launch_trace_only(const DevObject *dobj, const RaysArg &rays, int32_t *k, float *t01,
                              float *pts, int32_t *vox, int *err, cudaStream_t st);
cudaError_t launch_encode(const DevObject *dobj, const DevObject &host_obj, const float *pts, int64_t n,
                          float *feats, int precision, cudaStream_t st);
cudaError_t launch_corners(const DevObject *dobj, const DevObject &host_obj, const float *pts,
                           int64_t n, uint32_t *out, cudaStream_t st);
cudaError_t launch_mlp_plain(const DevObject *dobj, const DevObject &host_obj, const float *X,
                             int64_t n, float *Z, cudaStream_t st);
// builds both tensor-core blobs (umma: BF16, umma_h: FP16) and the padded FP32 output layer
cudaError_t launch_build_umma(const DevObject &host_obj, cudaStream_t st);
cudaError_t launch_tables_to_half(const float *src, uint16_t *dst, int64_t n, cudaStream_t st);

// ---- fused tensor-core path (fused.cu) ----
// Returns cudaErrorNotSupported when the object's shape is outside the
// fused kernel's instantiations.
bool fused8_supported(const DevObject &host_obj);
size_t fused8_smem_bytes(const DevObject &host_obj, int H_max);
cudaError_t launch_fused8(const QueryLaunch &q, const DevObject &host_obj, int variant, int *launches);
// exact nearest-triangle query of the rays whose object is a mesh object
cudaError_t launch_mesh_query(const QueryLaunch &q, int *launches);
int fused8_variant_count();
void fused8_variant_shape(int variant, int *threads, int *levels);
cudaError_t launch_max_abs_half(const uint16_t *v, int64_t n, uint32_t *out_bits, cudaStream_t st);
bool fused_supported(const DevObject &host_obj);
// smallest ring; H_max: the query's largest H; fp16: FP16 operands (the BF16
// path also holds the two-term residual weights and activations)
size_t fused_smem_bytes(const DevObject &host_obj, int H_max, bool fp16);
// fp16: FP16 operands (weights from umma_h) instead of BF16
cudaError_t launch_fused(const QueryLaunch &q, const DevObject &host_obj, int variant, bool fp16, int *launches);
int fused_variant_count();
void fused_variant_shape(int variant, int *threads, int *levels);
// FP16 fused query for networks whose weights do not fit shared memory (the
// first layer streamed per chunk, later layers per layer; fused16s.cu)
bool fused16s_supported(const DevObject &host_obj);
size_t fused16s_smem_bytes(const DevObject &host_obj, int H_max);
cudaError_t launch_fused16s(const QueryLaunch &q, const DevObject &host_obj, int *launches);
cudaError_t launch_mlp_fused(const DevObject *dobj, const DevObject &host_obj, const float *X,
                             int64_t n, float *Z, bool fp16, int *err, cudaStream_t st);

// ---- training (train.cu) ----
struct TrainBuffers {
  float *feats;     // B x n_in (FP32)
  float *acts;      // B x width x n_hidden (post-activation)
  float *pre;       // B x width x n_hidden (pre-activation)
  float *Z;         // B x n_out
  float *dZ;        // B x n_out
  float *dA;        // B x max(width, n_in) scratch
  float *dB;        // B x max(width, n_in) scratch
  float *pts;       // B x H x 3
  float *t01;       // B x 2
  int32_t *k;       // B
  // the query traversal's own outputs for the batch: one-byte point counts
  // (widened into k), shared-point bits, object slots, its histogram
  // (kMaxSlots x kBuckets) and counters
  uint8_t *k8;
  uint32_t *dup;
  int16_t *slot;
  int32_t *counts;
  int32_t *meta;
  float *loss;      // 8 accumulators
  float *grad_mlp;  // n_params_mlp
  float *grad_tab;  // L x T x F
  float *m_mlp, *v_mlp, *m_tab, *v_tab;
};

cudaError_t launch_make_training_rays(const DevObject *dobj, const DevObject &h, const float *u, int64_t n,
                                      int64_t n_outside, float *rays_out, uint8_t *surface,
                                      cudaStream_t st);
cudaError_t launch_label_rays(const DevObject *dobj, const DevObject &h, const RaysArg &rays,
                              const lsnif_labels &out, cudaStream_t st);
// objs, n_slots: the context's object array up to this object's slot (the
// traversal resolves the rays' handle in it)
cudaError_t launch_train_step(const DevObject *objs, int n_slots, const DevObject *dobj, const DevObject &h,
                              const RaysArg &rays, const lsnif_labels &lab, const lsnif_train_opts &opts,
                              int64_t step, TrainBuffers &tb, int64_t n_params_mlp, int *err, cudaStream_t st);
// C[M x N] = op(A) . op(B) on the tensor cores (two-term BF16, FP32
// accumulation), op(A)[m][k] = tA ? A[k lda + m] : A[m lda + k], op(B)[k][n] =
// tB ? B[n ldb + k] : B[k ldb + n]; mode 0 store, 1 atomic add (k_split > 1
// allowed), 2 + bias[n] -> C, act -> post, 3 + bias[n], 4 times act'(aux) (train_gemm.cu)
cudaError_t launch_tc_gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, int tA, const float *B,
                           int ldb, int tB, float *C, int ldc, int mode, const float *bias, float *post,
                           const float *aux, int act, int k_split, int *err);

}  // namespace lsnif
