// lsnif_gather_rate: the request ceiling that a hash-grid gather runs
// against. The fused query's corner loads are small (4- and 8-byte) loads at
// hashed, effectively random positions of an object's FP16 tables; when the
// tables fit L2, the rate at which L2 answers such requests -- not HBM
// bandwidth -- bounds the gather. This kernel measures that rate on the
// object's own table copy: independent random 8-byte loads spread uniformly
// over it, 16 in flight per thread, every SM at full occupancy, nothing else
// in the loop. Each load touches one 32-byte sector.
#include <cuda_runtime.h>

#include <algorithm>

#include "lsnif_impl.h"
#include "runtime.h"

using namespace lsnif;

namespace {

constexpr int kInFlight = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) gather_rate_kernel(const uint2 *tab, uint32_t n_words, int iters,
                                                               uint32_t seed, int *sink) {
  // per-thread linear congruential sequence (Numerical Recipes constants):
  // the addresses never depend on loaded values, so all 16 loads of a round
  // are in flight together
  uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u ^ seed;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    uint2 v[kInFlight];
#pragma unroll
    for (int j = 0; j < kInFlight; ++j) {
      h = h * 1664525u + 1013904223u;
      v[j] = __ldg(tab + __umulhi(h, n_words));
    }
#pragma unroll
    for (int j = 0; j < kInFlight; ++j) acc ^= v[j].x + v[j].y;
  }
  if (acc == 0x9E3779B9u) atomicOr(sink, 1);  // keeps the loads; almost never taken
}

}  // namespace

extern "C" int lsnif_gather_rate(lsnif_ctx *ctx, lsnif_obj obj, int64_t loads, void *stream, double *requests_per_s) {
  if (!ctx || !requests_per_s) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_gather_rate: NULL argument");
  if (loads < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_gather_rate: loads < 0");
  Object *o = find_object(ctx, obj);
  if (!o) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_gather_rate: bad handle %u", obj);
  if (o->d.kind != 0) return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_gather_rate: object %u has no tables", obj);
  const uint64_t words = (((uint64_t)o->d.L << o->d.log2T) * (uint64_t)o->d.F) / 4;  // 8-byte words of FP16
  if (words < 1 || words > 0xFFFFFFFFull)
    return fail(LSNIF_ERR_UNSUPPORTED, "lsnif_gather_rate: table of %llu words", (unsigned long long)words);
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = ctx->sms * kBlocksPerSm;
  const int64_t per_round = (int64_t)grid * kThreads * kInFlight;
  if (loads == 0) loads = int64_t(3) << 29;  // about 1.6e9 loads: a few milliseconds
  const int iters = (int)std::max<int64_t>(1, std::min<int64_t>((loads + per_round - 1) / per_round, 1 << 20));
  void *sink = nullptr;
  int rc = dev_alloc(ctx, sizeof(int), &sink, "gather-rate sink");
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint2 *tab = reinterpret_cast<const uint2 *>(o->d.tab16);
  if (e == cudaSuccess) {  // warm-up: brings the table into L2 when it fits
    gather_rate_kernel<<<grid, kThreads, 0, st>>>(tab, (uint32_t)words, std::max(1, iters / 8), 7u, (int *)sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    gather_rate_kernel<<<grid, kThreads, 0, st>>>(tab, (uint32_t)words, iters, 11u, (int *)sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(ctx, sink);
  if (e != cudaSuccess) return cuda_fail(e, "lsnif_gather_rate");
  *requests_per_s = (double)per_round * iters / (ms * 1e-3);
  return LSNIF_OK;
}
