// Dense-layer products of the training step on the tensor cores (Sec. 5:
// the network's products in reduced precision, gradients accumulated in
// FP32; Sec. 5.2 training). One kernel serves every product of the forward
// and backward pass:
//
//   C[M x N] = op(A)[M x K] . op(B)[K x N]
//   op(A)[m][k] = tA ? A[k lda + m] : A[m lda + k]
//   op(B)[k][n] = tB ? B[n ldb + k] : B[k ldb + n]
//
// with the epilogues of the FP32 path it replaces: store; atomic add (the
// weight gradients, whose reduction over the batch is split over CTAs);
// + bias, store the pre-activation and the activation; + bias; multiply by
// the activation's derivative at a saved pre-activation.
//
// Operands are FP32 in global memory (features, activations, gradients and
// the FP32 master weights). All threads of a CTA stage them into shared
// memory as two-term BF16 -- hi = BF16(x), lo = BF16(x - hi) -- in the
// no-swizzle K-major core-matrix layout, transposing on the way where the
// product reads an operand along its rows (weight gradients: dY^T . X; input
// gradients: dY . W). One thread issues tcgen05.mma kind::f16 hi.hi + hi.lo
// + lo.hi per K step of 16 with FP32 accumulation in tensor memory (the
// lo.lo product, about 2^-16 of the rest, is left out), so the gradients keep
// FP32-level accuracy and the FP32 exponent range (no loss scaling). Two
// shared-memory stages: a stage is refilled once the MMAs that read it have
// completed; the loads of the next chunk go to registers before the current
// chunk's MMAs are issued, so their latency overlaps them.
//
// Tiles: 128 rows (the tcgen05 M; rows past M are zero), N_CH <= 96 columns
// (the grid's y dimension walks larger N), K in chunks of 64; the grid's z
// dimension splits K (the batch, for weight gradients) into ranges whose
// partial products are added atomically.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "device.cuh"
#include "tc_common.cuh"

namespace lsnif {

namespace {

constexpr int kGM = 128;        // tile rows (tcgen05 M)
constexpr int kGK = 64;         // K chunk per stage
constexpr int kGThreads = 256;  // eight warps; warps w and w + 4 share TMEM lane quarter w

// kind::f16 instruction descriptor, BF16 A and B (K-major), FP32 D, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// two-term BF16 of two values: hi word and lo word (element 0 in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = *reinterpret_cast<const uint32_t *>(&l);
}

// byte offset of element (row, k) in a K = 64 core-matrix tile
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

struct GemmArgs {
  int M, N, K;
  const float *A;
  int lda, tA;
  const float *B;
  int ldb, tB;
  float *C;
  int ldc, mode;
  const float *bias;
  float *post;
  const float *aux;
  int act;
  int n_ch;      // columns per CTA (multiple of 16, <= 96)
  int k_per_z;   // K range per grid z (a multiple of kGK)
  int nst;       // shared-memory stages (1 when a CTA's K range is one chunk)
  int *err;      // device error word (bounded waits that give up)
};

// Stage rows [r0, r0 + rows) x k [k0, k0 + 64) of an operand X(row, k) into
// the hi and lo tiles; k >= kend is zero (the other operand's garbage times 0
// must stay 0), rows past the operand's end are not written (they only feed
// rows or columns of the product that are not stored). kc: X(row, k) =
// P[row ld + k] (contiguous along k); else X(row, k) = P[k ld + row]
// (contiguous along rows: the transposed read of dY^T, X^T and W^T).
//
// An item is one row's 8 consecutive k -- the 16 bytes that row holds in one
// core matrix -- so a thread converts it to two 16-byte words (hi, lo) and
// stores each with one instruction. Items are laid out over a warp so that
// each quarter-warp stores one whole 128-byte core matrix (8 consecutive
// rows, the same k), which touches every shared-memory bank once:
//   kc:   a warp's 32 items are 8 rows x 4 groups of k; a thread reads its
//         row's 8 values as two 16-byte loads;
//   else: a warp's 32 items are 32 consecutive rows at one group of k; a
//         thread reads its 8 values one k at a time, and each of those loads
//         reads 128 consecutive bytes across the warp.
// (Storing 2 or 4 bytes per element along the other axis of a core matrix
// put 8 lanes of a warp on one bank.) A chunk of one operand is at most 128
// rows x 8 groups = 1024 items, kItems per thread. Staging is split in two:
// stage_load issues a thread's loads into registers, stage_store converts and
// writes them, so that the loads of chunk c + 1 are in flight while chunk c
// is multiplied.
constexpr int kItems = 4;

__device__ __forceinline__ void item_rk(bool kc, int it, int &row, int &k) {
  if (kc) {
    row = (it & 7) + ((it >> 6) << 3);
    k = ((it >> 3) & 7) * 8;
  } else {
    row = (it & 31) + ((it >> 8) << 5);
    k = ((it >> 5) & 7) * 8;
  }
}

__device__ __forceinline__ int chunk_items(bool kc, int rows) {
  return kc ? ((rows + 7) & ~7) * 8 : ((rows + 31) & ~31) * 8;
}

__device__ __forceinline__ void stage_load(float (&v)[kItems][8], const float *P, int ld, bool kc, int r0,
                                           int tile_rows, int nrows, int k0, int kend, int tid) {
  const int rows = min(nrows - r0, tile_rows);
  const int items = chunk_items(kc, rows);
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
#pragma unroll
  for (int b = 0; b < kItems; ++b) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[b][j] = 0.f;
    const int it = tid + b * kGThreads;
    if (it >= items) continue;
    int row, k;
    item_rk(kc, it, row, k);
    if (row >= rows) continue;
    const int gk = k0 + k;
    if (kc) {
      const float *src = P + (int64_t)(r0 + row) * ld + gk;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (vec && gk + 4 * h + 3 < kend) {
          const float4 f = __ldg(reinterpret_cast<const float4 *>(src + 4 * h));
          v[b][4 * h + 0] = f.x; v[b][4 * h + 1] = f.y; v[b][4 * h + 2] = f.z; v[b][4 * h + 3] = f.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (gk + 4 * h + j < kend) v[b][4 * h + j] = __ldg(src + 4 * h + j);
        }
      }
    } else {
      const float *src = P + (int64_t)gk * ld + r0 + row;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (gk + j < kend) v[b][j] = __ldg(src + (int64_t)j * ld);
    }
  }
}

__device__ __forceinline__ void stage_store(uint8_t *hi, uint8_t *lo, const float (&v)[kItems][8], bool kc, int r0,
                                            int tile_rows, int nrows, int tid) {
  const int rows = min(nrows - r0, tile_rows);
  const int items = chunk_items(kc, rows);
#pragma unroll
  for (int b = 0; b < kItems; ++b) {
    const int it = tid + b * kGThreads;
    if (it >= items) break;
    int row, k;
    item_rk(kc, it, row, k);
    if (row >= rows) continue;
    uint4 h, l;
    split2(v[b][0], v[b][1], h.x, l.x);
    split2(v[b][2], v[b][3], h.y, l.y);
    split2(v[b][4], v[b][5], h.z, l.z);
    split2(v[b][6], v[b][7], h.w, l.w);
    const uint32_t o = tile_off(row, k);  // k is a multiple of 8: 16-byte aligned
    *reinterpret_cast<uint4 *>(hi + o) = h;
    *reinterpret_cast<uint4 *>(lo + o) = l;
  }
}

// One operand of a chunk loaded and stored before the other: the short
// products' form, which holds one operand's registers at a time.
__device__ __forceinline__ void stage(uint8_t *hi, uint8_t *lo, const float *P, int ld, bool kc, int r0,
                                      int tile_rows, int nrows, int k0, int kend, int tid) {
  float v[kItems][8];
  stage_load(v, P, ld, kc, r0, tile_rows, nrows, k0, kend, tid);
  stage_store(hi, lo, v, kc, r0, tile_rows, nrows, tid);
}

// One CTA: rows [blockIdx.x 128, +128) x columns [blockIdx.y n_ch, +n_ch) of
// C, K range [blockIdx.z k_per_z, +k_per_z).
// PIPE: the next chunk's loads are issued before this chunk's MMAs (CTAs
// with more than one chunk); otherwise one operand's registers at a time, so
// that short products keep more CTAs per SM.
template <bool PIPE>
__global__ void __launch_bounds__(kGThreads) tc_gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t gsm_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ch = g.n_ch;
  const uint32_t a_bytes = kGM * kGK * 2, b_bytes = (uint32_t)n_ch * kGK * 2;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;  // A hi, A lo, B hi, B lo
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + g.nst * stage_bytes);  // [0..1] stages, [2] accumulator
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 3);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(s_tmem + 1);
  const int tmem_cols = n_ch <= 32 ? 32 : (n_ch <= 64 ? 64 : (n_ch <= 128 ? 128 : 256));

  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * n_ch;
  const int kb = blockIdx.z * g.k_per_z, ke = min(g.K, kb + g.k_per_z);
  const int nchunks = max(0, (ke - kb + kGK - 1) / kGK);
  const bool a_kc = !g.tA, b_kc = g.tB != 0;

  if (tid == 0) {
    mbar_init(su32(&bars[0]), 1);
    mbar_init(su32(&bars[1]), 1);
    mbar_init(su32(&bars[2]), 1);
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = idesc_bf16(n_ch);

  float va[kItems][8], vb[kItems][8];  // PIPE only
  if (PIPE && nchunks > 0) {
    stage_load(va, g.A, g.lda, a_kc, m0, kGM, g.M, kb, ke, tid);
    stage_load(vb, g.B, g.ldb, b_kc, n0, n_ch, g.N, kb, ke, tid);
  }
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c % g.nst, use = c / g.nst;
    uint8_t *st = base + buf * stage_bytes;
    if (use > 0) {  // the MMAs of chunk c - nst read this stage
      if (tid == 0 && !mbar_wait(su32(&bars[buf]), (uint32_t)((use - 1) & 1), abort_flag)) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) break;
    }
    if constexpr (PIPE) {
      stage_store(st, st + a_bytes, va, a_kc, m0, kGM, g.M, tid);
      stage_store(st + 2 * a_bytes, st + 2 * a_bytes + b_bytes, vb, b_kc, n0, n_ch, g.N, tid);
      if (c + 1 < nchunks) {  // the next chunk's loads fly during this chunk's sync and MMAs
        const int k1 = kb + (c + 1) * kGK;
        stage_load(va, g.A, g.lda, a_kc, m0, kGM, g.M, k1, ke, tid);
        stage_load(vb, g.B, g.ldb, b_kc, n0, n_ch, g.N, k1, ke, tid);
      }
    } else {
      const int k0 = kb + c * kGK;
      stage(st, st + a_bytes, g.A, g.lda, a_kc, m0, kGM, g.M, k0, ke, tid);
      stage(st + 2 * a_bytes, st + 2 * a_bytes + b_bytes, g.B, g.ldb, b_kc, n0, n_ch, g.N, k0, ke, tid);
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    if (tid == 0) {
      tc_after();
      const uint32_t ah = su32(st), al = ah + a_bytes, bh = ah + 2 * a_bytes, bl = bh + b_bytes;
#pragma unroll
      for (int ks = 0; ks < kGK / 16; ++ks) {
        const uint64_t dah = umma_desc(ah + ks * 256, 128, 1024), dal = umma_desc(al + ks * 256, 128, 1024);
        const uint64_t dbh = umma_desc(bh + ks * 256, 128, 1024), dbl = umma_desc(bl + ks * 256, 128, 1024);
        mma_bf16(tmem, dah, dbh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, idesc, 1u);
        mma_bf16(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(su32(&bars[buf]));
    }
  }
  // every MMA issued so far completes before the accumulator is read (and
  // before shared memory and TMEM are released, also after an abort)
  if (tid == 0) {
    mma_commit(su32(&bars[2]));
    if (!mbar_wait_teardown(su32(&bars[2]), 0u)) *abort_flag = 1;
  }
  __syncthreads();
  tc_after();
  const bool ok = !*abort_flag;
  // The product goes TMEM -> shared memory -> global memory, 32 columns at a
  // time: each piece is written to a tile of rows padded by one float (a
  // warp's row-wise writes hit distinct banks), then stored row after row
  // with consecutive threads on consecutive columns.
  float *tile = reinterpret_cast<float *>(base);  // the stages are free now
  constexpr int kPc = 32, kLdT = kPc + 1;
  const int rows = min(kGM, g.M - m0), cols = min(n_ch, g.N - n0);
  const int row = (warp & 3) * 32 + lane;  // TMEM lane = tile row
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  for (int p0 = 0; ok && p0 < cols; p0 += kPc) {
    const int c0 = p0 + (warp >> 2) * 16;
    if (c0 < n_ch) {
      uint32_t v[16];
      if (nchunks > 0) {
        TMEM_LD16(trow + c0, (&v[0]));
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;  // an empty K range: the product is 0
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) tile[row * kLdT + (warp >> 2) * 16 + j] = __uint_as_float(v[j]);
    }
    __syncthreads();
    const int pc = min(kPc, cols - p0);
    for (int idx = tid; idx < rows * pc; idx += kGThreads) {
      const int r = idx / pc, cc = idx - r * pc;
      const int gn = n0 + p0 + cc;
      const int64_t o = (int64_t)(m0 + r) * g.ldc + gn;
      float x = tile[r * kLdT + cc];
      if (g.mode == 0) g.C[o] = x;
      else if (g.mode == 1) { if (nchunks > 0) atomicAdd(g.C + o, x); }
      else if (g.mode == 2) { x += g.bias[gn]; g.C[o] = x; g.post[o] = act_fn(x, g.act); }
      else if (g.mode == 3) g.C[o] = x + g.bias[gn];
      else g.C[o] = x * act_grad(g.aux[o], g.act);
    }
    __syncthreads();
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (tid == 0 && !ok) atomicOr(g.err, kErrWaitTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace

// Host launcher with the FP32 path's argument convention (see the top of
// this file). k_split: ranges the K dimension is cut into (atomic mode).
cudaError_t launch_tc_gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, int tA, const float *B,
                           int ldb, int tB, float *C, int ldc, int mode, const float *bias, float *post,
                           const float *aux, int act, int k_split, int *err) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  GemmArgs g{M, N, K, A, lda, tA, B, ldb, tB, C, ldc, mode, bias, post, aux, act, 0, 0, 1, err};
  const int n16 = (N + 15) / 16 * 16;
  // Column tiles of equal width, at most 96 columns (64 for the split-K
  // weight gradients, whose CTAs hold two stages): narrower tiles let
  // several CTAs share an SM, so that one CTA's loads overlap another's
  // MMAs and stores (a CTA's own phases run one after the other).
  const int max_n = (mode == 1 && k_split > 1) ? 64 : 96;
  const int ny = (n16 + max_n - 1) / max_n;
  g.n_ch = ((n16 / 16 + ny - 1) / ny) * 16;
  const int ks = std::max(1, k_split);
  g.k_per_z = std::max(kGK, ((K + ks - 1) / ks + kGK - 1) / kGK * kGK);
  const int nz = std::max(1, (K + g.k_per_z - 1) / g.k_per_z);
  if (nz > 1 && mode != 1) return cudaErrorInvalidValue;  // split K needs the atomic epilogue
  const size_t stage = 2 * (size_t)kGM * kGK * 2 + 2 * (size_t)g.n_ch * kGK * 2;
  g.nst = g.k_per_z > kGK ? 2 : 1;
  // the stages (reused for a 128 x 33 piece of the product) + barriers + alignment slack
  const size_t smem = g.nst * stage + 64 + 1024;
  static int attr = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = 1;
  }
  dim3 grid((M + kGM - 1) / kGM, (N + g.n_ch - 1) / g.n_ch, nz);
  if (g.nst > 1) tc_gemm_kernel<true><<<grid, kGThreads, smem, st>>>(g);
  else tc_gemm_kernel<false><<<grid, kGThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace lsnif
