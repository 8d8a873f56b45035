// Fused BF16 tensor-core query kernel for sm_103a: hash-grid gather ->
// every MLP layer on tcgen05 (TMEM accumulators) -> decode, one persistent
// CTA per SM. The paper fuses all layers of its FP16 network into one kernel
// on its own hardware (Sec. 5); here the gather is fused in as well, so the
// concatenated input vector (Sec. 3.2) never leaves shared memory.
//
// Per 128-ray tile (the tcgen05 M), for each occupied-voxel segment s
// (= points 2s and 2s+1, the K chunk of 2*L*F input columns):
//   all 16 warps gather the chunk's features into a BF16 A tile in shared
//   memory (no-swizzle K-major core-matrix layout), one thread issues the
//   chunk's MMAs against the resident first-layer weights, and a ring of
//   buffers lets the next chunk's gather overlap the MMAs. Chunks no ray of
//   the tile reaches are skipped (tiles are sorted by point count).
// Hidden and output layers: warps 0-3 (one TMEM lane = one ray each) read
// the accumulator, add bias, apply the activation, write BF16 activations
// back to shared memory for the next MMA, and finally decode the logits.
//
// Every mbarrier wait is bounded by a clock limit; on expiry the kernel sets
// the device error word, stops, frees its TMEM and returns.
#include <cstdio>

#include "device.cuh"
#include "encode.cuh"

namespace lsnif {

namespace {

constexpr int kNBuf = 3;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: BF16 A and B (K-major), FP32 D, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

#define TMEM_LD16(taddr, r)                                                                                        \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
               "[%16];"                                                                                            \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                       \
               : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

// byte offset of the 16-byte row piece (row r, core K-group kg) in a
// [rows/8][K/8][8][8] BF16 tile with row-group stride sbo
__device__ __forceinline__ uint32_t core_off(int r, int kg, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(r & 7) * 16u;
}

struct FusedArgs {
  QueryLaunch q;
  // X-rows mode (lsnif_mlp): X n x n_in FP32 in, Z n x n_out FP32 out
  const float *X;
  float *Z;
  int64_t xrows;
  uint32_t smem_blob;  // bytes reserved for the weight blob
};

struct Smem {
  uint8_t *blob, *ring, *act;
  int32_t *ray;
  int32_t *kk;
  float *t0, *t1;
  uint64_t *mbar;  // kNBuf "empty" ring barriers (MMA done), the accumulator
                   // barrier, then kNBuf "full" ring barriers (tile written)
  uint32_t *tmem_slot;
  int32_t *misc;   // [0] tile, [1] abort
};

}  // namespace

// F: features per level; W: hidden width; XROWS: read the network input
// from global rows instead of gathering it; NT: threads per CTA; NLB:
// levels whose corner loads are in flight together per gather item.
template <int F, int W, bool XROWS, int NT, int NLB>
__global__ void __launch_bounds__(NT, 1) fused_kernel(FusedArgs a) {
  constexpr int kThreads = NT;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;

  // carve shared memory (offsets are multiples of 1024)
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Smem S;
  S.blob = base;
  const DevObject *objs = q.objs;
  uint32_t off = (a.smem_blob + 1023u) & ~1023u;
  S.ring = base + off;
  // ring buffers hold one K chunk (2 points x L x F columns) for L <= 16
  const uint32_t ring_stride = (uint32_t)kTileM * (uint32_t)(2 * 16 * F) * 2u;
  off += kNBuf * ring_stride;
  S.act = base + off;
  off += (uint32_t)kTileM * W * 2u;
  S.ray = reinterpret_cast<int32_t *>(base + off);
  off += kTileM * 4;
  S.kk = reinterpret_cast<int32_t *>(base + off);
  off += kTileM * 4;
  S.t0 = reinterpret_cast<float *>(base + off);
  off += kTileM * 4;
  S.t1 = reinterpret_cast<float *>(base + off);
  off += kTileM * 4;
  S.mbar = reinterpret_cast<uint64_t *>(base + off);
  off += 8 * (2 * kNBuf + 1);
  S.tmem_slot = reinterpret_cast<uint32_t *>(base + off);
  off += 16;
  S.misc = reinterpret_cast<int32_t *>(base + off);
  off += 16;
  float *s_res = reinterpret_cast<float *>(base + off);  // lattice resolution per level

  constexpr int kTmemCols = W < 32 ? 32 : W;
  if (tid == 0) {
    for (int i = 0; i < kNBuf + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.mbar[i])) : "memory");
    for (int i = kNBuf + 1; i < 2 * kNBuf + 1; ++i)   // every thread arrives once per chunk
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&S.mbar[i])), "r"(kThreads) : "memory");
    S.misc[1] = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(S.tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *S.tmem_slot;

  int chunk_ctr = 0;  // chunks issued (ring phase tracking)
  int acc_ctr = 0;    // accumulator-barrier completions consumed
  int cur_slot = -1;
  int L = 0, H = 0, n_hidden = 0, n_out = 0, n_out_pad = 0, n_mat = 0, act = 0, n_in = 0, Hs = q.H_max;
  uint32_t mask = 0;
  const uint16_t *tab = nullptr;
  uint32_t w0_sbo = 0, bias_off = 0;
  bool aborted = false;

  const int64_t n_tiles = XROWS ? (a.xrows + kTileM - 1) / kTileM : (int64_t)q.s.meta[1];
  for (;;) {
    // ---- fetch the next tile ----
    if (tid == 0) {
      int t = XROWS ? atomicAdd(a.q.s.meta + 3, 1) : atomicAdd(q.s.meta + 3, 1);
      S.misc[0] = t;
      S.misc[2] = 0;   // the tile's largest segment count
    }
    __syncthreads();
    const int64_t tile = S.misc[0];
    if (tile >= n_tiles || S.misc[1]) break;
    int slot, start, cnt;
    if (XROWS) {
      slot = 0;
      start = (int)(tile * kTileM);
      cnt = (int)min((int64_t)kTileM, a.xrows - tile * kTileM);
    } else {
      slot = q.s.tiles[3 * tile + 0];
      start = q.s.tiles[3 * tile + 1];
      cnt = q.s.tiles[3 * tile + 2];
    }
    // ---- (re)load the object's weights ----
    if (slot != cur_slot) {
      const DevObject &ob = objs[slot];
      L = ob.L; H = ob.H; n_hidden = ob.n_hidden; n_out = ob.n_out; n_out_pad = ob.n_out_pad;
      n_mat = ob.n_mat; act = ob.act; n_in = ob.n_in; mask = ob.mask; tab = ob.tab16;
      w0_sbo = (uint32_t)(n_in / 8) * 128u;
      bias_off = ob.umma_bias_off;
      const uint4 *src = reinterpret_cast<const uint4 *>(ob.umma);
      uint4 *dst = reinterpret_cast<uint4 *>(S.blob);
      const int nvec = (int)(ob.umma_bytes / 16);
      for (int i = tid; i < nvec; i += kThreads) dst[i] = __ldg(src + i);
      if (tid < LSNIF_MAX_LEVELS) s_res[tid] = (float)ob.res[tid];
      fence_async_smem();
      __syncthreads();
      cur_slot = slot;
    }
    if (tid < kTileM) {
      int r = tid;
      if (r < cnt) {
        if (XROWS) {
          S.ray[r] = start + r;
          S.kk[r] = H / 2;
          atomicMax(&S.misc[2], H / 2);
        } else {
          int32_t ray = q.s.order[start + r];
          S.ray[r] = ray;
          S.kk[r] = q.s.k[ray];
          atomicMax(&S.misc[2], S.kk[r]);
          float2 tt = reinterpret_cast<const float2 *>(q.s.t01)[ray];
          S.t0[r] = tt.x;
          S.t1[r] = tt.y;
        }
      } else {
        S.ray[r] = -1;
        S.kk[r] = 0;
      }
    }
    __syncthreads();
    const int kmax = S.misc[2];  // chunks no ray of the tile reaches are skipped
    const int CHK = 2 * L * F;              // columns per chunk (one segment)
    const int G = (L * F) / 8;              // 16-byte column groups per point
    const uint32_t a_sbo = (uint32_t)(CHK / 8) * 128u;
    const uint32_t idesc_h = idesc_bf16(W);

    // ---- layer 0: gather chunk by chunk, MMA against resident W0 ----
    for (int s = 0; s < kmax; ++s) {
      const int buf = chunk_ctr % kNBuf;
      const int use = chunk_ctr / kNBuf;
      if (use > 0) {
        if (!mbar_wait(su32(&S.mbar[buf]), (uint32_t)((use - 1) & 1))) { aborted = true; }
      }
      uint8_t *A = S.ring + buf * ring_stride;
      const int items = kTileM * 2 * G;
      for (int e = tid; e < items; e += kThreads) {
        const int r = e & (kTileM - 1);
        const int rest = e >> 7;
        const int j = rest % 2, g = rest / 2;
        uint4 outv = make_uint4(0, 0, 0, 0);
        if (XROWS) {
          const int row = S.ray[r];
          if (row >= 0) {
            const float *xr = a.X + (int64_t)row * n_in + (size_t)(2 * s + j) * L * F + g * 8;
            float4 x0 = *reinterpret_cast<const float4 *>(xr);
            float4 x1 = *reinterpret_cast<const float4 *>(xr + 4);
            outv = make_uint4(pack_bf16(x0.x, x0.y), pack_bf16(x0.z, x0.w), pack_bf16(x1.x, x1.y),
                              pack_bf16(x1.z, x1.w));
          }
        } else if (S.kk[r] > s) {
          const int32_t ray = S.ray[r];
          const float *P = q.s.pts + ((size_t)ray * Hs + 2 * s + j) * 3;
          const float3 p = make_float3(P[0], P[1], P[2]);
          constexpr int LPG = 8 / F;  // levels per 16-byte group of the A tile
          float flat[8];
          const size_t lstride = (size_t)(mask + 1) * F;
#pragma unroll
          for (int u0 = 0; u0 < LPG; u0 += NLB) {
            const int l = g * LPG + u0;
            if constexpr (F == 2) {
              __half2 h[NLB];
              encode_levels_h2<NLB>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride, lstride * 2, mask, p,
                                    s_res + l, h);
#pragma unroll
              for (int u = 0; u < NLB; ++u) {
                const float2 f2 = __half22float2(h[u]);
                flat[(u0 + u) * 2] = f2.x;
                flat[(u0 + u) * 2 + 1] = f2.y;
              }
            } else {
              float f[NLB][F];
              encode_levels_f16<F, NLB>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride, lstride * 2,
                                        mask, p, s_res + l, f);
#pragma unroll
              for (int u = 0; u < NLB; ++u)
#pragma unroll
                for (int c = 0; c < F; ++c) flat[(u0 + u) * F + c] = f[u][c];
            }
          }
          outv = make_uint4(pack_bf16(flat[0], flat[1]), pack_bf16(flat[2], flat[3]), pack_bf16(flat[4], flat[5]),
                            pack_bf16(flat[6], flat[7]));
        }
        const int kg = j * G + g;
        *reinterpret_cast<uint4 *>(A + core_off(r, kg, a_sbo)) = outv;
      }
      // publish this thread's part of the tile to the tensor core; only the
      // issuing thread waits for the whole tile, the other warps run ahead
      fence_async_smem();
      mbar_arrive(su32(&S.mbar[kNBuf + 1 + buf]));
      if (tid == 0) {
        if (!mbar_wait(su32(&S.mbar[kNBuf + 1 + buf]), (uint32_t)(use & 1))) aborted = true;
        tc_after();
        const uint32_t a0 = su32(A), b0 = su32(S.blob);
        for (int ks = 0; ks < CHK / 16; ++ks) {
          const uint64_t ad = umma_desc(a0 + ks * 256, 128, a_sbo);
          const uint64_t bd = umma_desc(b0 + (uint32_t)((s * CHK) / 8 + 2 * ks) * 128u, 128, w0_sbo);
          mma_bf16(tmem, ad, bd, idesc_h, (s > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(su32(&S.mbar[buf]));
      }
      ++chunk_ctr;
    }
    if (tid == 0) mma_commit(su32(&S.mbar[kNBuf]));

    // ---- hidden layers and the output layer ----
    const uint32_t act_sbo = (uint32_t)(W / 8) * 128u;
    uint32_t wl_off = (uint32_t)W * n_in * 2u;  // byte offset of W1 in the blob
    const float *bias = reinterpret_cast<const float *>(S.blob + bias_off);
    for (int layer = 0; layer <= n_hidden; ++layer) {
      const bool last = layer == n_hidden;
      if (warp < 4) {
        if (!mbar_wait(su32(&S.mbar[kNBuf]), (uint32_t)(acc_ctr & 1))) aborted = true;
        tc_after();
        const int r = warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        if (!last) {
          const float *bl = bias + layer * W;
#pragma unroll 1
          for (int c0 = 0; c0 < W; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; c += 8) {
              float h8[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) h8[u] = act_fn(__uint_as_float(v[c + u]) + bl[c0 + c + u], act);
              uint4 pk = make_uint4(pack_bf16(h8[0], h8[1]), pack_bf16(h8[2], h8[3]), pack_bf16(h8[4], h8[5]),
                                    pack_bf16(h8[6], h8[7]));
              *reinterpret_cast<uint4 *>(S.act + core_off(r, (c0 + c) / 8, act_sbo)) = pk;
            }
          }
        } else {
          // logits 16 columns at a time into a per-thread array, then decode
          float z[64];
          const float *bl = bias + layer * W;
#pragma unroll 1
          for (int c0 = 0; c0 < n_out_pad; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) z[c0 + u] = __uint_as_float(v[u]) + bl[c0 + u];
          }
          const int32_t ray = S.ray[r];
          if (ray >= 0 && !aborted) {
            if (XROWS) {
              for (int j = 0; j < n_out; ++j) a.Z[(int64_t)ray * n_out + j] = z[j];
            } else {
              decode_store(q.hits, ray, z, n_out, n_mat, S.t0[r], S.t1[r], q.rays.tmin[ray], q.rays.tmax[ray]);
            }
          }
        }
        if (!last) fence_async_smem();
        tc_before();
      }
      ++acc_ctr;
      if (aborted) S.misc[1] = 1;
      __syncthreads();
      if (!last && tid == 0) {
        tc_after();
        const int N = (layer + 1 < n_hidden) ? W : n_out_pad;
        const uint32_t a0 = su32(S.act), b0 = su32(S.blob) + wl_off;
        const uint32_t idesc = idesc_bf16(N);
        for (int ks = 0; ks < W / 16; ++ks) {
          const uint64_t ad = umma_desc(a0 + ks * 256, 128, act_sbo);
          const uint64_t bd = umma_desc(b0 + ks * 256, 128, act_sbo);
          mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(su32(&S.mbar[kNBuf]));
      }
      if (!last) wl_off += (uint32_t)((layer + 1 < n_hidden) ? W : n_out_pad) * W * 2u;
    }
    if (aborted) S.misc[1] = 1;
  }
  if (aborted || S.misc[1]) {
    if (tid == 0) atomicOr(q.err, kErrWaitTimeout);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

bool fused_supported(const DevObject &h) {
  if (!(h.F == 2 || h.F == 4)) return false;
  if (!(h.width == 64 || h.width == 128)) return false;
  if ((h.L * h.F) % 8 != 0 || h.L > 16) return false;
  if (h.n_out_pad > 64) return false;
  return true;
}

size_t fused_smem_bytes(const DevObject &h) {
  size_t blob = ((size_t)h.umma_bytes + 1023) & ~size_t(1023);
  size_t ring = (size_t)kNBuf * kTileM * (2 * 16 * h.F) * 2;
  size_t actb = (size_t)kTileM * h.width * 2;
  size_t tail = kTileM * 16 + 8 * (2 * kNBuf + 1) + 16 + 16 + 4 * LSNIF_MAX_LEVELS;
  return 1024 + blob + ring + actb + tail;
}

template <int F, int W, bool XR, int NT, int NLB>
static cudaError_t launch_one(const FusedArgs &a, size_t smem, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<F, W, XR, NT, NLB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = 1;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  fused_kernel<F, W, XR, NT, NLB><<<sms, NT, smem, st>>>(a);
  return cudaGetLastError();
}

// Tile-shape variants the autotuner chooses between: threads per CTA and
// levels of corner loads in flight per gather item.
struct Variant {
  int threads, levels;
};
static const Variant kVariants[] = {{512, 1}, {512, 2}, {512, 4}, {1024, 1}, {1024, 2}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

template <int F, int W, bool XR>
static cudaError_t dispatch_variant(const FusedArgs &a, int v, size_t smem, cudaStream_t st) {
  constexpr int LPG = 8 / F;
  switch (v) {
    case 0: return launch_one<F, W, XR, 512, 1>(a, smem, st);
    case 1: return launch_one<F, W, XR, 512, (2 < LPG ? 2 : LPG)>(a, smem, st);
    case 2: return launch_one<F, W, XR, 512, LPG>(a, smem, st);
    case 3: return launch_one<F, W, XR, 1024, 1>(a, smem, st);
    case 4: return launch_one<F, W, XR, 1024, (2 < LPG ? 2 : LPG)>(a, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

template <bool XR>
static cudaError_t dispatch(const FusedArgs &a, const DevObject &h, int variant, size_t smem, cudaStream_t st) {
  if (h.F == 2 && h.width == 64) return dispatch_variant<2, 64, XR>(a, variant, smem, st);
  if (h.F == 2 && h.width == 128) return dispatch_variant<2, 128, XR>(a, variant, smem, st);
  if (h.F == 4 && h.width == 64) return dispatch_variant<4, 64, XR>(a, variant, smem, st);
  if (h.F == 4 && h.width == 128) return dispatch_variant<4, 128, XR>(a, variant, smem, st);
  return cudaErrorNotSupported;
}

int fused_variant_count() { return kNumVariants; }

void fused_variant_shape(int v, int *threads, int *levels) {
  *threads = kVariants[v].threads;
  *levels = kVariants[v].levels;
}

cudaError_t launch_fused(const QueryLaunch &q, const DevObject &h, int variant, int *launches) {
  if (!fused_supported(h)) return cudaErrorNotSupported;
  size_t smem = fused_smem_bytes(h);
  if (smem > 232448) return cudaErrorNotSupported;
  if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.q = q;
  a.smem_blob = h.umma_bytes;
  *launches += 1;
  return dispatch<false>(a, h, variant, smem, q.stream);
}

cudaError_t launch_mlp_fused(const DevObject *dobj, const DevObject &h, const float *X, int64_t n, float *Z,
                             int *err, cudaStream_t st) {
  if (!fused_supported(h)) return cudaErrorNotSupported;
  size_t smem = fused_smem_bytes(h);
  if (smem > 232448) return cudaErrorNotSupported;
  int32_t *meta = nullptr;
  cudaError_t e = cudaMallocAsync(&meta, 16 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(meta, 0, 16 * sizeof(int32_t), st);
  FusedArgs a{};
  a.q.objs = dobj;
  a.q.n_slots = 1;
  a.q.H_max = h.H;
  a.q.err = err;
  a.q.s.meta = meta;
  a.X = X;
  a.Z = Z;
  a.xrows = n;
  a.smem_blob = h.umma_bytes;
  e = dispatch<true>(a, h, 1, smem, st);
  cudaFreeAsync(meta, st);
  return e;
}

}  // namespace lsnif
