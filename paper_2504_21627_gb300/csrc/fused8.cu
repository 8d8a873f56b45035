// FP8 (E4M3) fused query kernel for sm_103a. Same structure as the BF16
// kernel in fused.cu (per-tile work lists, gather warps, one MMA warp, four
// epilogue warps that also set tiles up ahead, two TMEM accumulators), with
// FP8 operands and tcgen05.mma kind::f8f6f4 (FP32 accumulation):
//   - the network input is E4M3(s_0 x), layer l's weights E4M3(w_l W_l), and
//     every hidden activation E4M3(s_{l+1} h); each accumulator is multiplied
//     by 1 / (s_l w_l) before the bias (power-of-two scales chosen on the
//     host from the parameters, rounding to nearest even, saturating);
//   - the first layer's weights are streamed chunk by chunk into the ring
//     next to each chunk's A tile: with F = 4, L = 16 and 4 x 128 neurons
//     they are 147 KB, which do not fit shared memory beside the rest; the
//     hidden and output layers stay resident.
// One 16-byte column group of a point holds 16 E4M3 features (16 / F
// levels).
#include <algorithm>
#include <climits>
#include <cstdio>

#include <cuda_fp8.h>

#include "device.cuh"
#include "encode.cuh"
#include "tc_common.cuh"

namespace lsnif {

namespace {

constexpr int kNBufMax = 4;
constexpr int kEpiWarps = 4;

// kind::f8f6f4 instruction descriptor: E4M3 A and B (K-major), FP32 D, M = 128
__device__ __forceinline__ uint32_t idesc_e4m3(int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// two values -> two E4M3 bytes (lo in the low byte), round to nearest even,
// saturating to +-448; one cvt instruction converts the pair
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}

// four values -> four E4M3 bytes, the first in the lowest byte
__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d) {
  return e4m3x2(a, b) | (e4m3x2(c, d) << 16);
}

// 1-D bulk copy global -> shared, completing on an mbarrier (sizes and both
// addresses multiples of 16 bytes)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

struct Fused8Args {
  QueryLaunch q;
  uint32_t smem_blob;  // bytes of the resident blob (hidden + output layers, biases, scales)
  int nbuf;            // ring buffers (2..kNBufMax)
  int list_chunks;     // work-list capacity in chunks (H_max / 2)
};

// Shared-memory layout; one ring slot holds a chunk's A tile (128 x CHK
// bytes) and its first-layer weights (W x CHK bytes), for L <= 16.
struct Layout8 {
  uint32_t blob, ring, slot_a, slot_w, ring_stride, act, ray, t0, t1, list, wsum, info, bars, tmem, misc, res,
      total;
};

// mbarriers: full[kNBufMax], empty[kNBufMax], tile_ready[2], acc_full[2],
// acc_empty[2], layer_done, fin[2], wfull[kNBufMax] (first-layer weights
// of a ring slot landed)
constexpr int kNumBars8 = 2 * kNBufMax + 2 + 2 + 2 + 1 + 2 + kNBufMax;

__host__ __device__ inline Layout8 make_layout8(uint32_t blob_bytes, int F, int W, int nbuf, int list_chunks) {
  Layout8 o{};
  uint32_t off = 0;
  const uint32_t chk = 2u * 16u * (uint32_t)F;
  o.slot_a = 0;
  o.slot_w = (uint32_t)kTileM * chk;
  o.ring_stride = o.slot_w + (uint32_t)W * chk;
  o.blob = lay_take(off, blob_bytes, 1024);
  o.ring = lay_take(off, (uint32_t)nbuf * o.ring_stride, 1024);
  o.act = lay_take(off, (uint32_t)kTileM * W, 1024);
  o.ray = lay_take(off, 2 * kTileM * 4, 16);
  o.t0 = lay_take(off, 2 * kTileM * 4, 16);
  o.t1 = lay_take(off, 2 * kTileM * 4, 16);
  o.list = lay_take(off, 2u * (uint32_t)list_chunks * kListStride * 2u, 16);
  o.wsum = lay_take(off, 2u * (uint32_t)list_chunks * 4u * 4u, 16);
  o.info = lay_take(off, 2 * sizeof(TileInfo), 16);
  o.bars = lay_take(off, 8 * kNumBars8, 8);
  o.tmem = lay_take(off, 16, 16);
  o.misc = lay_take(off, 16 * 4, 16);
  o.res = lay_take(off, 4 * LSNIF_MAX_LEVELS, 16);
  o.total = off + 1024;
  return o;
}

struct Smem8 {
  uint8_t *blob, *ring, *act;
  int32_t *ray;
  float *t0, *t1;
  uint16_t *list;
  uint32_t *wsum;
  TileInfo *info;
  uint64_t *full, *empty, *ready, *accf, *acce, *layer, *fin, *wfull;
  uint32_t *tmem;
  int32_t *misc;
  volatile int *abort_flag;
  float *res;
  uint32_t ring_stride, slot_w;
};

template <int F, int W>
__device__ __forceinline__ Smem8 carve8(const Fused8Args &a, uint8_t *base) {
  const Layout8 l = make_layout8(a.smem_blob, F, W, a.nbuf, a.list_chunks);
  Smem8 S;
  S.blob = base + l.blob;
  S.ring = base + l.ring;
  S.act = base + l.act;
  S.ray = reinterpret_cast<int32_t *>(base + l.ray);
  S.t0 = reinterpret_cast<float *>(base + l.t0);
  S.t1 = reinterpret_cast<float *>(base + l.t1);
  S.list = reinterpret_cast<uint16_t *>(base + l.list);
  S.wsum = reinterpret_cast<uint32_t *>(base + l.wsum);
  S.info = reinterpret_cast<TileInfo *>(base + l.info);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + l.bars);
  S.full = bars;
  S.empty = bars + kNBufMax;
  S.ready = bars + 2 * kNBufMax;
  S.accf = S.ready + 2;
  S.acce = S.ready + 4;
  S.layer = S.ready + 6;
  S.fin = S.ready + 7;
  S.wfull = S.ready + 9;
  S.tmem = reinterpret_cast<uint32_t *>(base + l.tmem);
  S.misc = reinterpret_cast<int32_t *>(base + l.misc);
  S.abort_flag = reinterpret_cast<volatile int *>(S.misc + 4);
  S.res = reinterpret_cast<float *>(base + l.res);
  S.ring_stride = l.ring_stride;
  S.slot_w = l.slot_w;
  return S;
}

// FP32 trailer of the resident blob: biases of every layer, then 1 / (s_l w_l)
// per layer, then the input scale s_l per layer
struct Trailer8 {
  const float *bias, *inv_sw, *s_in;
};

__device__ __forceinline__ Trailer8 trailer8(const DevObject &ob, const uint8_t *blob) {
  const float *b = reinterpret_cast<const float *>(blob + ob.blob8_bias_off);
  const float *sc = reinterpret_cast<const float *>(blob + ob.blob8_scale_off);
  return Trailer8{b, sc, sc + (ob.n_hidden + 1)};
}

}  // namespace

// ---------------------------------------------------------------------------
// MMA warp: per chunk, stream the first-layer weight slice into the ring slot
// once the slot is free, wait for the gathered A tile, issue the MMAs.
// ---------------------------------------------------------------------------
template <int F, int W, int NG>
__device__ __noinline__ void mma8_role(const Fused8Args *ap, uint8_t *base, uint32_t tmem) {
  const Fused8Args &a = *ap;
  const int lane = threadIdx.x & 31;
  const DevObject *objs = a.q.objs;
  const int nbuf = a.nbuf;
  const Smem8 S = carve8<F, W>(a, base);
  int rbuf = 0, ruse = 0;  // ring slot and pass of the next chunk
  const uint32_t idesc0 = idesc_e4m3(W);
  for (int i = 0;; ++i) {
    const int tb = i & 1;
    if (!mbar_wait_sleep(su32(&S.ready[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag)) break;
    const TileInfo ti = S.info[tb];
    if (ti.stop) break;
    const DevObject &ob = objs[ti.slot];
    const int CHK = 2 * ob.L * F;  // bytes = elements
    const uint32_t sbo = (uint32_t)(CHK / 16) * 128u;
    const uint32_t slice = (uint32_t)W * CHK;
    if (i >= 2 && !mbar_wait_sleep(su32(&S.acce[tb]), (uint32_t)(((i - 2) >> 1) & 1), S.abort_flag)) break;
    tc_after();
    const uint32_t dacc = tmem + (uint32_t)(tb * W);
    bool ok = true;
    for (int s = 0; s < ti.kmax; ++s) {
      // ring slot and pass of the next chunk, kept as counters (no division
      // by the run-time ring size)
      const int buf = rbuf, use = ruse;
      if (++rbuf == nbuf) {
        rbuf = 0;
        ++ruse;
      }
      uint8_t *slot = S.ring + buf * S.ring_stride;
      // the slot's previous MMAs must be done before its weights are replaced
      if (use > 0 && !mbar_wait_sleep(su32(&S.empty[buf]), (uint32_t)((use - 1) & 1), S.abort_flag)) {
        ok = false;
        break;
      }
      // the weight slice travels by bulk copy while the gather warps fill
      // the A tile of the same slot
      if (lane == 0) bulk_g2s(su32(slot + S.slot_w), ob.w0_8 + (size_t)s * slice, slice, su32(&S.wfull[buf]));
      const bool got_a = mbar_wait_sleep(su32(&S.full[buf]), (uint32_t)(use & 1), S.abort_flag);
      // the copy is waited for even after an abort: it must land before the
      // shared memory is released
      const bool got_w = got_a ? mbar_wait_sleep(su32(&S.wfull[buf]), (uint32_t)(use & 1), S.abort_flag)
                               : mbar_wait_teardown(su32(&S.wfull[buf]), (uint32_t)(use & 1));
      if (!got_a || !got_w) {
        if (!got_w) *S.abort_flag = 1;
        ok = false;
        break;
      }
      tc_after();
      if (lane == 0) {
        const uint32_t a0 = su32(slot), b0 = su32(slot + S.slot_w);
        for (int ks = 0; ks < CHK / 32; ++ks) {
          const uint64_t ad = umma_desc(a0 + ks * 256, 128, sbo);
          const uint64_t bd = umma_desc(b0 + ks * 256, 128, sbo);
          mma_e4m3(dacc, ad, bd, idesc0, (s > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(su32(&S.empty[buf]));
      }
      __syncwarp();
    }
    if (!ok) break;
    if (lane == 0) mma_commit(su32(&S.accf[tb]));
    __syncwarp();
  }
  if (lane == 0) {
    mma_commit(su32(&S.fin[0]));
    if (!mbar_wait_teardown(su32(&S.fin[0]), 0u)) *S.abort_flag = 1;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Epilogue warps: tile setup one tile ahead, then the hidden and output
// layers (dequantise, bias, activation, requantise to E4M3) and the decode.
// ---------------------------------------------------------------------------
template <int F, int W, int NG>
__device__ __noinline__ void epilogue8_role(const Fused8Args *ap, uint8_t *base, uint32_t tmem) {
  const Fused8Args &a = *ap;
  constexpr int kEpiWarp0 = NG + 1;
  constexpr int kEpiThreads = kEpiWarps * 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  const Smem8 S = carve8<F, W>(a, base);
  const int64_t n_tiles = (int64_t)q.s.meta[1];
  const int etid = tid - kEpiWarp0 * 32;
  const int ew = etid >> 5;
  const int quarter = warp & 3;
  const int r = quarter * 32 + lane;
  const uint32_t act_sbo = (uint32_t)(W / 16) * 128u;
  int layer_ctr = 0;
  int su_slot = -1;

  auto fetch = [&]() -> int {
    named_sync(2, kEpiThreads);
    if (etid == 0) S.misc[0] = *S.abort_flag ? INT_MAX : atomicAdd(q.s.meta + 3, 1);
    named_sync(2, kEpiThreads);
    return S.misc[0];
  };
  auto slot_of_tile = [&](int tile) -> int { return q.s.tiles[3 * tile + 0]; };
  auto setup = [&](int j, int tile) {
    const int sb = j & 1;
    if ((int64_t)tile >= n_tiles) {
      if (etid == 0) {
        S.info[sb].stop = 1;
        mbar_arrive(su32(&S.ready[sb]));
      }
      return;
    }
    const int slot = q.s.tiles[3 * tile + 0];
    const int start = q.s.tiles[3 * tile + 1];
    const int cnt = q.s.tiles[3 * tile + 2];
    const DevObject &ob = objs[slot];
    if (slot != su_slot) {
      const uint4 *src = reinterpret_cast<const uint4 *>(ob.blob8);
      uint4 *dst = reinterpret_cast<uint4 *>(S.blob);
      const int nvec = (int)(ob.blob8_bytes / 16);
      for (int k = etid; k < nvec; k += kEpiThreads) dst[k] = __ldg(src + k);
      if (etid < LSNIF_MAX_LEVELS) S.res[etid] = (float)ob.res[etid];
      fence_async_smem();
      su_slot = slot;
    }
    if (etid == 0) S.misc[1] = 0;
    named_sync(2, kEpiThreads);
    int my_kk = 0;
    uint32_t my_dm = 0u;
    {
      int ray = -1;
      float t0v = 0.f, t1v = 0.f;
      if (etid < cnt) {
        ray = q.s.order[start + etid];
        my_kk = q.s.k[ray];
        my_dm = q.s.dup[ray];
        const float2 tt = reinterpret_cast<const float2 *>(q.s.t01)[ray];
        t0v = tt.x;
        t1v = tt.y;
      }
      S.ray[sb * kTileM + etid] = ray;
      S.t0[sb * kTileM + etid] = t0v;
      S.t1[sb * kTileM + etid] = t1v;
      const int wm = __reduce_max_sync(0xffffffffu, my_kk);
      if (lane == 0) atomicMax(&S.misc[1], wm);
    }
    named_sync(2, kEpiThreads);
    const int kmax = S.misc[1];
    uint16_t *lst = S.list + (size_t)sb * a.list_chunks * kListStride;
    uint32_t *ws = S.wsum + (size_t)sb * a.list_chunks * 4;
    for (int s = 0; s < kmax; ++s) {
      const uint32_t tot = __reduce_add_sync(0xffffffffu, row_counts(my_kk, my_dm, s));
      if (lane == 0) ws[s * 4 + ew] = tot;
    }
    named_sync(2, kEpiThreads);
    for (int s = 0; s < kmax; ++s) {
      const uint32_t v = row_counts(my_kk, my_dm, s);
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t woff = 0, all = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const uint32_t x = ws[s * 4 + w];
        all += x;
        woff += w < ew ? x : 0u;
      }
      const uint32_t pos = incl - v + woff;
      const int ngt = (int)(all & 1023u), nct = (int)((all >> 10) & 1023u);
      uint16_t *Ls = lst + s * kListStride;
      if (v & 1023u) {
        const int pg = (int)(pos & 1023u);
        if (v & (1023u << 10)) {
          Ls[pg] = (uint16_t)(etid | 128);
          Ls[ngt + (int)((pos >> 10) & 1023u)] = (uint16_t)etid;
        } else {
          Ls[pg] = (uint16_t)etid;
          Ls[pg + 1] = (uint16_t)(etid | 128);
        }
      } else {
        const int pz = ngt + nct + (int)((pos >> 20) & 1023u);
        Ls[pz] = (uint16_t)etid;
        Ls[pz + 1] = (uint16_t)(etid | 128);
      }
    }
    named_sync(2, kEpiThreads);
    if (etid == 0) {
      S.info[sb].kmax = kmax;
      S.info[sb].slot = slot;
      S.info[sb].stop = 0;
      mbar_arrive(su32(&S.ready[sb]));
    }
  };

  int stop_at = INT_MAX;
  {
    const int t0i = fetch();
    setup(0, t0i);
    if ((int64_t)t0i >= n_tiles) stop_at = 0;
  }
  for (int i = 0; i < stop_at; ++i) {
    const int tb = i & 1;
    const int tn = fetch();
    const bool last = (int64_t)tn >= n_tiles;
    const bool deferred = !last && slot_of_tile(tn) != su_slot;
    if (!deferred) setup(i + 1, tn);
    if (last) stop_at = i + 1;

    if (etid == 0) S.misc[2] = mbar_wait_sleep(su32(&S.accf[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag) ? 0 : 1;
    named_sync(2, kEpiThreads);
    if (!S.misc[2]) {
      tc_after();
      const TileInfo ti = S.info[tb];
      const DevObject &ob = objs[ti.slot];
      const int n_hidden = ob.n_hidden, n_out = ob.n_out, n_out_pad = ob.n_out_pad, n_mat = ob.n_mat,
                act = ob.act;
      const Trailer8 tr = trailer8(ob, S.blob);
      uint32_t wl_off = 0;  // byte offset of the next layer's weights in the blob
      const uint32_t dacc = tmem + (uint32_t)(tb * W);
      const uint32_t trow = dacc + ((uint32_t)(quarter * 32) << 16);
      for (int layer = 0; layer <= n_hidden; ++layer) {
        const bool out_layer = layer == n_hidden;
        const float *bl = tr.bias + layer * W;
        const float isw = tr.inv_sw[layer];
        if (!out_layer) {
          const float s_next = tr.s_in[layer + 1];
#pragma unroll 1
          for (int c0 = 0; c0 < W; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
            float h[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) h[u] = act_fn(fmaf(__uint_as_float(v[u]), isw, bl[c0 + u]), act) * s_next;
            const uint4 pk = make_uint4(pack_e4m3(h[0], h[1], h[2], h[3]), pack_e4m3(h[4], h[5], h[6], h[7]),
                                        pack_e4m3(h[8], h[9], h[10], h[11]), pack_e4m3(h[12], h[13], h[14], h[15]));
            *reinterpret_cast<uint4 *>(S.act + core_off(r, c0 / 16, act_sbo)) = pk;
          }
          fence_async_smem();
          tc_before();
          named_sync(2, kEpiThreads);
          const int N = (layer + 1 < n_hidden) ? W : n_out_pad;
          if (etid == 0) {
            tc_after();
            const uint32_t a0 = su32(S.act), b0 = su32(S.blob) + wl_off;
            const uint32_t idesc = idesc_e4m3(N);
            for (int ks = 0; ks < W / 32; ++ks) {
              const uint64_t ad = umma_desc(a0 + ks * 256, 128, act_sbo);
              const uint64_t bd = umma_desc(b0 + ks * 256, 128, act_sbo);
              mma_e4m3(dacc, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            mma_commit(su32(S.layer));
            mbar_wait_sleep(su32(S.layer), (uint32_t)(layer_ctr & 1), S.abort_flag);
          }
          ++layer_ctr;
          named_sync(2, kEpiThreads);
          tc_after();
          wl_off += (uint32_t)N * W;
        } else {
          float z[64];
#pragma unroll 1
          for (int c0 = 0; c0 < n_out_pad; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) z[c0 + u] = fmaf(__uint_as_float(v[u]), isw, bl[c0 + u]);
          }
          const int32_t ray = S.ray[tb * kTileM + r];
          if (ray >= 0 && !*S.abort_flag)
            decode_store(q.hits, ray, z, n_out, n_mat, S.t0[tb * kTileM + r], S.t1[tb * kTileM + r],
                         q.rays.tmin[ray], q.rays.tmax[ray]);
        }
      }
    }
    tc_before();
    mbar_arrive(su32(&S.acce[tb]));
    if (deferred) {
      named_sync(2, kEpiThreads);
      setup(i + 1, tn);
    }
  }
  if (etid == 0) {
    mma_commit(su32(&S.fin[1]));
    if (!mbar_wait_teardown(su32(&S.fin[1]), 0u)) *S.abort_flag = 1;
  }
}

// ---------------------------------------------------------------------------
// the kernel: setup, gather warps inline, the other roles as functions
// ---------------------------------------------------------------------------
template <int F, int W, int NG, int NL>
__global__ void __launch_bounds__((NG + 1 + kEpiWarps) * 32, 1) fused8_kernel(const __grid_constant__ Fused8Args a) {
  constexpr int kGatherThreads = NG * 32;
  constexpr int kMmaWarp = NG;
  constexpr int kTmemCols = 2 * W;
  constexpr int LPG = 16 / F;  // levels per 16-byte column group
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  const int nbuf = a.nbuf;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem8 S = carve8<F, W>(a, base);

  if (tid == 0) {
    for (int b = 0; b < nbuf; ++b) {
      mbar_init(su32(&S.full[b]), kGatherThreads);
      mbar_init(su32(&S.empty[b]), 1);
      mbar_init(su32(&S.wfull[b]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&S.ready[b]), 1);
      mbar_init(su32(&S.accf[b]), 1);
      mbar_init(su32(&S.acce[b]), kEpiWarps * 32);
      mbar_init(su32(&S.fin[b]), 1);
    }
    mbar_init(su32(S.layer), 1);
    // make the initialised barriers visible to the bulk-copy unit
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *S.abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(S.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *S.tmem;
  const int Hs = q.H_max;

  if (warp < NG) {
    // =================== gather warps ===================
    int cur_slot = -1;
    int L = 0;
    uint32_t mask = 0;
    const uint16_t *tab = nullptr;
    float s0 = 1.f;  // scale of the network input
    int rbuf = 0, ruse = 0;  // ring slot and pass of the next chunk
    int rot_g = 0, rot_o = 0;
    for (int i = 0;; ++i) {
      const int tb = i & 1;
      if (!mbar_wait_sleep(su32(&S.ready[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag)) break;
      const TileInfo ti = S.info[tb];
      if (ti.stop) break;
      const int kmax = ti.kmax;
      if (ti.slot != cur_slot) {
        const DevObject &ob = objs[ti.slot];
        L = ob.L;
        mask = ob.mask;
        tab = ob.tab16;
        s0 = trailer8(ob, S.blob).s_in[0];
        cur_slot = ti.slot;
      }
      const uint16_t *s_lst = S.list + (size_t)tb * a.list_chunks * kListStride;
      const uint32_t *s_ws = S.wsum + (size_t)tb * a.list_chunks * 4;
      const int G = (L * F) / 16;  // 16-byte column groups per point
      const int CHK = 2 * L * F;   // bytes per chunk row
      const uint32_t a_sbo = (uint32_t)(CHK / 16) * 128u;
      const size_t lstride = (size_t)(mask + 1) * F;
      for (int s = 0; s < kmax; ++s) {
        // ring slot and pass of this warp's c-th chunk (c = use nbuf + buf),
        // kept as counters: no division by the run-time ring size
        const int buf = rbuf, use = ruse;
        if (++rbuf == nbuf) {
          rbuf = 0;
          ++ruse;
        }
        // chunk c - 1 (whose exit points the copies read) and chunk
        // c - nbuf + 1 (which read this slot's previous chunk)
        const int pbuf = buf > 0 ? buf - 1 : nbuf - 1, puse = buf > 0 ? use : use - 1;
        const bool wrap = buf + 1 == nbuf;
        const int nbuf1 = wrap ? 0 : buf + 1, nuse1 = wrap ? use : use - 1;
        uint8_t *A = S.ring + buf * S.ring_stride;
        uint32_t all = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) all += s_ws[s * 4 + w];
        const int ngt = (int)(all & 1023u), nct = (int)((all >> 10) & 1023u);
        const int n_gi = ngt * G, n_oi = (kListStride - ngt) * G;
        const int nb_g = (n_gi + 31) >> 5, nb_o = (n_oi + 31) >> 5;
        const int first_g = (warp - rot_g + NG) % NG, first_o = (warp - rot_o + NG) % NG;
        if (use > 0) mbar_wait_sleep(su32(&S.empty[buf]), (uint32_t)((use - 1) & 1), S.abort_flag);
        if (nbuf > 1 && nuse1 >= 0) mbar_wait_sleep(su32(&S.full[nbuf1]), (uint32_t)(nuse1 & 1), S.abort_flag);
        const float inv_g = 1.f / (float)max(ngt, 1);
        for (int b = first_g; b < nb_g; b += NG) {
          const int it = b * 32 + lane;
          if (it < n_gi) {
            const int g = __float2int_rz(((float)it + 0.5f) * inv_g);
            const int t = it - g * ngt;
            const int e = s_lst[s * kListStride + t];
            const int r = e & 127, j = e >> 7;
            const int ray = S.ray[tb * kTileM + r];
            const float *P = q.s.pts + ((size_t)ray * Hs + 2 * s + j) * 3;
            const float3 p = make_float3(P[0], P[1], P[2]);
            // FP32 interpolation of the FP16 entries: the E4M3 rounding that
            // follows then sees the feature to FP32 accuracy. Each pair of
            // levels is scaled and packed at once (2F bytes).
            uint32_t wv[4];
            static_assert(F == 4 || NL % 2 == 0, "F = 2 packs levels in pairs");
#pragma unroll
            for (int u0 = 0; u0 < LPG; u0 += NL) {
              const int l = g * LPG + u0;
              float f[NL][F];
              encode_levels_f16<F, NL>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride, lstride * 2,
                                       mask, p, S.res + l, f);
#pragma unroll
              for (int u = 0; u < NL; ++u) {
                if constexpr (F == 4) {
                  wv[u0 + u] = pack_e4m3(f[u][0] * s0, f[u][1] * s0, f[u][2] * s0, f[u][3] * s0);
                } else if (u % 2 == 0) {
                  wv[(u0 + u) / 2] = pack_e4m3(f[u][0] * s0, f[u][1] * s0, f[u + 1][0] * s0, f[u + 1][1] * s0);
                }
              }
            }
            const uint4 outv = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            *reinterpret_cast<uint4 *>(A + core_off(r, j * G + g, a_sbo)) = outv;
          }
        }
        const int n_o = kListStride - ngt;
        if (nct > 0 && first_o < nb_o) mbar_wait_sleep(su32(&S.full[pbuf]), (uint32_t)(puse & 1), S.abort_flag);
        const float inv_o = 1.f / (float)max(n_o, 1);
        for (int b = first_o; b < nb_o; b += NG) {
          const int it = b * 32 + lane;
          if (it < n_oi) {
            const int g = __float2int_rz(((float)it + 0.5f) * inv_o);
            const int t = it - g * n_o;
            const int e = s_lst[s * kListStride + ngt + t];
            const int r = e & 127, j = e >> 7;
            uint4 outv = make_uint4(0u, 0u, 0u, 0u);
            if (t < nct) {
              const uint8_t *Ap = S.ring + pbuf * S.ring_stride;
              outv = *reinterpret_cast<const uint4 *>(Ap + core_off(r, G + g, a_sbo));
            }
            *reinterpret_cast<uint4 *>(A + core_off(r, j * G + g, a_sbo)) = outv;
          }
        }
        rot_g = (rot_g + nb_g) % NG;
        rot_o = (rot_o + nb_o) % NG;
        fence_async_smem();
        mbar_arrive(su32(&S.full[buf]));
      }
    }
  } else if (warp == kMmaWarp) {
    mma8_role<F, W, NG>(&a, base, tmem);
  } else {
    epilogue8_role<F, W, NG>(&a, base, tmem);
  }

  tc_before();
  __syncthreads();
  tc_after();
  if (tid == 0 && *S.abort_flag) atomicOr(q.err, kErrWaitTimeout);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {
__global__ void max_abs_half_kernel(const uint16_t *v, int64_t n, uint32_t *out) {
  uint32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float f = fabsf(__half2float(__ushort_as_half(v[i])));
    m = max(m, f == f ? __float_as_uint(f) : 0u);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
}  // namespace

// largest |value| of an FP16 array, as FP32 bits in *out_bits (device)
cudaError_t launch_max_abs_half(const uint16_t *v, int64_t n, uint32_t *out_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out_bits, 0, 4, st);
  if (e != cudaSuccess) return e;
  max_abs_half_kernel<<<1024, 256, 0, st>>>(v, n, out_bits);
  return cudaGetLastError();
}

bool fused8_supported(const DevObject &h) {
  if (!(h.F == 2 || h.F == 4)) return false;
  if (!(h.width == 64 || h.width == 128)) return false;
  if ((h.L * h.F) % 16 != 0 || h.L > 16) return false;
  if (h.n_out_pad > 64) return false;
  return true;
}

static int pick_nbuf8(const DevObject &h, int list_chunks, uint32_t blob) {
  for (int nb = kNBufMax; nb >= 2; --nb)
    if (make_layout8(blob, h.F, h.width, nb, list_chunks).total <= 232448) return nb;
  return 0;
}

size_t fused8_smem_bytes(const DevObject &h, int H_max) {
  return make_layout8((h.blob8_bytes + 15u) & ~15u, h.F, h.width, 2, std::max(H_max, h.H) / 2).total;
}

// kernel shapes: gather warps x levels per corner-load batch (F = 4; F = 2
// always runs the first)
struct Variant8 {
  int ng, nl;
};
constexpr Variant8 kVariants8[] = {{11, 2}, {15, 2}, {19, 1}};
constexpr int kNumVariants8 = (int)(sizeof(kVariants8) / sizeof(kVariants8[0]));

template <int F, int W, int NG, int NL>
static cudaError_t launch8_shape(const Fused8Args &a, size_t smem, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(fused8_kernel<F, W, NG, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = 1;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one persistent CTA per SM, but no more CTAs than the batch can have tiles
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (int64_t)a.q.s.max_tiles));
  fused8_kernel<F, W, NG, NL><<<grid, (NG + 1 + kEpiWarps) * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int F, int W>
static cudaError_t launch8_one(const Fused8Args &a, size_t smem, cudaStream_t st, int variant) {
  if constexpr (F == 4) {
    if (variant == 1) return launch8_shape<F, W, 15, 2>(a, smem, st);
    if (variant == 2) return launch8_shape<F, W, 19, 1>(a, smem, st);
  }
  return launch8_shape<F, W, 11, 2>(a, smem, st);
}

int fused8_variant_count() { return kNumVariants8; }

void fused8_variant_shape(int v, int *threads, int *levels) {
  *threads = kVariants8[v].ng * 32;
  *levels = kVariants8[v].nl;
}

cudaError_t launch_fused8(const QueryLaunch &q, const DevObject &h, int variant, int *launches) {
  if (!fused8_supported(h)) return cudaErrorNotSupported;
  Fused8Args a{};
  a.q = q;
  a.smem_blob = (h.blob8_bytes + 15u) & ~15u;
  a.list_chunks = std::max(q.H_max, h.H) / 2;
  a.nbuf = pick_nbuf8(h, a.list_chunks, a.smem_blob);
  if (!a.nbuf) return cudaErrorNotSupported;
  const size_t smem = make_layout8(a.smem_blob, h.F, h.width, a.nbuf, a.list_chunks).total;
  *launches += 1;
  if (h.F == 2 && h.width == 64) return launch8_one<2, 64>(a, smem, q.stream, variant);
  if (h.F == 2 && h.width == 128) return launch8_one<2, 128>(a, smem, q.stream, variant);
  if (h.F == 4 && h.width == 64) return launch8_one<4, 64>(a, smem, q.stream, variant);
  if (h.F == 4 && h.width == 128) return launch8_one<4, 128>(a, smem, q.stream, variant);
  return cudaErrorNotSupported;
}

}  // namespace lsnif
