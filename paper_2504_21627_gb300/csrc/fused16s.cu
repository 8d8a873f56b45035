// Fused FP16 query kernel for networks whose weights do not fit shared
// memory beside the ring: the path-tracing stress configuration's objects
// (16 levels x 4 features, 1152 -> 128 x 4 -> 12: 295 KB of FP16 first-layer
// weights alone). Same work units, roles, work lists, shared-point copies,
// two TMEM accumulators and bounded waits as the resident kernel in
// fused.cu, with two differences:
//   - the first layer's weights are streamed: the MMA warp moves each
//     chunk's W x CHK slice (a contiguous part of the chunk-major copy
//     w0_16c) into the ring slot beside the chunk's A tile with a 1-D bulk
//     copy completing on a per-slot mbarrier, then issues the chunk's MMAs;
//   - the later layers' weights are loaded one layer at a time into one
//     shared buffer by a bulk copy the epilogue issues as soon as the
//     previous layer's MMAs have read it; the activations go to TMEM.
// Operands FP16 (tcgen05 kind::f16, A and B FP16), FP32 accumulation: the
// gather interpolates in FP32 from the FP16 tables and rounds each feature
// once to FP16 (saturating at +-65504), as the FP8 kernel rounds to E4M3.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "device.cuh"
#include "encode.cuh"
#include "tc_common.cuh"

namespace lsnif {

namespace {

constexpr int kNBuf16s = 2;
constexpr int kEpiWarps16s = 4;

// kind::f16 instruction descriptor: FP16 A and B (K-major), FP32 D, M = 128
__device__ __forceinline__ uint32_t idesc_h16(int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_h16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// the same with A read from tensor memory (lane i = row i, two FP16 per column)
__device__ __forceinline__ void mma_h16_ts(uint32_t tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t h2_sat(float a, float b) {
  a = fminf(fmaxf(a, -65504.f), 65504.f);
  b = fminf(fmaxf(b, -65504.f), 65504.f);
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

// 1-D bulk copy global -> shared completing on an mbarrier (both addresses
// and the size multiples of 16 bytes)
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__host__ __device__ constexpr int tmem_cols16s(int W) { return 3 * W <= 256 ? 256 : 512; }

struct Fused16sArgs {
  QueryLaunch q;
  int list_chunks;  // work-list capacity in chunks (H_max / 2)
  int max_bias;     // floats of the bias buffer (largest object: n_hidden W + n_out_pad)
};

// Shared-memory layout: ring slots [A tile 128 x CHK | first-layer slice
// W x CHK] (16-bit, CHK = 2 x 16 x F columns at most), the layer buffer
// (W x W 16-bit weights), the biases, then the per-tile state.
struct Layout16s {
  uint32_t ring, slot_w, ring_stride, lbuf, bias, ray, t0, t1, list, wsum, info, bars, tmem, misc, res, total;
};

// mbarriers: full[2], empty[2], wfull[2] (a slot's first-layer slice
// landed), tile_ready[2], acc_full[2], acc_empty[2], layer_done, lw_full
// (layer weights landed), fin[2]
constexpr int kNumBars16s = 3 * kNBuf16s + 2 + 2 + 2 + 1 + 1 + 2;

__host__ __device__ inline Layout16s make_layout16s(int F, int W, int list_chunks, int max_bias) {
  Layout16s o{};
  uint32_t off = 0;
  const uint32_t chk = 2u * 16u * (uint32_t)F;
  o.slot_w = (uint32_t)kTileM * chk * 2u;
  o.ring_stride = o.slot_w + (uint32_t)W * chk * 2u;
  o.ring = lay_take(off, (uint32_t)kNBuf16s * o.ring_stride, 1024);
  o.lbuf = lay_take(off, (uint32_t)W * W * 2u, 1024);
  o.bias = lay_take(off, (uint32_t)max_bias * 4u, 16);
  o.ray = lay_take(off, 2 * kTileM * 4, 16);
  o.t0 = lay_take(off, 2 * kTileM * 4, 16);
  o.t1 = lay_take(off, 2 * kTileM * 4, 16);
  o.list = lay_take(off, 2u * (uint32_t)list_chunks * kListStride * 2u, 16);
  o.wsum = lay_take(off, 2u * (uint32_t)list_chunks * 4u * 4u, 16);
  o.info = lay_take(off, 2 * sizeof(TileInfo), 16);
  o.bars = lay_take(off, 8 * kNumBars16s, 8);
  o.tmem = lay_take(off, 16, 16);
  o.misc = lay_take(off, 16 * 4, 16);
  o.res = lay_take(off, 4 * LSNIF_MAX_LEVELS, 16);
  o.total = off + 1024;
  return o;
}

struct Smem16s {
  uint8_t *ring, *lbuf;
  float *bias;
  int32_t *ray;
  float *t0, *t1;
  uint16_t *list;
  uint32_t *wsum;
  TileInfo *info;
  uint64_t *full, *empty, *wfull, *ready, *accf, *acce, *layer, *lwfull, *fin;
  uint32_t *tmem;
  int32_t *misc;
  volatile int *abort_flag;
  float *res;
  uint32_t ring_stride, slot_w;
};

template <int F, int W>
__device__ __forceinline__ Smem16s carve16s(const Fused16sArgs &a, uint8_t *base) {
  const Layout16s l = make_layout16s(F, W, a.list_chunks, a.max_bias);
  Smem16s S;
  S.ring = base + l.ring;
  S.lbuf = base + l.lbuf;
  S.bias = reinterpret_cast<float *>(base + l.bias);
  S.ray = reinterpret_cast<int32_t *>(base + l.ray);
  S.t0 = reinterpret_cast<float *>(base + l.t0);
  S.t1 = reinterpret_cast<float *>(base + l.t1);
  S.list = reinterpret_cast<uint16_t *>(base + l.list);
  S.wsum = reinterpret_cast<uint32_t *>(base + l.wsum);
  S.info = reinterpret_cast<TileInfo *>(base + l.info);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + l.bars);
  S.full = bars;
  S.empty = bars + kNBuf16s;
  S.wfull = bars + 2 * kNBuf16s;
  S.ready = bars + 3 * kNBuf16s;
  S.accf = S.ready + 2;
  S.acce = S.ready + 4;
  S.layer = S.ready + 6;
  S.lwfull = S.ready + 7;
  S.fin = S.ready + 8;
  S.tmem = reinterpret_cast<uint32_t *>(base + l.tmem);
  S.misc = reinterpret_cast<int32_t *>(base + l.misc);
  S.abort_flag = reinterpret_cast<volatile int *>(S.misc + 4);
  S.res = reinterpret_cast<float *>(base + l.res);
  S.ring_stride = l.ring_stride;
  S.slot_w = l.slot_w;
  return S;
}

}  // namespace

// ---------------------------------------------------------------------------
// MMA warp: per chunk, stream the first-layer slice into the ring slot once
// the slot is free, wait for the gathered A tile and the slice, issue the
// chunk's MMAs.
// ---------------------------------------------------------------------------
template <int F, int W, int NG>
__device__ __noinline__ void mma16s_role(const Fused16sArgs *ap, uint8_t *base, uint32_t tmem) {
  const Fused16sArgs &a = *ap;
  const int lane = threadIdx.x & 31;
  const DevObject *objs = a.q.objs;
  const Smem16s S = carve16s<F, W>(a, base);
  int chunk_ctr = 0;
  const uint32_t idesc0 = idesc_h16(W);
  for (int i = 0;; ++i) {
    const int tb = i & 1;
    if (!mbar_wait(su32(&S.ready[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag)) break;
    const TileInfo ti = S.info[tb];
    if (ti.stop) break;
    const DevObject &ob = objs[ti.slot];
    const int CHK = 2 * ob.L * F;  // 16-bit columns per chunk
    const uint32_t sbo = (uint32_t)(CHK / 8) * 128u;
    const uint32_t slice = (uint32_t)W * CHK * 2u;
    if (i >= 2 && !mbar_wait(su32(&S.acce[tb]), (uint32_t)(((i - 2) >> 1) & 1), S.abort_flag)) break;
    tc_after();
    const uint32_t dacc = tmem + (uint32_t)(tb * W);
    bool ok = true;
    for (int s = 0; s < ti.kmax; ++s) {
      const int c = chunk_ctr + s;
      const int buf = c % kNBuf16s, use = c / kNBuf16s;
      uint8_t *slot = S.ring + buf * S.ring_stride;
      // the slot's previous MMAs must be done before its weights are replaced
      if (use > 0 && !mbar_wait(su32(&S.empty[buf]), (uint32_t)((use - 1) & 1), S.abort_flag)) {
        ok = false;
        break;
      }
      if (lane == 0) bulk_copy(su32(slot + S.slot_w), ob.w0_16c + (size_t)s * slice, slice, su32(&S.wfull[buf]));
      const bool got_a = mbar_wait(su32(&S.full[buf]), (uint32_t)(use & 1), S.abort_flag);
      // the copy is waited for even after an abort: it must land before the
      // shared memory is released
      const bool got_w = got_a ? mbar_wait(su32(&S.wfull[buf]), (uint32_t)(use & 1), S.abort_flag)
                               : mbar_wait_teardown(su32(&S.wfull[buf]), (uint32_t)(use & 1));
      if (!got_a || !got_w) {
        if (!got_w) *S.abort_flag = 1;
        ok = false;
        break;
      }
      tc_after();
      if (lane == 0) {
        const uint32_t a0 = su32(slot), b0 = su32(slot + S.slot_w);
        for (int ks = 0; ks < CHK / 16; ++ks) {
          const uint64_t ad = umma_desc(a0 + ks * 256, 128, sbo);
          const uint64_t bd = umma_desc(b0 + ks * 256, 128, sbo);
          mma_h16(dacc, ad, bd, idesc0, (s > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(su32(&S.empty[buf]));
      }
      __syncwarp();
    }
    if (!ok) break;
    chunk_ctr += ti.kmax;
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
// Epilogue warps: tile setup one tile ahead (rows, work lists, biases on an
// object change), then the later layers -- each layer's weights by bulk copy
// into the layer buffer, activations to TMEM, MMA -- and the decode.
// ---------------------------------------------------------------------------
template <int F, int W, int NG>
__device__ __noinline__ void epilogue16s_role(const Fused16sArgs *ap, uint8_t *base, uint32_t tmem) {
  const Fused16sArgs &a = *ap;
  constexpr int kEpiWarp0 = NG + 1;
  constexpr int kEpiThreads = kEpiWarps16s * 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  const Smem16s S = carve16s<F, W>(a, base);
  const int64_t n_tiles = (int64_t)q.s.meta[1];
  const int etid = tid - kEpiWarp0 * 32;
  const int ew = etid >> 5;
  const int quarter = warp & 3;
  const int r = quarter * 32 + lane;
  const uint32_t w_sbo = (uint32_t)(W / 8) * 128u;  // SBO of a K = W core-matrix tile
  int layer_ctr = 0;
  // layer-weight copies (thread etid 0 only): at most one in flight; its phase
  int lw_ctr = 0;
  uint32_t lw_phase = 0;
  bool lw_pending = false;
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
      const float *src = reinterpret_cast<const float *>(ob.umma_h + ob.umma_bias_off);
      const int nb = ob.n_hidden * W + ob.n_out_pad;
      for (int k = etid; k < nb; k += kEpiThreads) S.bias[k] = __ldg(src + k);
      if (etid < LSNIF_MAX_LEVELS) S.res[etid] = (float)ob.res[etid];
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
        if (v & (1023u << 10)) {  // entry point shared with the previous exit
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
    // set up tile i+1 now, unless it needs other biases: then after the
    // layers of tile i, which still read the current ones
    const int tn = fetch();
    const bool last = (int64_t)tn >= n_tiles;
    const bool deferred = !last && slot_of_tile(tn) != su_slot;
    if (!deferred) setup(i + 1, tn);
    if (last) stop_at = i + 1;

    if (etid == 0) S.misc[2] = mbar_wait(su32(&S.accf[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag) ? 0 : 1;
    named_sync(2, kEpiThreads);
    if (!S.misc[2]) {
      tc_after();
      const TileInfo ti = S.info[tb];
      const DevObject &ob = objs[ti.slot];
      const int n_hidden = ob.n_hidden, n_out = ob.n_out, n_out_pad = ob.n_out_pad, n_mat = ob.n_mat,
                act = ob.act;
      const uint8_t *wsrc = ob.umma_h + (size_t)W * ob.n_in * 2;  // the later layers' FP16 weights
      const uint32_t dacc = tmem + (uint32_t)(tb * W);
      const uint32_t trow = dacc + ((uint32_t)(quarter * 32) << 16);
      const uint32_t act_col = tmem + (uint32_t)(2 * W);  // activation tile, lane 0
      const uint32_t tact = act_col + ((uint32_t)(quarter * 32) << 16);
      for (int layer = 0; layer <= n_hidden; ++layer) {
        const bool out_layer = layer == n_hidden;
        const float *bl = S.bias + layer * W;
        if (!out_layer) {
          const int N = (layer + 1 < n_hidden) ? W : n_out_pad;
          const uint32_t wbytes = (uint32_t)N * W * 2u;
          // the next layer's weights: the buffer's last reader (the previous
          // layer's MMAs) has completed
          if (etid == 0 && !lw_pending && !*S.abort_flag) {
            bulk_copy(su32(S.lbuf), wsrc, wbytes, su32(S.lwfull));
            lw_pending = true;
            lw_phase = (uint32_t)(lw_ctr++ & 1);
          }
          wsrc += wbytes;
#pragma unroll
          for (int c0 = 0; c0 < W; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
            uint32_t hw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
              hw[u] = h2_sat(act_fn(__uint_as_float(v[2 * u]) + bl[c0 + 2 * u], act),
                             act_fn(__uint_as_float(v[2 * u + 1]) + bl[c0 + 2 * u + 1], act));
            TMEM_ST8(tact + (uint32_t)(c0 / 2), hw);
          }
          tmem_wait_st();
          tc_before();
          named_sync(2, kEpiThreads);
          if (etid == 0) {
            tc_after();
            if (lw_pending && mbar_wait(su32(S.lwfull), lw_phase, S.abort_flag)) {
              lw_pending = false;
              const uint32_t b0 = su32(S.lbuf);
              const uint32_t idesc = idesc_h16(N);
              for (int ks = 0; ks < W / 16; ++ks)
                mma_h16_ts(dacc, act_col + (uint32_t)(ks * 8), umma_desc(b0 + ks * 256, 128, w_sbo), idesc,
                           ks > 0 ? 1u : 0u);
              mma_commit(su32(S.layer));
              mbar_wait(su32(S.layer), (uint32_t)(layer_ctr & 1), S.abort_flag);
            }
          }
          ++layer_ctr;
          named_sync(2, kEpiThreads);
          tc_after();
        } else {
          // logits 16 columns at a time into a per-thread array, then decode
          float z[64];
#pragma unroll 1
          for (int c0 = 0; c0 < n_out_pad; c0 += 16) {
            uint32_t v[16];
            TMEM_LD16(trow + c0, (&v[0]));
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) z[c0 + u] = __uint_as_float(v[u]) + bl[c0 + u];
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
      named_sync(2, kEpiThreads);  // every thread is done with the old biases
      setup(i + 1, tn);
    }
  }
  if (etid == 0) {
    // a layer-weight copy still in flight (after an abort) lands before the
    // shared memory is released
    if (lw_pending && !mbar_wait_teardown(su32(S.lwfull), lw_phase)) *S.abort_flag = 1;
    mma_commit(su32(&S.fin[1]));
    if (!mbar_wait_teardown(su32(&S.fin[1]), 0u)) *S.abort_flag = 1;
  }
}

// ---------------------------------------------------------------------------
// the kernel: setup, gather warps inline, the other roles as functions
// ---------------------------------------------------------------------------
template <int F, int W, int NG, int NL>
__global__ void __launch_bounds__((NG + 1 + kEpiWarps16s) * 32, 1)
    fused16s_kernel(const __grid_constant__ Fused16sArgs a) {
  constexpr int kGatherThreads = NG * 32;
  constexpr int kMmaWarp = NG;
  constexpr int kTmemCols = tmem_cols16s(W);
  constexpr int LPG = 8 / F;  // levels per 16-byte column group
  static_assert(LPG % NL == 0, "levels per load batch must divide the group");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem16s S = carve16s<F, W>(a, base);

  if (tid == 0) {
    for (int b = 0; b < kNBuf16s; ++b) {
      mbar_init(su32(&S.full[b]), kGatherThreads);
      mbar_init(su32(&S.empty[b]), 1);
      mbar_init(su32(&S.wfull[b]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&S.ready[b]), 1);
      mbar_init(su32(&S.accf[b]), 1);
      mbar_init(su32(&S.acce[b]), kEpiWarps16s * 32);
      mbar_init(su32(&S.fin[b]), 1);
    }
    mbar_init(su32(S.layer), 1);
    mbar_init(su32(S.lwfull), 1);
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
    int chunk_ctr = 0;
    int rot_g = 0, rot_o = 0;
    for (int i = 0;; ++i) {
      const int tb = i & 1;
      if (!mbar_wait(su32(&S.ready[tb]), (uint32_t)((i >> 1) & 1), S.abort_flag)) break;
      const TileInfo ti = S.info[tb];
      if (ti.stop) break;
      const int kmax = ti.kmax;
      if (ti.slot != cur_slot) {
        const DevObject &ob = objs[ti.slot];
        L = ob.L;
        mask = ob.mask;
        tab = ob.tab16;
        cur_slot = ti.slot;
      }
      const uint16_t *s_lst = S.list + (size_t)tb * a.list_chunks * kListStride;
      const uint32_t *s_ws = S.wsum + (size_t)tb * a.list_chunks * 4;
      const int G = (L * F) / 8;  // 16-byte column groups per point
      const int CHK = 2 * L * F;  // 16-bit columns per chunk
      const uint32_t a_sbo = (uint32_t)(CHK / 8) * 128u;
      const size_t lstride = (size_t)(mask + 1) * F;
      for (int s = 0; s < kmax; ++s) {
        const int c = chunk_ctr + s;
        const int buf = c % kNBuf16s, use = c / kNBuf16s;
        uint8_t *A = S.ring + buf * S.ring_stride;
        uint32_t all = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) all += s_ws[s * 4 + w];
        const int ngt = (int)(all & 1023u), nct = (int)((all >> 10) & 1023u);
        const int n_gi = ngt * G, n_oi = (kListStride - ngt) * G;
        const int nb_g = (n_gi + 31) >> 5, nb_o = (n_oi + 31) >> 5;
        const int first_g = (warp - rot_g + NG) % NG, first_o = (warp - rot_o + NG) % NG;
        // the slot is free once the MMAs of chunk c - 2 are done and the
        // copies of chunk c - 1 (which read it) are written
        if (use > 0) mbar_wait(su32(&S.empty[buf]), (uint32_t)((use - 1) & 1), S.abort_flag);
        {
          const int cp = c - kNBuf16s + 1;
          if (cp >= 0 && cp < c) mbar_wait(su32(&S.full[cp % kNBuf16s]), (uint32_t)((cp / kNBuf16s) & 1), S.abort_flag);
        }
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
            // FP32 interpolation of the FP16 entries, one FP16 rounding per feature
            uint32_t wv[4];
#pragma unroll
            for (int u0 = 0; u0 < LPG; u0 += NL) {
              const int l = g * LPG + u0;
              float f[NL][F];
              encode_levels_f16<F, NL>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride, lstride * 2,
                                       mask, p, S.res + l, f);
#pragma unroll
              for (int u = 0; u < NL; ++u)
#pragma unroll
                for (int cc = 0; cc < F; cc += 2) wv[((u0 + u) * F + cc) / 2] = h2_sat(f[u][cc], f[u][cc + 1]);
            }
            *reinterpret_cast<uint4 *>(A + core_off(r, j * G + g, a_sbo)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
          }
        }
        // copies (entry point = previous chunk's exit point) and zero fills
        const int n_o = kListStride - ngt;
        if (nct > 0 && first_o < nb_o) {  // copies read the previous chunk: it must be complete
          const int cq = c - 1;
          mbar_wait(su32(&S.full[cq % kNBuf16s]), (uint32_t)((cq / kNBuf16s) & 1), S.abort_flag);
        }
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
              const uint8_t *Ap = S.ring + ((c - 1) % kNBuf16s) * S.ring_stride;
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
      chunk_ctr += kmax;
    }
  } else if (warp == kMmaWarp) {
    mma16s_role<F, W, NG>(&a, base, tmem);
  } else {
    epilogue16s_role<F, W, NG>(&a, base, tmem);
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

bool fused16s_supported(const DevObject &h) {
  if (!(h.F == 2 || h.F == 4)) return false;
  if (!(h.width == 64 || h.width == 128)) return false;
  if ((h.L * h.F) % 8 != 0 || h.L > 16) return false;
  if (h.n_out_pad > 64 || h.n_out_pad > h.width) return false;
  return true;
}

static int max_bias16s(const DevObject &h) { return LSNIF_MAX_HIDDEN * h.width + 64; }

size_t fused16s_smem_bytes(const DevObject &h, int H_max) {
  return make_layout16s(h.F, h.width, std::max(H_max, h.H) / 2, max_bias16s(h)).total;
}

template <int F, int W, int NG, int NL>
static cudaError_t launch16s_shape(const Fused16sArgs &a, size_t smem, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(fused16s_kernel<F, W, NG, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = 1;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one persistent CTA per SM, but no more CTAs than the batch can have tiles
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (int64_t)a.q.s.max_tiles));
  fused16s_kernel<F, W, NG, NL><<<grid, (NG + 1 + kEpiWarps16s) * 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused16s(const QueryLaunch &q, const DevObject &h, int *launches) {
  if (!fused16s_supported(h)) return cudaErrorNotSupported;
  Fused16sArgs a{};
  a.q = q;
  a.list_chunks = std::max(q.H_max, h.H) / 2;
  a.max_bias = max_bias16s(h);
  const size_t smem = make_layout16s(h.F, h.width, a.list_chunks, a.max_bias).total;
  if (smem > 232448) return cudaErrorNotSupported;
  *launches += 1;
  if (h.F == 2 && h.width == 64) return launch16s_shape<2, 64, 11, 2>(a, smem, q.stream);
  if (h.F == 2 && h.width == 128) return launch16s_shape<2, 128, 11, 2>(a, smem, q.stream);
  if (h.F == 4 && h.width == 64) return launch16s_shape<4, 64, 11, 2>(a, smem, q.stream);
  if (h.F == 4 && h.width == 128) return launch16s_shape<4, 128, 11, 2>(a, smem, q.stream);
  return cudaErrorNotSupported;
}

}  // namespace lsnif
