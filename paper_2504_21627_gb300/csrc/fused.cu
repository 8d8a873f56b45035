// Fused half-precision tensor-core query kernel for sm_103a: hash-grid
// gather -> every MLP layer on tcgen05 (TMEM accumulators) -> decode, one
// persistent CTA per SM. The paper fuses all layers of its FP16 network into
// one kernel on its own hardware (Sec. 5); here the gather is fused in as
// well, so the concatenated input vector (Sec. 3.2) never leaves shared
// memory. The network's operands are BF16 or, in the H16 instantiations,
// FP16 (kind::f16 takes either, A and B always of the same type); FP32
// accumulation in both.
//
// Work unit: a tile of 128 rays (the tcgen05 M). The first layer's K runs
// over the tile's occupied-voxel segments: chunk s holds the features of
// points 2s and 2s+1 (2*L*F 16-bit columns, no-swizzle K-major core-matrix
// layout). Chunks no ray of the tile reaches are skipped (tiles are sorted
// by point count).
//
// Warp roles:
//   gather warps (NG): build the tile's work lists, then fill chunk after
//     chunk into a ring of shared-memory A tiles;
//   one MMA warp: issues each filled chunk's MMAs against the resident
//     first-layer weights into the tile's TMEM accumulator;
//   four epilogue warps (TMEM lane = ray): hidden and output layers (bias,
//     activation, 16-bit activations back to shared memory, next MMA) and the
//     decode, while the gather warps fill the next tile. Two TMEM
//     accumulators alternate between tiles.
//
// Shared boundary points: consecutive occupied voxels along a ray share a
// face, and the traversal marks an entry point that is bit-identical to the
// previous segment's exit (bit s of the ray's dup mask). Such a point is
// gathered once: its chunk copies the features from the previous chunk's A
// tile. A chunk's work is thus a list of gathers, copies and zero fills (two
// entries per ray); gathers go round-robin over the gather warps in blocks
// of 32 items (item = one point x one 16-byte column group), so every warp
// gets the same share whatever the mix.
//
// Every mbarrier wait is bounded by a clock limit; on expiry the kernel flags
// an abort, every role stops, the device error word is set, in-flight MMAs
// are waited for (again bounded), TMEM is freed and the kernel returns.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "device.cuh"
#include "encode.cuh"
#include "tc_common.cuh"

namespace lsnif {

namespace {

constexpr int kNBufMax = 4;
constexpr int kEpiWarps = 4;

// kind::f16 instruction descriptor: A and B both BF16 (fp16 = 0) or both
// FP16 (fp16 = 1), K-major, FP32 D, M = 128.
__device__ __forceinline__ uint32_t idesc_f16(int N, int fp16) {
  const uint32_t ab = fp16 ? 0u : (1u << 7) | (1u << 10);
  return (1u << 4) | ab | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// The same with the A operand read from tensor memory (a_tmem: lane 0 and
// the first column of a 128-lane x K/2-column tile, row i in lane i, two
// 16-bit values per column).
__device__ __forceinline__ void mma_f16_ts(uint32_t tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// TMEM columns a CTA allocates: two W-column accumulators and a W-column
// activation tile (W/2 columns of hi words, W/2 of lo words), rounded up to
// the power of two the allocator takes
__host__ __device__ constexpr int tmem_cols(int W) { return 3 * W <= 256 ? 256 : 512; }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

// FP16 operands saturate at the largest finite half (65504) instead of
// overflowing to infinity; rounding to nearest even below that.
__device__ __forceinline__ uint32_t pack_h2_sat(float a, float b) {
  a = fminf(fmaxf(a, -65504.f), 65504.f);
  b = fminf(fmaxf(b, -65504.f), 65504.f);
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_op(float a, float b, int fp16) {
  return fp16 ? pack_h2_sat(a, b) : pack_bf16(a, b);
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }

// Two FP16 features (one half2 word) rounded to BF16 through their exact
// FP32 values.
__device__ __forceinline__ uint32_t h2_bits_to_bf16(uint32_t w) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
  return pack_bf16(f.x, f.y);
}

struct FusedArgs {
  QueryLaunch q;
  // X-rows mode (lsnif_mlp): X n x n_in FP32 in, Z n x n_out FP32 out
  const float *X;
  float *Z;
  int64_t xrows;
  uint32_t smem_blob;  // bytes of the weight blob
  uint32_t smem_lo;    // bytes of the BF16 residual weights of the later layers (0 with FP16 operands)
  int nbuf;            // ring buffers (2..kNBufMax)
  int list_chunks;     // work-list capacity in chunks (H_max / 2)
  int fp16;            // operand type: 0 BF16 (weights from umma), 1 FP16 (weights from umma_h);
                       // selects the kernel instantiation
};

// Shared-memory layout (byte offsets from a 1024-aligned base), the same on
// host (sizing) and device (carving).
struct Layout {
  uint32_t blob, blob_lo, ring, ring_stride, ray, t0, t1, list, wsum, info, bars, tmem, misc, res, total;
};

// mbarriers: full[kNBufMax], empty[kNBufMax], tile_ready[2], acc_full[2],
// acc_empty[2], layer_done, fin[2]
constexpr int kNumBars = 2 * kNBufMax + 2 + 2 + 2 + 1 + 2;

// lo_bytes > 0 (BF16 operands): the later layers' residual weights, the lo
// terms of their two-term products.
__host__ __device__ inline Layout make_layout(uint32_t blob_bytes, uint32_t lo_bytes, int F, int W, int nbuf,
                                              int list_chunks) {
  Layout o{};
  uint32_t off = 0;
  o.ring_stride = (uint32_t)kTileM * (uint32_t)(2 * 16 * F) * 2u;  // one chunk for L <= 16
  o.blob = lay_take(off, blob_bytes, 1024);
  o.blob_lo = lay_take(off, lo_bytes, 1024);
  o.ring = lay_take(off, (uint32_t)nbuf * o.ring_stride, 1024);
  o.ray = lay_take(off, 2 * kTileM * 4, 16);
  o.t0 = lay_take(off, 2 * kTileM * 4, 16);
  o.t1 = lay_take(off, 2 * kTileM * 4, 16);
  o.list = lay_take(off, 2u * (uint32_t)list_chunks * kListStride * 2u, 16);  // two tiles
  o.wsum = lay_take(off, 2u * (uint32_t)list_chunks * 4u * 4u, 16);
  o.info = lay_take(off, 2 * sizeof(TileInfo), 16);
  o.bars = lay_take(off, 8 * kNumBars, 8);
  o.tmem = lay_take(off, 16, 16);
  o.misc = lay_take(off, 16 * 4, 16);
  o.res = lay_take(off, 4 * LSNIF_MAX_LEVELS, 16);
  o.total = off + 1024;  // slack for aligning the dynamic base
  return o;
}

}  // namespace

// The MMA warp's work (see epilogue_role for why it is a function).
template <int F, int W, bool XROWS, int NG, bool H16>
__device__ __noinline__ void mma_role(const FusedArgs *ap, uint8_t *base, uint32_t tmem) {
  const FusedArgs &a = *ap;
  const int lane = threadIdx.x & 31;
  const DevObject *objs = a.q.objs;
  const int nbuf = a.nbuf;
  const Layout lay = make_layout(a.smem_blob, a.smem_lo, F, W, nbuf, a.list_chunks);
  uint8_t *s_blob = base + lay.blob;
  uint8_t *s_ring = base + lay.ring;
  TileInfo *s_info = reinterpret_cast<TileInfo *>(base + lay.info);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
  uint64_t *b_full = bars, *b_empty = bars + kNBufMax, *b_ready = bars + 2 * kNBufMax;
  uint64_t *b_accf = b_ready + 2, *b_acce = b_ready + 4, *b_fin = b_ready + 7;
  int32_t *s_misc = reinterpret_cast<int32_t *>(base + lay.misc);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(s_misc + 4);
  const uint32_t ring_stride = lay.ring_stride;
  {
    // =================== MMA warp ===================
    int rbuf = 0, ruse = 0;  // ring slot and pass of the next chunk
    const uint32_t idesc0 = idesc_f16(W, H16);
    for (int i = 0;; ++i) {
      const int tb = i & 1;
      if (!mbar_wait_sleep(su32(&b_ready[tb]), (uint32_t)((i >> 1) & 1), abort_flag)) break;
      const TileInfo ti = s_info[tb];
      if (ti.stop) break;
      const DevObject &ob = objs[ti.slot];
      const int CHK = 2 * ob.L * F;
      const uint32_t a_sbo = (uint32_t)(CHK / 8) * 128u, w0_sbo = (uint32_t)(ob.n_in / 8) * 128u;
      if (i >= 2 && !mbar_wait_sleep(su32(&b_acce[tb]), (uint32_t)(((i - 2) >> 1) & 1), abort_flag)) break;
      tc_after();
      const uint32_t dacc = tmem + (uint32_t)(tb * W);
      bool ok = true;
      for (int s = 0; s < ti.kmax; ++s) {
        // ring position of the next chunk, kept as counters (no division by
        // the run-time ring size)
        const int buf = rbuf;
        const uint32_t phase = (uint32_t)(ruse & 1);
        if (++rbuf == nbuf) {
          rbuf = 0;
          ++ruse;
        }
        if (!mbar_wait_sleep(su32(&b_full[buf]), phase, abort_flag)) {
          ok = false;
          break;
        }
        tc_after();
        if (lane == 0) {
          const uint32_t a0 = su32(s_ring + buf * ring_stride), b0 = su32(s_blob);
          for (int ks = 0; ks < CHK / 16; ++ks) {
            const uint64_t ad = umma_desc(a0 + ks * 256, 128, a_sbo);
            const uint64_t bd = umma_desc(b0 + (uint32_t)((s * CHK) / 8 + 2 * ks) * 128u, 128, w0_sbo);
            mma_f16(dacc, ad, bd, idesc0, (s > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(su32(&b_empty[buf]));
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(su32(&b_accf[tb]));
      __syncwarp();
    }
    if (lane == 0) {
      mma_commit(su32(&b_fin[0]));
      if (!mbar_wait_teardown(su32(&b_fin[0]), 0u)) *abort_flag = 1;
    }
    __syncwarp();
    }
}

// The epilogue warps' work, compiled as its own function so that its
// registers do not add to the gather warps' allocation.
template <int F, int W, bool XROWS, int NG, bool H16>
__device__ __noinline__ void epilogue_role(const FusedArgs *ap, uint8_t *base, uint32_t tmem) {
  const FusedArgs &a = *ap;
  constexpr int fp16 = H16;
  constexpr int kEpiWarp0 = NG + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  const Layout lay = make_layout(a.smem_blob, a.smem_lo, F, W, a.nbuf, a.list_chunks);
  uint8_t *s_blob = base + lay.blob;
  uint8_t *s_blob_lo = base + lay.blob_lo;
  int32_t *s_ray = reinterpret_cast<int32_t *>(base + lay.ray);
  float *s_t0 = reinterpret_cast<float *>(base + lay.t0);
  float *s_t1 = reinterpret_cast<float *>(base + lay.t1);
  uint16_t *s_list = reinterpret_cast<uint16_t *>(base + lay.list);
  uint32_t *s_wsum = reinterpret_cast<uint32_t *>(base + lay.wsum);
  TileInfo *s_info = reinterpret_cast<TileInfo *>(base + lay.info);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
  uint64_t *b_ready = bars + 2 * kNBufMax;
  uint64_t *b_accf = b_ready + 2, *b_acce = b_ready + 4, *b_layer = b_ready + 6, *b_fin = b_ready + 7;
  int32_t *s_misc = reinterpret_cast<int32_t *>(base + lay.misc);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(s_misc + 4);
  float *s_res = reinterpret_cast<float *>(base + lay.res);
  const int64_t n_tiles = XROWS ? (a.xrows + kTileM - 1) / kTileM : (int64_t)q.s.meta[1];
  {
    // =================== epilogue warps ===================
    // Besides the layers after the first, these four warps set up every
    // tile (fetch, rows, work lists, weights on an object change) one tile
    // ahead, so the gather warps never stop between tiles.
    constexpr int kEpiThreads = kEpiWarps * 32;
    const int etid = tid - kEpiWarp0 * 32;  // 0..127: the row a setup thread handles
    const int ew = etid >> 5;
    const int quarter = warp & 3;           // the TMEM lane quarter this warp may access
    const int r = quarter * 32 + lane;      // the row (ray) of the layers
    const uint32_t act_sbo = (uint32_t)(W / 8) * 128u;
    int layer_ctr = 0;
    int su_slot = -1;  // object whose weights are in shared memory

    // next tile index (INT_MAX once aborted), uniform over the epilogue warps
    auto fetch = [&]() -> int {
      named_sync(2, kEpiThreads);
      if (etid == 0) s_misc[0] = *abort_flag ? INT_MAX : atomicAdd(q.s.meta + 3, 1);
      named_sync(2, kEpiThreads);
      return s_misc[0];
    };
    auto slot_of_tile = [&](int tile) -> int { return XROWS ? 0 : q.s.tiles[3 * tile + 0]; };
    // Set tile `tile` up as the j-th tile (slot j & 1). The slot's previous
    // tile (j - 2) is finished by every role; a weight reload is only asked
    // for once the previous tile's layers are done.
    auto setup = [&](int j, int tile) {
      const int sb = j & 1;
      if ((int64_t)tile >= n_tiles) {
        if (etid == 0) {
          s_info[sb].stop = 1;
          mbar_arrive(su32(&b_ready[sb]));
        }
        return;
      }
      int slot, start, cnt;
      if (XROWS) {
        slot = 0;
        start = tile * kTileM;
        cnt = (int)min((int64_t)kTileM, a.xrows - (int64_t)tile * kTileM);
      } else {
        slot = q.s.tiles[3 * tile + 0];
        start = q.s.tiles[3 * tile + 1];
        cnt = q.s.tiles[3 * tile + 2];
      }
      const DevObject &ob = objs[slot];
      if (slot != su_slot) {
        const uint4 *src = reinterpret_cast<const uint4 *>(H16 ? ob.umma_h : ob.umma);
        uint4 *dst = reinterpret_cast<uint4 *>(s_blob);
        const int nvec = (int)(ob.umma_bytes / 16);
        for (int k = etid; k < nvec; k += kEpiThreads) dst[k] = __ldg(src + k);
        if constexpr (!H16) {
          const uint4 *src_lo = reinterpret_cast<const uint4 *>(ob.umma_lo);
          uint4 *dst_lo = reinterpret_cast<uint4 *>(s_blob_lo);
          const int nlo = (int)(ob.umma_lo_bytes / 16);
          for (int k = etid; k < nlo; k += kEpiThreads) dst_lo[k] = __ldg(src_lo + k);
        }
        if (etid < LSNIF_MAX_LEVELS) s_res[etid] = (float)ob.res[etid];
        fence_async_smem();
        su_slot = slot;
      }
      if (etid == 0) s_misc[1] = 0;
      named_sync(2, kEpiThreads);
      // rows
      int my_kk = 0;
      uint32_t my_dm = 0u;
      {
        int ray = -1;
        float t0v = 0.f, t1v = 0.f;
        if (etid < cnt) {
          if (XROWS) {
            ray = start + etid;
            my_kk = ob.H / 2;
          } else {
            ray = q.s.order[start + etid];
            my_kk = q.s.k[ray];
            my_dm = q.s.dup[ray];
            const float2 tt = reinterpret_cast<const float2 *>(q.s.t01)[ray];
            t0v = tt.x;
            t1v = tt.y;
          }
        }
        s_ray[sb * kTileM + etid] = ray;
        s_t0[sb * kTileM + etid] = t0v;
        s_t1[sb * kTileM + etid] = t1v;
        const int wm = __reduce_max_sync(0xffffffffu, my_kk);
        if (lane == 0) atomicMax(&s_misc[1], wm);
      }
      named_sync(2, kEpiThreads);
      const int kmax = s_misc[1];
      // work lists: per chunk, [gathers | copies | zero fills]
      uint16_t *lst = s_list + (size_t)sb * a.list_chunks * kListStride;
      uint32_t *ws = s_wsum + (size_t)sb * a.list_chunks * 4;
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
        s_info[sb].kmax = kmax;
        s_info[sb].slot = slot;
        s_info[sb].stop = 0;
        mbar_arrive(su32(&b_ready[sb]));
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
      // set up tile i+1 now, unless it needs other weights: then after the
      // layers of tile i, which still read the current ones
      const int tn = fetch();
      const bool last = (int64_t)tn >= n_tiles;
      const bool deferred = !last && slot_of_tile(tn) != su_slot;
      if (!deferred) setup(i + 1, tn);
      if (last) stop_at = i + 1;

      // ---- layers after the first, decode ----
      if (etid == 0) s_misc[2] = mbar_wait_sleep(su32(&b_accf[tb]), (uint32_t)((i >> 1) & 1), abort_flag) ? 0 : 1;
      named_sync(2, kEpiThreads);
      if (!s_misc[2]) {
        tc_after();
        const TileInfo ti = s_info[tb];
        const DevObject &ob = objs[ti.slot];
        const int n_hidden = ob.n_hidden, n_out = ob.n_out, n_out_pad = ob.n_out_pad, n_mat = ob.n_mat,
                  act = ob.act;
        const float *bias = reinterpret_cast<const float *>(s_blob + ob.umma_bias_off);
        const uint32_t wl_off0 = (uint32_t)W * ob.n_in * 2u;  // byte offset of W1 in the blob
        uint32_t wl_off = wl_off0;
        const uint32_t dacc = tmem + (uint32_t)(tb * W);
        const uint32_t trow = dacc + ((uint32_t)(quarter * 32) << 16);
        const uint32_t act_col = tmem + (uint32_t)(2 * W);  // activation tile (A operand), lane 0
        const uint32_t tact = act_col + ((uint32_t)(quarter * 32) << 16), tact_lo = tact + (uint32_t)(W / 2);
        for (int layer = 0; layer <= n_hidden; ++layer) {
          const bool out_layer = layer == n_hidden;
          const float *bl = bias + layer * W;
          if (!out_layer) {
            const int N = (layer + 1 < n_hidden) ? W : n_out_pad;
            const uint32_t idesc = idesc_f16(N, fp16);
            // The activations go to tensor memory, row r in lane r, two 16-bit
            // values per 32-bit column (the A operand of tcgen05.mma read from
            // TMEM): hi at columns [2W, 2W + W/2), lo (two-term BF16) after it.
#pragma unroll
            for (int c0 = 0; c0 < W; c0 += 16) {
              uint32_t v[16];
              TMEM_LD16(trow + c0, (&v[0]));
              tmem_wait_ld();
              uint32_t hw[8];
              if constexpr (H16) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                  hw[u] = pack_op(act_fn(__uint_as_float(v[2 * u]) + bl[c0 + 2 * u], act),
                                  act_fn(__uint_as_float(v[2 * u + 1]) + bl[c0 + 2 * u + 1], act), fp16);
              } else {
                // two-term BF16: hi = BF16(h), lo = BF16(h - hi) (the difference is exact in FP32)
                uint32_t lw[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const float x0 = act_fn(__uint_as_float(v[2 * u]) + bl[c0 + 2 * u], act);
                  const float x1 = act_fn(__uint_as_float(v[2 * u + 1]) + bl[c0 + 2 * u + 1], act);
                  const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
                  const float2 hf = __bfloat1622float2(hb);
                  hw[u] = *reinterpret_cast<const uint32_t *>(&hb);
                  lw[u] = pack_bf16(x0 - hf.x, x1 - hf.y);
                }
                TMEM_ST8(tact_lo + (uint32_t)(c0 / 2), lw);
              }
              TMEM_ST8(tact + (uint32_t)(c0 / 2), hw);
            }
            tmem_wait_st();
            tc_before();
            named_sync(2, kEpiThreads);
            if (etid == 0) {
              tc_after();
              const uint32_t b0 = su32(s_blob) + wl_off, b0l = su32(s_blob_lo) + (wl_off - wl_off0);
              for (int ks = 0; ks < W / 16; ++ks) {
                const uint64_t bd = umma_desc(b0 + ks * 256, 128, act_sbo);
                mma_f16_ts(dacc, act_col + (uint32_t)(ks * 8), bd, idesc, ks > 0 ? 1u : 0u);
                if constexpr (!H16) {
                  // the lo terms: hi_a . lo_w + lo_a . hi_w (lo_a . lo_w is left out)
                  mma_f16_ts(dacc, act_col + (uint32_t)(ks * 8), umma_desc(b0l + ks * 256, 128, act_sbo), idesc, 1u);
                  mma_f16_ts(dacc, act_col + (uint32_t)(W / 2 + ks * 8), bd, idesc, 1u);
                }
              }
              mma_commit(su32(b_layer));
              mbar_wait_sleep(su32(b_layer), (uint32_t)(layer_ctr & 1), abort_flag);
            }
            ++layer_ctr;
            named_sync(2, kEpiThreads);
            tc_after();
            wl_off += (uint32_t)N * W * 2u;
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
            const int32_t ray = s_ray[tb * kTileM + r];
            if (ray >= 0 && !*abort_flag) {
              if (XROWS) {
                for (int j = 0; j < n_out; ++j) a.Z[(int64_t)ray * n_out + j] = z[j];
              } else {
                decode_store(q.hits, ray, z, n_out, n_mat, s_t0[tb * kTileM + r], s_t1[tb * kTileM + r],
                             q.rays.tmin[ray], q.rays.tmax[ray]);
              }
            }
          }
        }
      }
      tc_before();
      mbar_arrive(su32(&b_acce[tb]));
      if (deferred) {
        named_sync(2, kEpiThreads);  // every thread is done with the old weights
        setup(i + 1, tn);
      }
    }
    if (etid == 0) {
      mma_commit(su32(&b_fin[1]));
      if (!mbar_wait_teardown(su32(&b_fin[1]), 0u)) *abort_flag = 1;
    }
    }
}

// F: features per level; W: hidden width; XROWS: read the network input
// from global rows instead of gathering it; NG: gather warps; NLB: levels
// whose corner loads are in flight together per gather item; GS (F = 2):
// 0 = 16-byte corner groups, 1 = the same with the next level's loads in
// flight during interpolation, 2 = 8-byte corner pairs (fewer registers).
// H16: FP16 operands (else BF16) -- features, weights and hidden
// activations; a template parameter so that no loop branches on it.
template <int F, int W, bool XROWS, int NG, int NLB, int GS, bool H16>
__global__ void __launch_bounds__((NG + 1 + kEpiWarps) * 32, 1) fused_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int kGatherThreads = NG * 32;
  constexpr int kMmaWarp = NG;
  constexpr int kTmemCols = tmem_cols(W);  // two accumulators, the activation tile (hi and lo)
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const QueryLaunch &q = a.q;
  const DevObject *objs = q.objs;
  const int nbuf = a.nbuf;

  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Layout lay = make_layout(a.smem_blob, a.smem_lo, F, W, nbuf, a.list_chunks);
  uint8_t *s_ring = base + lay.ring;
  int32_t *s_ray = reinterpret_cast<int32_t *>(base + lay.ray);
  uint16_t *s_list = reinterpret_cast<uint16_t *>(base + lay.list);
  uint32_t *s_wsum = reinterpret_cast<uint32_t *>(base + lay.wsum);
  TileInfo *s_info = reinterpret_cast<TileInfo *>(base + lay.info);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
  uint64_t *b_full = bars, *b_empty = bars + kNBufMax, *b_ready = bars + 2 * kNBufMax;
  uint64_t *b_accf = b_ready + 2, *b_acce = b_ready + 4, *b_layer = b_ready + 6, *b_fin = b_ready + 7;
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + lay.tmem);
  int32_t *s_misc = reinterpret_cast<int32_t *>(base + lay.misc);  // [0] tile [1] kmax [2] epi stop [4] abort
  volatile int *abort_flag = reinterpret_cast<volatile int *>(s_misc + 4);
  float *s_res = reinterpret_cast<float *>(base + lay.res);
  const uint32_t ring_stride = lay.ring_stride;

  if (tid == 0) {
    for (int b = 0; b < nbuf; ++b) {
      mbar_init(su32(&b_full[b]), kGatherThreads);
      mbar_init(su32(&b_empty[b]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&b_ready[b]), 1);
      mbar_init(su32(&b_accf[b]), 1);
      mbar_init(su32(&b_acce[b]), kEpiWarps * 32);
      mbar_init(su32(&b_fin[b]), 1);
    }
    mbar_init(su32(b_layer), 1);
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *s_tmem;
  const int Hs = q.H_max;

  if (warp < NG) {
    // =================== gather warps ===================
    int cur_slot = -1;
    int L = 0, n_in = 0;
    uint32_t mask = 0;
    const uint16_t *tab = nullptr;
    int rbuf = 0, ruse = 0;    // ring slot and pass of the next chunk
    int rot_g = 0, rot_o = 0;  // round-robin origin of the gather / other blocks
    for (int i = 0;; ++i) {
      const int tb = i & 1;
      // the epilogue warps set the tile up: rows, work lists, weights
      if (!mbar_wait_sleep(su32(&b_ready[tb]), (uint32_t)((i >> 1) & 1), abort_flag)) break;
      const TileInfo ti = s_info[tb];
      if (ti.stop) break;
      const int kmax = ti.kmax;
      if (ti.slot != cur_slot) {
        const DevObject &ob = objs[ti.slot];
        L = ob.L;
        n_in = ob.n_in;
        mask = ob.mask;
        tab = ob.tab16;
        cur_slot = ti.slot;
      }
      const uint16_t *s_lst = s_list + (size_t)tb * a.list_chunks * kListStride;
      const uint32_t *s_ws = s_wsum + (size_t)tb * a.list_chunks * 4;

      // ---- chunks ----
      const int G = (L * F) / 8;  // 16-byte column groups per point
      const int CHK = 2 * L * F;  // columns per chunk
      const uint32_t a_sbo = (uint32_t)(CHK / 8) * 128u;
      const size_t lstride = (size_t)(mask + 1) * F;
      // The boundary point of a thread's next gather item is loaded while
      // the current item's corner loads are in flight (across the chunks of
      // a tile too), so that the point's memory latency is not added to
      // every item's. pn_chunk: the chunk whose first item pn already holds.
      // Only for the 8-byte pair gather at 512 threads (128 registers): the
      // other variants have no registers to spare for it (it made them
      // spill and run slower).
      constexpr bool kPrefetch = !XROWS && GS == 2 && NG + 1 + kEpiWarps <= 16;
      float3 pn = make_float3(0.f, 0.f, 0.f);
      int pn_chunk = -1;
      auto load_point = [&](int s2, int it2, int ngt2, float inv2) {
        const int g2 = __float2int_rz(((float)it2 + 0.5f) * inv2);
        const int e2 = s_lst[s2 * kListStride + (it2 - g2 * ngt2)];
        const int ray2 = s_ray[tb * kTileM + (e2 & 127)];
        const float *P = q.s.pts + ((size_t)ray2 * Hs + 2 * s2 + (e2 >> 7)) * 3;
        return make_float3(P[0], P[1], P[2]);
      };
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
        uint8_t *A = s_ring + buf * ring_stride;
        uint32_t all = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) all += s_ws[s * 4 + w];
        const int ngt = (int)(all & 1023u), nct = (int)((all >> 10) & 1023u);
        const int n_gi = ngt * G, n_oi = (kListStride - ngt) * G;
        const int nb_g = (n_gi + 31) >> 5, nb_o = (n_oi + 31) >> 5;
        const int first_g = (warp - rot_g + NG) % NG, first_o = (warp - rot_o + NG) % NG;
        // The buffer is free once the MMAs of chunk c - nbuf are done and the
        // copies of chunk c - nbuf + 1 (which read it) are written. Every
        // thread waits, with or without items: an arrival on the full barrier
        // must not land in the phase of chunk c - nbuf.
        if (use > 0) mbar_wait_sleep(su32(&b_empty[buf]), (uint32_t)((use - 1) & 1), abort_flag);
        if (nbuf > 1 && nuse1 >= 0) mbar_wait_sleep(su32(&b_full[nbuf1]), (uint32_t)(nuse1 & 1), abort_flag);
        // gathers: the lanes of a warp take consecutive entries (neighbouring
        // rays) at the same column group, so at coarse levels they share
        // corners and cache sectors
        const float inv_g = 1.f / (float)max(ngt, 1);
        if (kPrefetch && pn_chunk != s && first_g < nb_g && first_g * 32 + lane < n_gi)
          pn = load_point(s, first_g * 32 + lane, ngt, inv_g);
        for (int b = first_g; b < nb_g; b += NG) {
          const int it = b * 32 + lane;
          float3 p = pn;
          if constexpr (kPrefetch) {
            const int bn = b + NG;
            if (bn < nb_g) {
              if (bn * 32 + lane < n_gi) pn = load_point(s, bn * 32 + lane, ngt, inv_g);
            } else if (s + 1 < kmax) {
              // this thread's first item of the next chunk
              uint32_t all2 = 0;
#pragma unroll
              for (int w = 0; w < 4; ++w) all2 += s_ws[(s + 1) * 4 + w];
              const int ngt2 = (int)(all2 & 1023u), n_gi2 = ngt2 * G;
              const int first2 = (warp - (rot_g + nb_g) % NG + NG) % NG;
              if (first2 * 32 + lane < n_gi2) {
                pn = load_point(s + 1, first2 * 32 + lane, ngt2, 1.f / (float)max(ngt2, 1));
                pn_chunk = s + 1;
              }
            }
          }
          if (it < n_gi) {
            const int g = __float2int_rz(((float)it + 0.5f) * inv_g);
            const int t = it - g * ngt;
            const int e = s_lst[s * kListStride + t];
            const int r = e & 127, j = e >> 7;
            uint4 outv;
            if (XROWS) {
              const int ray = s_ray[tb * kTileM + r];
              const float *xr = a.X + (int64_t)ray * n_in + (size_t)(2 * s + j) * L * F + g * 8;
              const float4 x0 = *reinterpret_cast<const float4 *>(xr);
              const float4 x1 = *reinterpret_cast<const float4 *>(xr + 4);
              outv = make_uint4(pack_op(x0.x, x0.y, H16), pack_op(x0.z, x0.w, H16), pack_op(x1.x, x1.y, H16),
                                pack_op(x1.z, x1.w, H16));
            } else {
              if constexpr (!kPrefetch) p = load_point(s, it, ngt, inv_g);
              constexpr int LPG = 8 / F;  // levels per 16-byte group
              // the group's 8 features as operand words: F = 2 gathers give
              // one half2 per level, F = 4 gathers FP32 values
              uint32_t ow[4];
              if constexpr (F == 2 && GS == 1) {
                // all LPG levels of the group, the next level's loads in flight
                __half2 h[LPG];
                encode_levels_h2_pipelined<LPG>(reinterpret_cast<const __half *>(tab) + (size_t)(g * LPG) * lstride,
                                                lstride * 2, mask, p, s_res + g * LPG, h);
#pragma unroll
                for (int u = 0; u < LPG; ++u) ow[u] = h2_bits(h[u]);
              } else
#pragma unroll
              for (int u0 = 0; u0 < LPG; u0 += NLB) {
                const int l = g * LPG + u0;
                if constexpr (F == 2) {
                  __half2 h[NLB];
                  if constexpr (GS == 2)
                    encode_levels_h2_pairs<NLB>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride,
                                                lstride * 2, mask, p, s_res + l, h);
                  else
                    encode_levels_h2<NLB>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride, lstride * 2,
                                          mask, p, s_res + l, h);
#pragma unroll
                  for (int u = 0; u < NLB; ++u) ow[u0 + u] = h2_bits(h[u]);
                } else {
                  float f[NLB][F];
                  encode_levels_f16<F, NLB>(reinterpret_cast<const __half *>(tab) + (size_t)l * lstride,
                                            lstride * 2, mask, p, s_res + l, f);
#pragma unroll
                  for (int u = 0; u < NLB; ++u)
#pragma unroll
                    for (int cc = 0; cc < F; cc += 2) ow[((u0 + u) * F + cc) / 2] = pack_op(f[u][cc], f[u][cc + 1], H16);
                }
              }
              if constexpr (F == 2 && !H16) {
#pragma unroll
                for (int k = 0; k < 4; ++k) ow[k] = h2_bits_to_bf16(ow[k]);
              }
              outv = make_uint4(ow[0], ow[1], ow[2], ow[3]);
            }
            *reinterpret_cast<uint4 *>(A + core_off(r, j * G + g, a_sbo)) = outv;
          }
        }
        // copies (entry point = previous chunk's exit point) and zero fills
        const int n_o = kListStride - ngt;
        if (nct > 0 && first_o < nb_o)  // copies read the previous chunk: it must be complete
          mbar_wait_sleep(su32(&b_full[pbuf]), (uint32_t)(puse & 1), abort_flag);
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
              const uint8_t *Ap = s_ring + pbuf * ring_stride;
              outv = *reinterpret_cast<const uint4 *>(Ap + core_off(r, G + g, a_sbo));
            }
            *reinterpret_cast<uint4 *>(A + core_off(r, j * G + g, a_sbo)) = outv;
          }
        }
        rot_g = (rot_g + nb_g) % NG;
        rot_o = (rot_o + nb_o) % NG;
        fence_async_smem();
        mbar_arrive(su32(&b_full[buf]));
      }
    }
  } else if (warp == kMmaWarp) {
    mma_role<F, W, XROWS, NG, H16>(&a, base, tmem);
  } else {
    epilogue_role<F, W, XROWS, NG, H16>(&a, base, tmem);
  }

  tc_before();
  __syncthreads();
  tc_after();
  if (tid == 0 && *abort_flag) atomicOr(q.err, kErrWaitTimeout);
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

static uint32_t blob_bytes(const DevObject &h) { return (h.umma_bytes + 15u) & ~15u; }
static uint32_t lo_bytes(const DevObject &h, bool fp16) { return fp16 ? 0u : (h.umma_lo_bytes + 15u) & ~15u; }

// with the smallest ring (2 buffers); launches use up to kNBufMax that fit
size_t fused_smem_bytes(const DevObject &h, int H_max, bool fp16) {
  return make_layout(blob_bytes(h), lo_bytes(h, fp16), h.F, h.width, 2, std::max(H_max, h.H) / 2).total;
}

// Shared memory and L1 share one array per SM. A CTA that needs more than
// the 196 KiB configuration (less the 1 KiB the system keeps per CTA) gets
// the 228 KiB one, which leaves L1 28 KiB instead of 60 KiB; the gather's
// coarse levels live in L1, and on the torus workload that alone took the
// fused kernel from 2.79 to 3.93 ms. A ring of 3 buffers ran as fast as 4,
// one of 2 about 13% slower; the FP16 kernel (no lo weights) with 3 buffers
// fits the 164 KiB configuration, whose 92 KiB of L1 made it 3% faster than
// with 4. So: 3 buffers when they stay within the 196 KiB configuration,
// else the largest ring that fits at all.
constexpr uint32_t kSmemL1Friendly = 195u * 1024u;

static int pick_nbuf(const DevObject &h, int list_chunks, bool fp16) {
  auto total = [&](int nb) { return make_layout(blob_bytes(h), lo_bytes(h, fp16), h.F, h.width, nb, list_chunks).total; };
  if (total(3) <= kSmemL1Friendly) return 3;
  for (int nb = kNBufMax; nb >= 2; --nb)
    if (total(nb) <= 232448) return nb;
  return 0;
}

template <int F, int W, bool XR, int NG, int NLB, int GS, bool H16>
static cudaError_t launch_op(const FusedArgs &a, size_t smem, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<F, W, XR, NG, NLB, GS, H16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    attr = 1;
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one persistent CTA per SM, but no more CTAs than the batch can have
  // tiles: a small request leaves the other SMs to concurrent work
  const int64_t tiles = XR ? (a.xrows + kTileM - 1) / kTileM : (int64_t)a.q.s.max_tiles;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, tiles));
  fused_kernel<F, W, XR, NG, NLB, GS, H16><<<grid, (NG + 1 + kEpiWarps) * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int F, int W, bool XR, int NG, int NLB, int GS>
static cudaError_t launch_one(const FusedArgs &a, size_t smem, cudaStream_t st) {
  return a.fp16 ? launch_op<F, W, XR, NG, NLB, GS, true>(a, smem, st)
                : launch_op<F, W, XR, NG, NLB, GS, false>(a, smem, st);
}

// Shapes the autotuner chooses between: gather warps per CTA (with the MMA
// warp and 4 epilogue warps: 4, 5 or 6 warps per SM sub-partition, so at
// most 128, 96 or 80 registers per thread), levels of corner loads in flight
// per gather item, and the F = 2 gather style. On the torus benchmark the
// first (fewer warps, all four levels of a column group in flight, 8-byte
// corner pairs) is fastest: latency is hidden by loads per thread rather
// than by more warps.
struct Variant {
  int gather_warps, levels, style;
};
static const Variant kVariants[] = {{11, 4, 2}, {11, 2, 1}, {15, 1, 2}, {19, 1, 2}, {15, 4, 2}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

template <int F, int W, bool XR>
static cudaError_t dispatch_variant(const FusedArgs &a, int v, size_t smem, cudaStream_t st) {
  constexpr int LPG = 8 / F;
  constexpr int NL2 = 2 < LPG ? 2 : LPG;
  constexpr int PAIRS = F == 2 ? 2 : 0;
  // rows given as input (lsnif_mlp) gather nothing: one shape serves them
  if constexpr (XR) {
    return v == 1 ? launch_one<F, W, XR, 11, NL2, F == 2 ? 1 : 0>(a, smem, st) : cudaErrorInvalidValue;
  } else {
    switch (v) {
      case 0: return launch_one<F, W, XR, 11, LPG, PAIRS>(a, smem, st);
      case 1: return launch_one<F, W, XR, 11, NL2, F == 2 ? 1 : 0>(a, smem, st);
      case 2: return launch_one<F, W, XR, 15, 1, PAIRS>(a, smem, st);
      case 3: return launch_one<F, W, XR, 19, 1, PAIRS>(a, smem, st);
      case 4: return launch_one<F, W, XR, 15, LPG, PAIRS>(a, smem, st);
      default: return cudaErrorInvalidValue;
    }
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
  *threads = kVariants[v].gather_warps * 32;
  *levels = kVariants[v].levels;
}

cudaError_t launch_fused(const QueryLaunch &q, const DevObject &h, int variant, bool fp16, int *launches) {
  if (!fused_supported(h)) return cudaErrorNotSupported;
  if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.q = q;
  a.fp16 = fp16 ? 1 : 0;
  a.smem_blob = blob_bytes(h);
  a.smem_lo = lo_bytes(h, fp16);
  a.list_chunks = std::max(q.H_max, h.H) / 2;
  a.nbuf = pick_nbuf(h, a.list_chunks, fp16);
  if (!a.nbuf) return cudaErrorNotSupported;
  const size_t smem = make_layout(a.smem_blob, a.smem_lo, h.F, h.width, a.nbuf, a.list_chunks).total;
  *launches += 1;
  return dispatch<false>(a, h, variant, smem, q.stream);
}

cudaError_t launch_mlp_fused(const DevObject *dobj, const DevObject &h, const float *X, int64_t n, float *Z,
                             bool fp16, int *err, cudaStream_t st) {
  if (!fused_supported(h)) return cudaErrorNotSupported;
  FusedArgs a{};
  a.fp16 = fp16 ? 1 : 0;
  a.smem_blob = blob_bytes(h);
  a.smem_lo = lo_bytes(h, fp16);
  a.list_chunks = h.H / 2;
  a.nbuf = pick_nbuf(h, a.list_chunks, fp16);
  if (!a.nbuf) return cudaErrorNotSupported;
  const size_t smem = make_layout(a.smem_blob, a.smem_lo, h.F, h.width, a.nbuf, a.list_chunks).total;
  int32_t *meta = nullptr;
  cudaError_t e = cudaMallocAsync(&meta, 16 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(meta, 0, 16 * sizeof(int32_t), st);
  a.q.objs = dobj;
  a.q.n_slots = 1;
  a.q.H_max = h.H;
  a.q.err = err;
  a.q.s.meta = meta;
  a.X = X;
  a.Z = Z;
  a.xrows = n;
  e = dispatch<true>(a, h, 1, smem, st);
  cudaFreeAsync(meta, st);
  return e;
}

}  // namespace lsnif
