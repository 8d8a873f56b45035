// Hash-grid corner gather and trilinear interpolation of one point at one
// level (Sec. 3.2), for FP32 or FP16 tables of F features per entry.
//
// The gather is bound by the number of L2 requests, not bytes: the two
// x-neighbours of a corner pair hash to indices that differ only in their
// low bits (the x multiplier is 1), so both usually fall in the same aligned
// 16-byte group of entries and one 16-byte load serves the pair.
#pragma once

#include "device.cuh"

namespace lsnif {

struct Cell {
  uint32_t cx, cy, cz;
  float wx, wy, wz;
};

// Lattice cell of a unit-cube point at resolution N (vertices 0..N, no
// offset): c = floor(p * N), w = p * N - c, from the EXACT product. The FP32
// product x = fl(p * N) is split with an FMA into x + e == p * N exactly
// (the error-free product of Ogita, Rump and Oishi, "Accurate Sum and Dot
// Product", 2005), so the cell is the floor of the exact value: for a
// non-integer x, |e| <= ulp(x)/2 cannot cross an integer; for an integer x
// the cell drops by one when e < 0. The weight keeps e. The decision thus
// equals the one an FP64 evaluation of p * N makes for the same FP32 p.
__device__ __forceinline__ void exact_cell(float p, float N, uint32_t &c, float &w) {
  const float x = p * N;
  const float e = fmaf(p, N, -x);
  float f = floorf(x);
  f -= (x == f && e < 0.f) ? 1.f : 0.f;
  c = (uint32_t)(int)f;
  w = (x - f) + e;
}

__device__ __forceinline__ Cell lattice_cell(const float3 &p, float N) {
  Cell c;
  exact_cell(p.x, N, c.cx, c.wx);
  exact_cell(p.y, N, c.cy, c.wy);
  exact_cell(p.z, N, c.cz, c.wz);
  return c;
}

template <typename T, int F>
struct Entry {
  static constexpr int kBytes = F * (int)sizeof(T);
  static constexpr int kGroup = 16 / kBytes;  // entries per 16-byte group
};

template <typename T, int F>
__device__ __forceinline__ void unpack_entry(const uint4 &g, uint32_t j, float (&v)[F]);

template <>
__device__ __forceinline__ void unpack_entry<float, 1>(const uint4 &g, uint32_t j, float (&v)[1]) {
  v[0] = __uint_as_float(pick4(g, j));
}
template <>
__device__ __forceinline__ void unpack_entry<float, 2>(const uint4 &g, uint32_t j, float (&v)[2]) {
  v[0] = __uint_as_float(j ? g.z : g.x);
  v[1] = __uint_as_float(j ? g.w : g.y);
}
template <>
__device__ __forceinline__ void unpack_entry<float, 4>(const uint4 &g, uint32_t, float (&v)[4]) {
  v[0] = __uint_as_float(g.x);
  v[1] = __uint_as_float(g.y);
  v[2] = __uint_as_float(g.z);
  v[3] = __uint_as_float(g.w);
}
template <>
__device__ __forceinline__ void unpack_entry<__half, 1>(const uint4 &g, uint32_t j, float (&v)[1]) {
  uint32_t w = pick4(g, j >> 1);
  v[0] = __half2float(__ushort_as_half((unsigned short)((j & 1) ? (w >> 16) : (w & 0xFFFFu))));
}
template <>
__device__ __forceinline__ void unpack_entry<__half, 2>(const uint4 &g, uint32_t j, float (&v)[2]) {
  uint32_t w = pick4(g, j);
  float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
  v[0] = f.x;
  v[1] = f.y;
}
template <>
__device__ __forceinline__ void unpack_entry<__half, 4>(const uint4 &g, uint32_t j, float (&v)[4]) {
  uint32_t w0 = j ? g.z : g.x, w1 = j ? g.w : g.y;
  float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&w0));
  float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&w1));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Load one entry on its own (bytes = F * sizeof(T)).
template <typename T, int F>
__device__ __forceinline__ void load_entry(const T *tab, uint32_t i, float (&v)[F]) {
  constexpr int B = Entry<T, F>::kBytes;
  const uint8_t *p = reinterpret_cast<const uint8_t *>(tab) + (size_t)i * B;
  uint4 g;
  if constexpr (B == 16) {
    g = ldg16(p);
    unpack_entry<T, F>(g, 0, v);
  } else if constexpr (B == 8) {
    uint2 u = ldg8(p);
    g = make_uint4(u.x, u.y, 0, 0);
    unpack_entry<T, F>(g, 0, v);
  } else if constexpr (B == 4) {
    g = make_uint4(ldg4(p), 0, 0, 0);
    unpack_entry<T, F>(g, 0, v);
  } else {  // 2 bytes
    uint32_t w = ldg4(reinterpret_cast<const uint8_t *>(tab) + (size_t)(i & ~1u) * 2);
    g = make_uint4(w, 0, 0, 0);
    unpack_entry<T, F>(g, i & 1u, v);
  }
}

// Entries i0 (always) and i1 (when need1): one 16-byte load when both sit
// in the same aligned group, otherwise a group load plus one entry load.
template <typename T, int F>
__device__ __forceinline__ void load_pair(const T *tab, uint32_t i0, uint32_t i1, bool need1, float (&v0)[F],
                                          float (&v1)[F]) {
  constexpr int G = Entry<T, F>::kGroup;
  constexpr int B = Entry<T, F>::kBytes;
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab);
  uint4 g = ldg16(base + (size_t)(i0 & ~(uint32_t)(G - 1)) * B);
  unpack_entry<T, F>(g, i0 & (G - 1), v0);
  if (need1) {
    if ((i0 ^ i1) < (uint32_t)G) unpack_entry<T, F>(g, i1 & (G - 1), v1);
    else load_entry<T, F>(tab, i1, v1);
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) v1[f] = 0.f;
  }
}

// Trilinear feature of point p at one level: sum over the 8 cell corners of
// prod_axis(d ? w : 1-w) * table[hash(c + d) & mask]. Corners whose weight is
// exactly zero (a coordinate on a lattice plane) are not fetched.
template <typename T, int F>
__device__ __forceinline__ void encode_level(const T *__restrict__ tab, uint32_t mask, const float3 &p, float N,
                                             float (&out)[F]) {
  Cell c = lattice_cell(p, N);
#pragma unroll
  for (int f = 0; f < F; ++f) out[f] = 0.f;
  const bool nx = c.wx != 0.f, ny = c.wy != 0.f, nz = c.wz != 0.f;
  const uint32_t hy0 = c.cy * kPi2, hy1 = (c.cy + 1u) * kPi2;
  const uint32_t hz0 = c.cz * kPi3, hz1 = (c.cz + 1u) * kPi3;
  float v0[4][F], v1[4][F];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const bool need = (dy == 0 || ny) && (dz == 0 || nz);
    const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
    const uint32_t i0 = (c.cx ^ b) & mask, i1 = ((c.cx + 1u) ^ b) & mask;
    if (need) {
      load_pair<T, F>(tab, i0, i1, nx, v0[q], v1[q]);
    } else {
#pragma unroll
      for (int f = 0; f < F; ++f) { v0[q][f] = 0.f; v1[q][f] = 0.f; }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const float wyz = (dy ? c.wy : 1.f - c.wy) * (dz ? c.wz : 1.f - c.wz);
#pragma unroll
    for (int f = 0; f < F; ++f) out[f] = fmaf(wyz, fmaf(c.wx, v1[q][f] - v0[q][f], v0[q][f]), out[f]);
  }
}

// ---------------------------------------------------------------------------
// Batched, branch-free gather of NL levels of one point (the fused kernel's
// hot loop). All corner addresses of the batch are formed first, then every
// load is issued as a predicated ld.global.nc (no branches between loads, so
// they are all in flight together), then the weights are applied. Pair
// loads: one 16-byte load of the aligned group holding corner x0; corner x1
// shares it when it falls in the same group, otherwise it is a second,
// predicated entry load. Zero-weight corners issue nothing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ldg16_if(const void *p, bool pred) {
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  asm("{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n@q ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%5];\n}\n"
      : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
      : "r"((int)pred), "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t ldg4_if(const void *p, bool pred) {
  uint32_t v = 0u;
  asm("{\n.reg .pred q;\nsetp.ne.b32 q, %1, 0;\n@q ld.global.nc.u32 %0, [%2];\n}\n" : "+r"(v) : "r"((int)pred), "l"(p));
  return v;
}

__device__ __forceinline__ uint2 ldg8_if(const void *p, bool pred) {
  uint2 v = make_uint2(0u, 0u);
  asm("{\n.reg .pred q;\nsetp.ne.b32 q, %2, 0;\n@q ld.global.nc.v2.u32 {%0,%1}, [%3];\n}\n"
      : "+r"(v.x), "+r"(v.y)
      : "r"((int)pred), "l"(p));
  return v;
}

// FP16 tables, F in {2, 4}: entries of 4 or 8 bytes.
template <int F, int NL>
__device__ __forceinline__ void encode_levels_f16(const __half *__restrict__ tab0, size_t level_stride, uint32_t mask,
                                                  const float3 &p, const float *Ns, float (&out)[NL][F]) {
  constexpr int EB = F * 2;        // entry bytes
  constexpr int G = 16 / EB;       // entries per 16-byte group
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab0);
  float wx[NL], wy[NL], wz[NL];
  uint32_t ia[NL][4], ib[NL][4];
  bool pa[NL][4], pb[NL][4];
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const Cell c = lattice_cell(p, Ns[u]);
    wx[u] = c.wx;
    wy[u] = c.wy;
    wz[u] = c.wz;
    const uint32_t hy0 = c.cy * kPi2, hy1 = (c.cy + 1u) * kPi2;
    const uint32_t hz0 = c.cz * kPi3, hz1 = (c.cz + 1u) * kPi3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
      ia[u][q] = (c.cx ^ b) & mask;
      ib[u][q] = ((c.cx + 1u) ^ b) & mask;
      pa[u][q] = (dy == 0 || c.wy != 0.f) && (dz == 0 || c.wz != 0.f);
      pb[u][q] = pa[u][q] && c.wx != 0.f && ((ia[u][q] ^ ib[u][q]) >= (uint32_t)G);
    }
  }
  uint4 ga[NL][4];
  uint32_t gb[NL][4][EB / 4];
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const uint8_t *tl = base + (size_t)u * level_stride;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ga[u][q] = ldg16_if(tl + (size_t)(ia[u][q] & ~(uint32_t)(G - 1)) * EB, pa[u][q]);
      if constexpr (EB == 4) {
        gb[u][q][0] = ldg4_if(tl + (size_t)ib[u][q] * EB, pb[u][q]);
      } else {
        const uint2 t = ldg8_if(tl + (size_t)ib[u][q] * EB, pb[u][q]);
        gb[u][q][0] = t.x;
        gb[u][q][1] = t.y;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NL; ++u) {
#pragma unroll
    for (int f = 0; f < F; ++f) out[u][f] = 0.f;
    if constexpr (F == 4) {
      // 8-byte entries, two per group. Which half of its group corner x0 of
      // row q takes is bit 0 of its index: that of row 0 flipped by dy and
      // by dz (the y and z multipliers are odd). Corner x1 shares the group
      // when cx ^ (cx + 1), masked, is below 2 -- the same for every row.
      // The words of each corner are selected first and converted once.
      static_assert((kPi2 & 1u) && (kPi3 & 1u), "the row parity needs odd y and z multipliers");
      const bool j0 = (ia[u][0] & 1u) != 0u;
      const bool same = (ia[u][0] ^ ib[u][0]) < (uint32_t)G;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int dy = q & 1, dz = q >> 1;
        const bool ja = (dy ^ dz) ? !j0 : j0;
        const uint32_t a0 = ja ? ga[u][q].z : ga[u][q].x, a1 = ja ? ga[u][q].w : ga[u][q].y;
        const uint32_t o0 = ja ? ga[u][q].x : ga[u][q].z, o1 = ja ? ga[u][q].y : ga[u][q].w;
        const uint32_t b0 = pb[u][q] ? gb[u][q][0] : (same ? o0 : a0);
        const uint32_t b1 = pb[u][q] ? gb[u][q][1] : (same ? o1 : a1);
        const float2 x00 = __half22float2(*reinterpret_cast<const __half2 *>(&a0));
        const float2 x01 = __half22float2(*reinterpret_cast<const __half2 *>(&a1));
        const float2 x10 = __half22float2(*reinterpret_cast<const __half2 *>(&b0));
        const float2 x11 = __half22float2(*reinterpret_cast<const __half2 *>(&b1));
        const float v0[4] = {x00.x, x00.y, x01.x, x01.y}, v1[4] = {x10.x, x10.y, x11.x, x11.y};
        const float wyz = (dy ? wy[u] : 1.f - wy[u]) * (dz ? wz[u] : 1.f - wz[u]);
#pragma unroll
        for (int f = 0; f < F; ++f) out[u][f] = fmaf(wyz, fmaf(wx[u], v1[f] - v0[f], v0[f]), out[u][f]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int dy = q & 1, dz = q >> 1;
        // all three sources of the x1 corner are formed, then selected
        float v0[F], vg[F], vb[F], v1[F];
        unpack_entry<__half, F>(ga[u][q], ia[u][q] & (G - 1), v0);
        unpack_entry<__half, F>(ga[u][q], ib[u][q] & (G - 1), vg);
        const uint4 t = make_uint4(gb[u][q][0], EB == 8 ? gb[u][q][EB / 4 - 1] : 0u, 0u, 0u);
        unpack_entry<__half, F>(t, 0, vb);
        const bool same = (ia[u][q] ^ ib[u][q]) < (uint32_t)G;
#pragma unroll
        for (int f = 0; f < F; ++f) v1[f] = pb[u][q] ? vb[f] : (same ? vg[f] : v0[f]);
        const float wyz = (dy ? wy[u] : 1.f - wy[u]) * (dz ? wz[u] : 1.f - wz[u]);
#pragma unroll
        for (int f = 0; f < F; ++f) out[u][f] = fmaf(wyz, fmaf(wx[u], v1[f] - v0[f], v0[f]), out[u][f]);
      }
    }
  }
}

// FP16 tables with F = 2 (one half2 word per entry), interpolated in half2
// arithmetic: corner words are selected from the loaded groups without
// unpacking, and each corner pair costs one HSUB2 and two HFMA2. The FP16
// accumulation error (about 2^-11 of the feature range) is far below the
// BF16 rounding the fused kernel applies to the result.
__device__ __forceinline__ uint32_t word4(const uint4 &g, uint32_t j) {
  const uint32_t lo = (j & 1u) ? g.y : g.x;
  const uint32_t hi = (j & 1u) ? g.w : g.z;
  return (j & 2u) ? hi : lo;
}

// Four predicated 4-byte loads sharing one predicate.
__device__ __forceinline__ void ldg4x4_if(uint32_t (&v)[4], const void *a0, const void *a1, const void *a2,
                                          const void *a3, bool pred) {
  asm("{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
      "@q ld.global.nc.u32 %0, [%5];\n@q ld.global.nc.u32 %1, [%6];\n"
      "@q ld.global.nc.u32 %2, [%7];\n@q ld.global.nc.u32 %3, [%8];\n}\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
      : "r"((int)pred), "l"(a0), "l"(a1), "l"(a2), "l"(a3));
}

// The four (y, z) rows of a level always load their 16-byte group of corner
// x0 (rows of zero weight too: their product is an exact zero, and skipping
// them saves too few requests to pay for the predicate logic). Corner x1
// lies in the same group unless cx = 3 mod 4 (the indices differ only in the
// bits of cx ^ (cx + 1), the same for all four rows); only then, and only
// when its weight wx is non-zero, it is a second 4-byte load. With wx = 0
// the x1 word is any word of the group: it enters with weight exactly 0
// (table values are finite FP16, so the difference v1 - v0 is finite for
// |v| < 32768).
template <int NL>
__device__ __forceinline__ void encode_levels_h2(const __half *__restrict__ tab0, size_t level_stride, uint32_t mask,
                                                 const float3 &p, const float *Ns, __half2 (&out)[NL]) {
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab0);
  float wx[NL], wy[NL], wz[NL];
  uint32_t ia[NL][4], ib[NL][4];
  bool far[NL];
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const Cell c = lattice_cell(p, Ns[u]);
    wx[u] = c.wx;
    wy[u] = c.wy;
    wz[u] = c.wz;
    const uint32_t hy0 = c.cy * kPi2, hy1 = hy0 + kPi2;
    const uint32_t hz0 = c.cz * kPi3, hz1 = hz0 + kPi3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
      ia[u][q] = (c.cx ^ b) & mask;
      ib[u][q] = ((c.cx + 1u) ^ b) & mask;
    }
    far[u] = ((ia[u][0] ^ ib[u][0]) >= 4u) && c.wx != 0.f;
  }
  uint4 ga[NL][4];
  uint32_t gb[NL][4];
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const uint8_t *tl = base + (size_t)u * level_stride;
#pragma unroll
    for (int q = 0; q < 4; ++q) ga[u][q] = __ldg(reinterpret_cast<const uint4 *>(tl + (size_t)(ia[u][q] & ~3u) * 4));
    ldg4x4_if(gb[u], tl + (size_t)ib[u][0] * 4, tl + (size_t)ib[u][1] * 4, tl + (size_t)ib[u][2] * 4,
              tl + (size_t)ib[u][3] * 4, far[u]);
  }
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const float w0y = 1.f - wy[u], w0z = 1.f - wz[u];
    const float wq[4] = {w0y * w0z, wy[u] * w0z, w0y * wz[u], wy[u] * wz[u]};
    const __half2 wx2 = __float2half2_rn(wx[u]);
    __half2 acc = __float2half2_rn(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t w0 = word4(ga[u][q], ia[u][q] & 3u);
      const uint32_t w1 = far[u] ? gb[u][q] : word4(ga[u][q], ib[u][q] & 3u);
      const __half2 v0 = *reinterpret_cast<const __half2 *>(&w0);
      const __half2 v1 = *reinterpret_cast<const __half2 *>(&w1);
      const __half2 lerp = __hfma2(wx2, __hsub2(v1, v0), v0);
      acc = __hfma2(__float2half2_rn(wq[q]), lerp, acc);
    }
    out[u] = acc;
  }
}

// Register-lean variant for F = 2: each row loads the aligned 8-byte pair
// holding corner x0; for even cx it also holds x1 (the indices differ in
// bit 0 only), for odd cx corner x1 is a second 4-byte load (skipped when
// wx = 0). 1.5 requests per row instead of 1.25, but 3 live registers per
// row instead of 5, which lets more warps share an SM.
template <int NL>
__device__ __forceinline__ void encode_levels_h2_pairs(const __half *__restrict__ tab0, size_t level_stride,
                                                       uint32_t mask, const float3 &p, const float *Ns,
                                                       __half2 (&out)[NL]) {
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab0);
  float wx[NL], wy[NL], wz[NL];
  // Corner x0 of row q is the odd word of its pair when bit 0 of its index
  // is set. The y and z multipliers are odd, so stepping y or z by one flips
  // bit 0 of the hash: bit 0 of row q's index is h0 ^ dy ^ dz, with h0 that
  // of row 0 (the table mask keeps bit 0).
  static_assert((kPi2 & 1u) && (kPi3 & 1u), "the row parity below needs odd y and z multipliers");
  bool h0[NL];
  bool odd[NL];
  uint2 ga[NL][4];
  uint32_t gb[NL][4];
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const Cell c = lattice_cell(p, Ns[u]);
    wx[u] = c.wx;
    wy[u] = c.wy;
    wz[u] = c.wz;
    const uint32_t hy0 = c.cy * kPi2, hy1 = hy0 + kPi2;
    const uint32_t hz0 = c.cz * kPi3, hz1 = hz0 + kPi3;
    const uint8_t *tl = base + (size_t)u * level_stride;
    odd[u] = (c.cx & 1u) && c.wx != 0.f;
    h0[u] = ((c.cx ^ hy0 ^ hz0) & 1u) != 0u;
    const void *pb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q & 1, dz = q >> 1;
      const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
      const uint32_t ia = (c.cx ^ b) & mask;
      const uint32_t ib = ((c.cx + 1u) ^ b) & mask;
      ga[u][q] = __ldg(reinterpret_cast<const uint2 *>(tl + (size_t)(ia & ~1u) * 4));
      pb[q] = tl + (size_t)ib * 4;
    }
    ldg4x4_if(gb[u], pb[0], pb[1], pb[2], pb[3], odd[u]);
  }
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    const float w0y = 1.f - wy[u], w0z = 1.f - wz[u];
    const float wq[4] = {w0y * w0z, wy[u] * w0z, w0y * wz[u], wy[u] * wz[u]};
    const __half2 wx2 = __float2half2_rn(wx[u]);
    // the four row weights rounded to FP16 two at a time, then broadcast
    const __half2 w01 = __floats2half2_rn(wq[0], wq[1]), w23 = __floats2half2_rn(wq[2], wq[3]);
    const __half2 wqh[4] = {__low2half2(w01), __high2half2(w01), __low2half2(w23), __high2half2(w23)};
    __half2 acc = __float2half2_rn(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool hi = (q == 0 || q == 3) ? h0[u] : !h0[u];
      const uint32_t w0 = hi ? ga[u][q].y : ga[u][q].x;
      // x1: the other word of the pair (even cx), its own load (odd cx), or,
      // with wx = 0, a word of weight exactly 0
      const uint32_t w1 = odd[u] ? gb[u][q] : (hi ? ga[u][q].x : ga[u][q].y);
      const __half2 v0 = *reinterpret_cast<const __half2 *>(&w0);
      const __half2 v1 = *reinterpret_cast<const __half2 *>(&w1);
      const __half2 lerp = __hfma2(wx2, __hsub2(v1, v0), v0);
      acc = __hfma2(wqh[q], lerp, acc);
    }
    out[u] = acc;
  }
}

// encode_level<float, 2> without branches between the loads: every row's
// 16-byte group of corner x0 (skipped for zero-weight rows) and, where x1
// lies in another group, x1's entry are loaded together, then selected by
// word. The half of its group x0 takes is known from row 0's (the y and z
// multipliers are odd), and x1 shares the group when cx ^ (cx + 1), masked,
// is below 2. The same values as encode_level: x1 reads 0 where wx = 0.
__device__ __forceinline__ void encode_level_f32x2(const float *__restrict__ tab, uint32_t mask, const float3 &p,
                                                   float N, float (&out)[2]) {
  static_assert((kPi2 & 1u) && (kPi3 & 1u), "the row parity needs odd y and z multipliers");
  const Cell c = lattice_cell(p, N);
  const bool nx = c.wx != 0.f, ny = c.wy != 0.f, nz = c.wz != 0.f;
  const uint32_t hy0 = c.cy * kPi2, hy1 = (c.cy + 1u) * kPi2;
  const uint32_t hz0 = c.cz * kPi3, hz1 = (c.cz + 1u) * kPi3;
  const bool j0 = ((c.cx ^ hy0 ^ hz0) & 1u) != 0u;
  const bool same = ((c.cx ^ (c.cx + 1u)) & mask) < 2u;
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab);
  uint4 ga[4];
  uint2 gb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const bool pa = (dy == 0 || ny) && (dz == 0 || nz);
    const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
    const uint32_t ia = (c.cx ^ b) & mask, ib = ((c.cx + 1u) ^ b) & mask;
    ga[q] = ldg16_if(base + (size_t)(ia & ~1u) * 8, pa);
    gb[q] = ldg8_if(base + (size_t)ib * 8, pa && nx && !same);
  }
  out[0] = out[1] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const bool ja = (dy ^ dz) ? !j0 : j0;
    const float a0 = __uint_as_float(ja ? ga[q].z : ga[q].x), a1 = __uint_as_float(ja ? ga[q].w : ga[q].y);
    const float o0 = __uint_as_float(ja ? ga[q].x : ga[q].z), o1 = __uint_as_float(ja ? ga[q].y : ga[q].w);
    const float b0 = nx ? (same ? o0 : __uint_as_float(gb[q].x)) : 0.f;
    const float b1 = nx ? (same ? o1 : __uint_as_float(gb[q].y)) : 0.f;
    const float wyz = (dy ? c.wy : 1.f - c.wy) * (dz ? c.wz : 1.f - c.wz);
    out[0] = fmaf(wyz, fmaf(c.wx, b0 - a0, a0), out[0]);
    out[1] = fmaf(wyz, fmaf(c.wx, b1 - a1, a1), out[1]);
  }
}

// The same gather split into issue and interpolation, so that the loads of
// the next level are in flight while the current level is interpolated
// (a two-stage software pipeline over the levels of a column group).
struct LevelLoads {
  uint4 ga[4];
  uint32_t gb[4];
  uint32_t sel;  // row q: bits 4q..4q+1 = low bits of the x0 index, 4q+2..4q+3 of the x1 index
  float wx, wy, wz;
  bool far;
};

__device__ __forceinline__ void level_issue(const uint8_t *tl, uint32_t mask, const float3 &p, float N, LevelLoads &s) {
  const Cell c = lattice_cell(p, N);
  s.wx = c.wx;
  s.wy = c.wy;
  s.wz = c.wz;
  const uint32_t hy0 = c.cy * kPi2, hy1 = hy0 + kPi2;
  const uint32_t hz0 = c.cz * kPi3, hz1 = hz0 + kPi3;
  uint32_t ia[4], ib[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int dy = q & 1, dz = q >> 1;
    const uint32_t b = (dy ? hy1 : hy0) ^ (dz ? hz1 : hz0);
    ia[q] = (c.cx ^ b) & mask;
    ib[q] = ((c.cx + 1u) ^ b) & mask;
  }
  s.far = ((ia[0] ^ ib[0]) >= 4u) && c.wx != 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) s.ga[q] = __ldg(reinterpret_cast<const uint4 *>(tl + (size_t)(ia[q] & ~3u) * 4));
  ldg4x4_if(s.gb, tl + (size_t)ib[0] * 4, tl + (size_t)ib[1] * 4, tl + (size_t)ib[2] * 4, tl + (size_t)ib[3] * 4,
            s.far);
  uint32_t sel = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) sel |= ((ia[q] & 3u) | ((ib[q] & 3u) << 2)) << (4 * q);
  s.sel = sel;
}

__device__ __forceinline__ __half2 level_finish(const LevelLoads &s) {
  const float w0y = 1.f - s.wy, w0z = 1.f - s.wz;
  const float wq[4] = {w0y * w0z, s.wy * w0z, w0y * s.wz, s.wy * s.wz};
  const __half2 wx2 = __float2half2_rn(s.wx);
  __half2 acc = __float2half2_rn(0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t w0 = word4(s.ga[q], (s.sel >> (4 * q)) & 3u);
    const uint32_t w1 = s.far ? s.gb[q] : word4(s.ga[q], (s.sel >> (4 * q + 2)) & 3u);
    const __half2 v0 = *reinterpret_cast<const __half2 *>(&w0);
    const __half2 v1 = *reinterpret_cast<const __half2 *>(&w1);
    const __half2 lerp = __hfma2(wx2, __hsub2(v1, v0), v0);
    acc = __hfma2(__float2half2_rn(wq[q]), lerp, acc);
  }
  return acc;
}

// NL consecutive levels (tables level_stride bytes apart) of one point.
template <int NL>
__device__ __forceinline__ void encode_levels_h2_pipelined(const __half *__restrict__ tab0, size_t level_stride,
                                                           uint32_t mask, const float3 &p, const float *Ns,
                                                           __half2 (&out)[NL]) {
  const uint8_t *base = reinterpret_cast<const uint8_t *>(tab0);
  LevelLoads st[2];
  level_issue(base, mask, p, Ns[0], st[0]);
#pragma unroll
  for (int u = 0; u < NL; ++u) {
    if (u + 1 < NL) level_issue(base + (size_t)(u + 1) * level_stride, mask, p, Ns[u + 1], st[(u + 1) & 1]);
    out[u] = level_finish(st[u & 1]);
  }
}

// Scatter of a feature gradient into the level's table (backward of
// encode_level): table[idx] += weight * g, every non-zero corner.
__device__ __forceinline__ void encode_level_backward(float *__restrict__ gtab, uint32_t mask, const float3 &p,
                                                      float N, const float *g, int F) {
  Cell c = lattice_cell(p, N);
#pragma unroll
  for (int corner = 0; corner < 8; ++corner) {
    const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
    const float w = (dx ? c.wx : 1.f - c.wx) * (dy ? c.wy : 1.f - c.wy) * (dz ? c.wz : 1.f - c.wz);
    if (w == 0.f) continue;
    const uint32_t idx = hash3(c.cx + dx, c.cy + dy, c.cz + dz) & mask;
    float *dst = gtab + (size_t)idx * F;
    // one vector reduction per entry where the entry is 8 or 16 bytes
    if (F == 2) {
      atomicAdd(reinterpret_cast<float2 *>(dst), make_float2(w * g[0], w * g[1]));
    } else if (F == 4) {
      atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(w * g[0], w * g[1], w * g[2], w * g[3]));
    } else {
      for (int f = 0; f < F; ++f) atomicAdd(dst + f, w * g[f]);
    }
  }
}

}  // namespace lsnif
