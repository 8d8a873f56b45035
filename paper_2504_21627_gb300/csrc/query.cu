// Query kernels shared by both precisions (traversal, grouping) and the plain
// FP32 path (gather kernel, SIMT network + decode kernel), plus the stage
// kernels behind lsnif_trace / lsnif_encode / lsnif_corner_indices /
// lsnif_mlp.
#include <algorithm>
#include <cstdio>

#include "device.cuh"
#include "encode.cuh"

namespace lsnif {

// ---------------------------------------------------------------------------
// a1-a5: transform, slab test, 3D-DDA over occupied voxels, boundary points.
// One thread per ray; also histograms live rays by (object slot, k).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trace_kernel(QueryLaunch q, int smem_hist) {
  extern __shared__ int sh_hist[];
  const int nb = q.n_slots * kBuckets;
  if (smem_hist) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
  }
  const int64_t n = q.rays.n;
  const int Hs = q.H_max;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = q.rays.obj ? q.rays.obj[i] : q.rays.single_handle;
    int s = slot_of(q.objs, q.n_slots, h);
    int k = 0;
    float t0 = CUDART_NAN_F, t1 = CUDART_NAN_F;
    if (s < 0) {
      atomicOr(q.err, kErrBadHandle);
      q.s.slot[i] = -1;
      q.s.k[i] = 0;
      q.s.dup[i] = 0u;
      miss_store(q.hits, i, 0);
      continue;
    }
    const DevObject &ob = q.objs[s];
    float3 o, d;
    int ea;
    uint32_t dupm = 0u;
    float tmin = q.rays.tmin[i];
    bool live = ob.kind == 0 &&
                to_unit(ob, q.rays.ox[i], q.rays.oy[i], q.rays.oz[i], q.rays.dx[i], q.rays.dy[i], q.rays.dz[i], o,
                        d) &&
                unit_slab(o, d, tmin, t0, t1, ea);
    if (live) {
      float *P = q.s.pts + (size_t)i * Hs * 3;
      const int cap = ob.H >> 1;
      const uint32_t *occ = ob.occ;
      // exit of the previous segment: an entry with the same (t, axis, face)
      // is the same point, bit for bit
      uint32_t lt = 0u, lf = 0u;
      int la = -2;
      dda_walk(
          ob, o, d, t0, t1, ea, [&](uint32_t vid) { return occupied(occ, vid); },
          [&](const Seg &sg) {
            if (k > 0 && __float_as_uint(sg.tin) == lt && sg.ain == la && __float_as_uint(sg.fin) == lf)
              dupm |= 1u << k;
            lt = __float_as_uint(sg.tout);
            la = sg.aout;
            lf = __float_as_uint(sg.fout);
            float3 a = seg_point(o, d, sg.tin, sg.ain, sg.fin);
            float3 b = seg_point(o, d, sg.tout, sg.aout, sg.fout);
            float *w = P + 6 * k;
            reinterpret_cast<float2 *>(w)[0] = make_float2(a.x, a.y);
            reinterpret_cast<float2 *>(w)[1] = make_float2(a.z, b.x);
            reinterpret_cast<float2 *>(w)[2] = make_float2(b.y, b.z);
            ++k;
            return k < cap;
          });
    } else {
      t0 = t1 = CUDART_NAN_F;
    }
    q.s.k[i] = (uint8_t)k;
    q.s.dup[i] = dupm;
    q.s.slot[i] = (int16_t)s;
    reinterpret_cast<float2 *>(q.s.t01)[i] = make_float2(t0, t1);
    if (k == 0) miss_store(q.hits, i, ob.n_out);
    if (k > 0) {
      if (smem_hist) atomicAdd(&sh_hist[s * kBuckets + k], 1);
      else atomicAdd(&q.s.counts[s * kBuckets + k], 1);
    }
  }
  if (smem_hist) {
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      if (sh_hist[b]) atomicAdd(&q.s.counts[b], sh_hist[b]);
  }
}

// bits 0..7 of v moved to bits 0, 3, 6, ..., 21
__device__ __forceinline__ uint32_t spread_bits3(uint32_t v) {
  v &= 0xffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// ---------------------------------------------------------------------------
// Presorted traversal (trace mode 2): before the persistent-lane kernel, a
// counting sort hands it the rays in the order (object, Morton cell of the
// point where the ray enters the object's unit cube, direction octant), so
// the lanes of a warp walk neighbouring voxels in similar directions even
// when the rays arrive shuffled (secondary rays, rays mixed across objects):
// their distance-field and occupancy loads share cache lines and their step
// counts are alike. Rays that miss their box or name an unknown object go to
// one last bin; the traversal answers them as before. The key of each ray
// is kept in q.s.dup (the traversal overwrites it later) and the order in
// q.s.order (the grouping overwrites it later).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t presort_key(const QueryLaunch &q, int64_t i, int key_bits, uint32_t last) {
  const uint32_t h = q.rays.obj ? q.rays.obj[i] : q.rays.single_handle;
  const int s = slot_of(q.objs, q.n_slots, h);
  if (s < 0) return last;
  const DevObject &ob = q.objs[s];
  float3 o, d;
  float t0, t1;
  int ea;
  if (!(ob.kind == 0 && to_unit(ob, q.rays.ox[i], q.rays.oy[i], q.rays.oz[i], q.rays.dx[i], q.rays.dy[i],
                                q.rays.dz[i], o, d) &&
        unit_slab(o, d, q.rays.tmin[i], t0, t1, ea)))
    return last;
  const int m = key_bits / 3 - 1;  // cell bits per axis; 3 bits go to the octant
  const float scale = (float)(1 << m);
  const float e[3] = {fmaf(t0, d.x, o.x), fmaf(t0, d.y, o.y), fmaf(t0, d.z, o.z)};
  uint32_t cell = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const uint32_t c = (uint32_t)min(max((int)(e[a] * scale), 0), (1 << m) - 1);
    cell |= spread_bits3(c) << a;
  }
  const uint32_t oct = (d.x < 0.f ? 1u : 0u) | (d.y < 0.f ? 2u : 0u) | (d.z < 0.f ? 4u : 0u);
  return ((uint32_t)s << key_bits) | (cell << 3) | oct;
}

__global__ void __launch_bounds__(256) presort_count_kernel(QueryLaunch q, int key_bits, uint32_t last) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < q.rays.n;
  const uint32_t key = in ? presort_key(q, i, key_bits, last) : 0u;
  if (in) q.s.dup[i] = key;
  const unsigned active = __ballot_sync(0xffffffffu, in);
  if (in) {
    const unsigned peers = __match_any_sync(active, key);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&q.s.bins[key], __popc(peers));
  }
}

__global__ void __launch_bounds__(256) presort_scatter_kernel(QueryLaunch q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool in = i < q.rays.n;
  const uint32_t key = in ? q.s.dup[i] : 0u;
  const unsigned active = __ballot_sync(0xffffffffu, in);
  if (in) {
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&q.s.bins[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    q.s.order[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// ---------------------------------------------------------------------------
// Persistent-lane traversal: after each round of cells a warp hands a new
// ray to every lane whose ray finished (global ray counter, warp-aggregated).
// Rays need anywhere from 0 to 3V DDA steps; with one ray per thread a warp
// runs as long as its longest ray.
//
// Empty-space skipping: every iteration crosses one cell: the cube of
// voxels within Chebyshev distance r of the current voxel, where r + 1 is
// the voxel's distance to the nearest occupied voxel (so the whole cube is
// empty; r = 0 is the voxel itself). All cells are crossed by the same
// instruction sequence (exit plane per axis, earliest axis with the lowest
// axis on ties, cross it), so lanes of a warp do not split between a voxel
// path and a skipping path. Crossing times are the same expression of the
// plane index as in the voxel-by-voxel walk (dda_walk), and when a cube is
// crossed the other axes first step over every plane the walk would cross
// before it, so the voxels visited, the boundary points and the shared-point
// marks are exactly those of the voxel-by-voxel walk (trace_kernel).
// ---------------------------------------------------------------------------
struct LaneRay {
  int64_t i;
  int s;           // object slot
  float3 o, d;
  float inv0, inv1, inv2;
  int ix0, ix1, ix2, st0, st1, st2;
  float tcur, t0, t1;
  int ain;
  float fin;
  int k, cap;
  int r;           // the current cell: voxels within r of (ix0, ix1, ix2), all empty when r > 0
  bool occ;        // the current voxel is occupied (its distance is 0)
  uint32_t dup;    // bit k: entry point of segment k equals the exit of segment k-1
  uint32_t lt, lf; // exit (t, face) of the last segment, as bits
  int la;          // and its axis
};

__device__ __forceinline__ float sel3(int a, float x, float y, float z) { return a == 0 ? x : (a == 1 ? y : z); }
__device__ __forceinline__ int sel3i(int a, int x, int y, int z) { return a == 0 ? x : (a == 1 ? y : z); }

// crossing time of plane index P on one axis (the expression dda_walk uses)
__device__ __forceinline__ float plane_t(int P, float invV, float o, float inv) { return ((float)P * invV - o) * inv; }

// Planes that one axis crosses before the current cell's exit time ea, as
// the voxel walk counts them: plane m of the axis (m = 0, 1, ...) is
// ix + 1 + m for st > 0 and ix - m for st < 0, crossed when its time is
// below ea, or equal to it when the axis wins the tie (`tie`). Plane times
// are monotone in m (each operation of plane_t is), so the crossed planes
// are a prefix: the count is guessed from the position at ea and then
// corrected with the exact comparisons until plane n is the first one not
// crossed. At most `cap` planes; 0 when the axis does not move.
__device__ __forceinline__ int planes_before(int ix, int st, float o, float d, float inv, float invV, int V,
                                             float ea, bool tie, int cap) {
  if (st == 0 || cap <= 0) return 0;
  auto crosses = [&](int m) {
    const float t = plane_t(st > 0 ? ix + 1 + m : ix - m, invV, o, inv);
    return t < ea || (tie && t == ea);
  };
  const float xe = fmaf(ea, d, o) * (float)V;  // position at ea, in voxels
  float g = st > 0 ? floorf(xe) - (float)ix : (float)ix - ceilf(xe) + 1.f;
  g = fminf(fmaxf(g, 0.f), (float)cap);          // also maps NaN to 0
  int n = (int)g;
  while (n > 0 && !crosses(n - 1)) --n;
  while (n < cap && crosses(n)) ++n;
  return n;
}

// occupancy distance of voxel (x, y, z): 0 when occupied, else the radius
// of the empty cube around it is D - 1
__device__ __forceinline__ int voxel_distance(const DevObject &ob, int x, int y, int z) {
  return __ldg(ob.dist + ((uint32_t)z * ob.V + (uint32_t)y) * ob.V + (uint32_t)x);
}

__global__ void __launch_bounds__(256) trace_pool_kernel(QueryLaunch q, int smem_hist, int steps_per_round,
                                                          const int32_t *__restrict__ perm) {
  extern __shared__ int sh_hist[];
  const int nb = q.n_slots * kBuckets;
  if (smem_hist) {
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
  }
  const int64_t n = q.rays.n;
  const int Hs = q.H_max;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  LaneRay R;
  R.i = -1;
  bool exhausted = false;
  int* counter = q.s.meta + 4;

  auto finish = [&](void) {
    const int64_t i = R.i;
    q.s.k[i] = (uint8_t)R.k;
    q.s.dup[i] = R.dup;
    q.s.slot[i] = (int16_t)R.s;
    reinterpret_cast<float2 *>(q.s.t01)[i] = make_float2(R.t0, R.t1);
    if (R.k == 0) miss_store(q.hits, i, q.objs[R.s].n_out);
    else if (smem_hist) atomicAdd(&sh_hist[R.s * kBuckets + R.k], 1);
    else atomicAdd(&q.s.counts[R.s * kBuckets + R.k], 1);
    R.i = -1;
  };

  for (;;) {
    // refill: a lane without a ray takes rays until one enters its object's
    // box (a ray that misses it is answered at once, so no lane spends the
    // round idle on it) or the pool is empty
    for (;;) {
      const bool need = R.i < 0 && !exhausted;
      const unsigned m = __ballot_sync(FULL, need);
      if (!m) break;
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(counter, __popc(m));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int64_t pos = (int64_t)base + __popc(m & ((1u << lane) - 1u));
        if (pos >= n) {
          exhausted = true;
        } else {
          // start ray `my` (the pos-th ray of the presorted order, if any)
          const int64_t my = perm ? (int64_t)__ldg(perm + pos) : pos;
          R.i = my;
          const uint32_t h = q.rays.obj ? q.rays.obj[my] : q.rays.single_handle;
          R.s = slot_of(q.objs, q.n_slots, h);
          R.k = 0;
          R.dup = 0u;
          R.la = -2;
          R.t0 = R.t1 = CUDART_NAN_F;
          if (R.s < 0) {
            atomicOr(q.err, kErrBadHandle);
            q.s.slot[my] = -1;
            q.s.k[my] = 0;
            q.s.dup[my] = 0u;
            miss_store(q.hits, my, 0);
            R.i = -1;
          } else {
            const DevObject &ob = q.objs[R.s];
            int ea;
            float t0, t1;
            bool live = ob.kind == 0 &&
                        to_unit(ob, q.rays.ox[my], q.rays.oy[my], q.rays.oz[my], q.rays.dx[my], q.rays.dy[my],
                                q.rays.dz[my], R.o, R.d) &&
                        unit_slab(R.o, R.d, q.rays.tmin[my], t0, t1, ea);
            if (!live) {
              finish();
            } else {
              R.t0 = t0;
              R.t1 = t1;
              R.cap = ob.H >> 1;
              const int V = ob.V;
              const float3 p = make_float3(fmaf(t0, R.d.x, R.o.x), fmaf(t0, R.d.y, R.o.y), fmaf(t0, R.d.z, R.o.z));
              int c[3];
              float dd[3] = {R.d.x, R.d.y, R.d.z}, pp[3] = {p.x, p.y, p.z};
              int stv[3];
              float invv[3];
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                int cc = (int)floorf(pp[a] * (float)V);
                cc = min(max(cc, 0), V - 1);
                if (a == ea) cc = dd[a] > 0.f ? 0 : V - 1;
                c[a] = cc;
                stv[a] = dd[a] > 0.f ? 1 : (dd[a] < 0.f ? -1 : 0);
                invv[a] = dd[a] != 0.f ? 1.f / dd[a] : 0.f;
              }
              R.ix0 = c[0]; R.ix1 = c[1]; R.ix2 = c[2];
              R.st0 = stv[0]; R.st1 = stv[1]; R.st2 = stv[2];
              R.inv0 = invv[0]; R.inv1 = invv[1]; R.inv2 = invv[2];
              R.tcur = t0;
              R.ain = ea;
              R.fin = ea >= 0 ? (dd[ea] > 0.f ? 0.f : 1.f) : 0.f;
              const int D = voxel_distance(ob, c[0], c[1], c[2]);
              R.r = D > 0 ? D - 1 : 0;
              R.occ = D == 0;
            }
          }
        }
      }
    }
    if (__all_sync(FULL, R.i < 0 && exhausted)) break;
    if (R.i < 0) continue;
    // up to steps_per_round cells of this lane's ray
    const DevObject &ob = q.objs[R.s];
    const int V = ob.V;
    const float invV = ob.invV;
    float *P = q.s.pts + (size_t)R.i * Hs * 3;
    for (int it = 0; it < steps_per_round; ++it) {
      bool done = false;
      const int rr = R.r;  // cell: the voxel, or the empty cube of radius rr around it
      // exit plane of the cell on each axis, and its crossing time
      const int P0 = R.st0 > 0 ? R.ix0 + rr + 1 : R.ix0 - rr;
      const int P1 = R.st1 > 0 ? R.ix1 + rr + 1 : R.ix1 - rr;
      const int P2 = R.st2 > 0 ? R.ix2 + rr + 1 : R.ix2 - rr;
      const float e0 = R.st0 != 0 ? plane_t(P0, invV, R.o.x, R.inv0) : CUDART_INF_F;
      const float e1 = R.st1 != 0 ? plane_t(P1, invV, R.o.y, R.inv1) : CUDART_INF_F;
      const float e2 = R.st2 != 0 ? plane_t(P2, invV, R.o.z, R.inv2) : CUDART_INF_F;
      const int a = (e0 <= e1) ? (e0 <= e2 ? 0 : 2) : (e1 <= e2 ? 1 : 2);
      const float ea = sel3(a, e0, e1, e2);
      const int Pa = sel3i(a, P0, P1, P2);
      const float tx = fminf(ea, R.t1);
      if (R.occ && tx > R.tcur) {
        const float fx = (float)Pa * invV;
        if (R.k > 0 && __float_as_uint(R.tcur) == R.lt && R.ain == R.la && __float_as_uint(R.fin) == R.lf)
          R.dup |= 1u << R.k;
        R.lt = __float_as_uint(tx);
        R.la = a;
        R.lf = __float_as_uint(fx);
        const float3 pa = seg_point(R.o, R.d, R.tcur, R.ain, R.fin);
        const float3 pb = seg_point(R.o, R.d, tx, a, fx);
        float *w = P + 6 * R.k;
        reinterpret_cast<float2 *>(w)[0] = make_float2(pa.x, pa.y);
        reinterpret_cast<float2 *>(w)[1] = make_float2(pa.z, pb.x);
        reinterpret_cast<float2 *>(w)[2] = make_float2(pb.y, pb.z);
        if (++R.k >= R.cap) done = true;
      }
      if (!done && ea >= R.t1) done = true;
      if (!done) {
        // when a cube is crossed, the other axes first cross the planes the
        // voxel walk crosses before (ea, a) -- at most 2 rr each; for a voxel
        // there are none
        // A cube may reach past the grid: an axis whose next plane is the
        // grid's own boundary leaves the grid there, and the voxel walk
        // ends at that crossing (the slab's exit time and the plane's
        // crossing time may round differently), so the ray ends here too
        // -- the cube holds no occupied voxel, so nothing is lost.
        bool out = false;
        if (rr) {
          // axis b moves n_b voxels; stepping onto voxel -1 or V (more steps
          // than the grid leaves, m_b) means the ray leaves the grid first
          const int n0 = a == 0 ? 0 : planes_before(R.ix0, R.st0, R.o.x, R.d.x, R.inv0, invV, V, ea, true, 2 * rr);
          const int n1 = a == 1 ? 0 : planes_before(R.ix1, R.st1, R.o.y, R.d.y, R.inv1, invV, V, ea, a == 2, 2 * rr);
          const int n2 = a == 2 ? 0 : planes_before(R.ix2, R.st2, R.o.z, R.d.z, R.inv2, invV, V, ea, false, 2 * rr);
          out = n0 > (R.st0 > 0 ? V - 1 - R.ix0 : R.ix0) || n1 > (R.st1 > 0 ? V - 1 - R.ix1 : R.ix1) ||
                n2 > (R.st2 > 0 ? V - 1 - R.ix2 : R.ix2);
          R.ix0 += R.st0 * n0;
          R.ix1 += R.st1 * n1;
          R.ix2 += R.st2 * n2;
        }
        // then axis a crosses its plane
        const int sa = sel3i(a, R.st0, R.st1, R.st2);
        const int ia = sa > 0 ? Pa : Pa - 1;
        if (out || ia < 0 || ia >= V) {
          done = true;
        } else {
          R.tcur = ea;
          R.ain = a;
          R.fin = (float)Pa * invV;
          if (a == 0) R.ix0 = ia;
          else if (a == 1) R.ix1 = ia;
          else R.ix2 = ia;
          // the next cell is centred on the voxel just entered (indices
          // are checked: a violation is reported, never read)
          if ((unsigned)R.ix0 >= (unsigned)V || (unsigned)R.ix1 >= (unsigned)V || (unsigned)R.ix2 >= (unsigned)V) {
            atomicOr(q.err, kErrCheck);
            done = true;
          } else {
            const int D = voxel_distance(ob, R.ix0, R.ix1, R.ix2);
            R.r = D > 0 ? D - 1 : 0;
            R.occ = D == 0;
          }
        }
      }
      if (done) {
        finish();
        break;
      }
    }
  }
  if (smem_hist) {
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      if (sh_hist[b]) atomicAdd(&q.s.counts[b], sh_hist[b]);
  }
}

// Single block: bucket offsets (object ascending, k descending), tiles of
// kTileM rays that never straddle objects, totals, cursors reset.
__global__ void __launch_bounds__(1024) scan_kernel(QueryLaunch q) {
  __shared__ int tile_off[1025];
  __shared__ int obj_live[1024];
  const int ns = q.n_slots;
  if (threadIdx.x == 0) {
    int run = 0, tiles = 0, pts = 0;
    for (int s = 0; s < ns; ++s) {
      int start = run;
      for (int k = kMaxCap; k >= 1; --k) {
        int c = q.s.counts[s * kBuckets + k];
        // group modes 2 and 3: one bucket per object (bucket k = 1 takes all)
        q.s.offsets[s * kBuckets + k] = q.group_mode >= 2 ? start : run;
        q.s.cursor[s * kBuckets + k] = 0;
        run += c;
        pts += 2 * k * c;
      }
      int live = run - start;
      if (s < 1024) {
        obj_live[s] = start;  // start of the object's range
        tile_off[s] = tiles;
      }
      tiles += (live + kTileM - 1) / kTileM;
    }
    if (ns <= 1024) tile_off[ns] = tiles;
    if (tiles > q.s.max_tiles) {
      atomicOr(q.err, kErrCheck);
      tiles = q.s.max_tiles;
    }
    q.s.meta[0] = run;
    q.s.meta[1] = tiles;
    q.s.meta[2] = pts;
    q.s.meta[3] = 0;
  }
  __syncthreads();
  const int tiles = q.s.meta[1];
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
    // object of tile t: last s with tile_off[s] <= t
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    int s = lo;
    int first = obj_live[s];
    int obj_end = first;
    for (int k = 1; k <= kMaxCap; ++k) obj_end += q.s.counts[s * kBuckets + k];
    int start = first + (t - tile_off[s]) * kTileM;
    int cnt = min(kTileM, obj_end - start);
    q.s.tiles[3 * t + 0] = s;
    q.s.tiles[3 * t + 1] = start;
    q.s.tiles[3 * t + 2] = cnt;
  }
}

// Scatter live rays into their bucket ranges; warp-aggregated atomics keep
// rays of one warp contiguous (spatially coherent rays stay together). In
// group mode 2 a bucket is a whole object (point counts mixed), so
// consecutive rays of an object stay close in the tile order.
__global__ void __launch_bounds__(256) scatter_kernel(QueryLaunch q) {
  const int64_t n = q.rays.n;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = base + threadIdx.x;
    int bucket = -1;
    if (i < n) {
      int k = q.s.k[i];
      int s = q.s.slot[i];
      if (k > 0 && s >= 0) bucket = s * kBuckets + (q.group_mode == 2 ? 1 : k);
    }
    unsigned active = __ballot_sync(0xffffffffu, bucket >= 0);
    if (bucket >= 0) {
      unsigned peers = __match_any_sync(active, bucket);
      int leader = __ffs(peers) - 1;
      int rank = __popc(peers & ((1u << lane) - 1u));
      int basep = 0;
      if (lane == leader) basep = atomicAdd(&q.s.cursor[bucket], __popc(peers));
      basep = __shfl_sync(peers, basep, leader);
      q.s.order[q.s.offsets[bucket] + basep + rank] = (int32_t)i;
    }
  }
}

// The same with each block's counts summed in shared memory first: one
// global atomic per block and bucket instead of one per warp and bucket (a
// query's few buckets otherwise take every warp's atomics). One ray per
// thread; nb = n_slots x kBuckets counts and as many block bases in shared
// memory.
__global__ void __launch_bounds__(1024) scatter_block_kernel(QueryLaunch q, int nb) {
  extern __shared__ int sh_scatter[];
  int *s_cnt = sh_scatter, *s_base = sh_scatter + nb;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s_cnt[b] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int bucket = -1;
  if (i < q.rays.n) {
    const int k = q.s.k[i];
    const int s = q.s.slot[i];
    if (k > 0 && s >= 0) bucket = s * kBuckets + (q.group_mode == 2 ? 1 : k);
  }
  const unsigned active = __ballot_sync(0xffffffffu, bucket >= 0);
  int rank = 0;
  if (bucket >= 0) {
    const unsigned peers = __match_any_sync(active, bucket);
    const int leader = __ffs(peers) - 1;
    int wbase = 0;
    if (lane == leader) wbase = atomicAdd(&s_cnt[bucket], __popc(peers));
    wbase = __shfl_sync(peers, wbase, leader);
    rank = wbase + __popc(peers & ((1u << lane) - 1u));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int c = s_cnt[b];
    s_base[b] = c ? atomicAdd(&q.s.cursor[b], c) : 0;
  }
  __syncthreads();
  if (bucket >= 0) q.s.order[q.s.offsets[bucket] + s_base[bucket] + rank] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// Order-keeping grouping for single-object queries: live rays are compacted
// in their original order, so a 128-ray tile holds neighbouring rays (for
// primary rays: neighbouring pixels, which share voxels and lattice cells).
// count: live rays and points per block of kGroupBlock rays; scan: block
// offsets, totals and the tile table; scatter: stable ranks within a block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) group_count_kernel(QueryLaunch q, int nblk) {
  __shared__ int s_live[32], s_pts[32];
  const int b = blockIdx.x;
  int live = 0, pts = 0;
  for (int r = 0; r < kGroupBlock / 1024; ++r) {
    const int64_t i = (int64_t)b * kGroupBlock + r * 1024 + threadIdx.x;
    if (i < q.rays.n && q.s.slot[i] >= 0) {
      const int k = q.s.k[i];
      live += k > 0;
      pts += 2 * k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    live += __shfl_down_sync(0xffffffffu, live, o);
    pts += __shfl_down_sync(0xffffffffu, pts, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_live[threadIdx.x >> 5] = live;
    s_pts[threadIdx.x >> 5] = pts;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, c = 0;
    for (int w = 0; w < 32; ++w) { a += s_live[w]; c += s_pts[w]; }
    q.s.blk[b] = a;
    q.s.blk[nblk + b] = c;
  }
}

__global__ void __launch_bounds__(1024) group_scan_kernel(QueryLaunch q, int nblk) {
  __shared__ int s_part[1024];
  __shared__ int s_pts[1024];
  const int per = (nblk + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int sum = 0, pts = 0;
  for (int b = b0; b < min(b0 + per, nblk); ++b) { sum += q.s.blk[b]; pts += q.s.blk[nblk + b]; }
  s_part[threadIdx.x] = sum;
  s_pts[threadIdx.x] = pts;
  __syncthreads();
  if (threadIdx.x == 0) {   // exclusive scan of the 1024 partial sums
    int run = 0, pr = 0;
    for (int t = 0; t < 1024; ++t) {
      const int v = s_part[t];
      s_part[t] = run;
      run += v;
      pr += s_pts[t];
    }
    int tiles = (run + kTileM - 1) / kTileM;
    if (tiles > q.s.max_tiles) {
      atomicOr(q.err, kErrCheck);
      tiles = q.s.max_tiles;
    }
    q.s.meta[0] = run;
    q.s.meta[1] = tiles;
    q.s.meta[2] = pr;
    q.s.meta[3] = 0;
  }
  __syncthreads();
  int run = s_part[threadIdx.x];
  for (int b = b0; b < min(b0 + per, nblk); ++b) {   // block offsets replace the counts
    const int v = q.s.blk[b];
    q.s.blk[b] = run;
    run += v;
  }
  const int n_live = q.s.meta[0], tiles = q.s.meta[1];
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
    q.s.tiles[3 * t + 0] = q.single_slot;
    q.s.tiles[3 * t + 1] = t * kTileM;
    q.s.tiles[3 * t + 2] = min(kTileM, n_live - t * kTileM);
  }
}

__global__ void __launch_bounds__(1024) group_scatter_kernel(QueryLaunch q) {
  __shared__ int s_warp[32];
  __shared__ int s_total;
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = q.s.blk[b];
  for (int r = 0; r < kGroupBlock / 1024; ++r) {
    const int64_t i = (int64_t)b * kGroupBlock + r * 1024 + threadIdx.x;
    const bool live = i < q.rays.n && q.s.slot[i] >= 0 && q.s.k[i] > 0;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int w = 0; w < 32; ++w) {
        const int v = s_warp[w];
        s_warp[w] = run;
        run += v;
      }
      s_total = run;
    }
    __syncthreads();
    if (live) q.s.order[base + s_warp[warp] + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    base += s_total;
    __syncthreads();
  }
}

// exclusive scan of n int32 in place, in blocks of 1024; block totals to sums
__global__ void __launch_bounds__(1024) scan_block_kernel(int32_t *v, int64_t n, int32_t *sums) {
  __shared__ int32_t ws[32];
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t x = i < n ? v[i] : 0;
  int32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int32_t before = (w > 0 ? ws[w - 1] : 0) + inc - x;
  if (i < n) v[i] = before;
  if (threadIdx.x == 1023) sums[blockIdx.x] = ws[31];
}

// single block: exclusive scan of the block sums (any count), total at sums[nb]
__global__ void __launch_bounds__(1024) scan_sums_kernel(int32_t *sums, int nb) {
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ int32_t ws[32];
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int32_t x = i < nb ? sums[i] : 0;
    int32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
      int32_t s = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const int32_t before = carry + (w > 0 ? ws[w - 1] : 0) + inc - x;
    if (i < nb) sums[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += ws[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_add_kernel(int32_t *v, int64_t n, const int32_t *sums) {
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) v[i] += sums[blockIdx.x];
}

// ---------------------------------------------------------------------------
// Spatial grouping (group mode 3): live rays sorted by object, then by the
// Morton code of the cell (2^m per axis of the object's unit cube) that
// holds their first boundary point -- a counting sort over (object, cell)
// bins: count, exclusive scan, scatter. A 128-ray tile then holds rays whose
// points lie close together whatever order the rays came in (secondary
// rays, rays shuffled across objects), so the gathers' corner loads share
// L1 and L2 lines. Objects stay in ascending slot order, so the object
// ranges and tiles of scan_kernel (one bucket per object) hold as they are.
// Rays of one bin land in any order; no result depends on it.
// ---------------------------------------------------------------------------
// (object slot, Morton cell) bin of ray i, or -1 when it is not live
__device__ __forceinline__ int spatial_bin(const QueryLaunch &q, int64_t i, int cell_bits) {
  if (q.s.k[i] == 0) return -1;
  const int s = q.s.slot[i];
  if (s < 0) return -1;
  const float *P = q.s.pts + (size_t)i * q.H_max * 3;
  const int side = 1 << (cell_bits / 3);
  const float scale = (float)side;
  uint32_t c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = (uint32_t)min(max((int)(P[a] * scale), 0), side - 1);
  return (s << cell_bits) | (int)(spread_bits3(c[0]) | (spread_bits3(c[1]) << 1) | (spread_bits3(c[2]) << 2));
}

__global__ void __launch_bounds__(256) spatial_count_kernel(QueryLaunch q, int cell_bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bin = i < q.rays.n ? spatial_bin(q, i, cell_bits) : -1;
  const unsigned active = __ballot_sync(0xffffffffu, bin >= 0);
  if (bin >= 0) {
    const unsigned peers = __match_any_sync(active, bin);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&q.s.bins[bin], __popc(peers));
  }
}

// bins hold the bins' first positions; each warp takes its rays' ranks
__global__ void __launch_bounds__(256) spatial_scatter_kernel(QueryLaunch q, int cell_bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int bin = i < q.rays.n ? spatial_bin(q, i, cell_bits) : -1;
  const unsigned active = __ballot_sync(0xffffffffu, bin >= 0);
  if (bin >= 0) {
    const unsigned peers = __match_any_sync(active, bin);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&q.s.bins[bin], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    q.s.order[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// ---------------------------------------------------------------------------
// FP32 path: gather into X, one chunk of tiles at a time. Row (t, r) of the
// chunk is ray r of tile t; the row stride is the largest input width.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void encode_level_any(const DevObject &ob, const float *tab, const float3 &p, int l,
                                                 float *out) {
  const float *tl = tab + (size_t)l * (ob.mask + 1) * ob.F;
  const float N = (float)ob.res[l];
  if (ob.F == 2) {
    float f[2];
    encode_level<float, 2>(tl, ob.mask, p, N, f);
    out[0] = f[0]; out[1] = f[1];
  } else if (ob.F == 4) {
    float f[4];
    encode_level<float, 4>(tl, ob.mask, p, N, f);
    out[0] = f[0]; out[1] = f[1]; out[2] = f[2]; out[3] = f[3];
  } else {
    float f[1];
    encode_level<float, 1>(tl, ob.mask, p, N, f);
    out[0] = f[0];
  }
}

__global__ void __launch_bounds__(256) gather_fp32_kernel(QueryLaunch q, int tile0, int ntile, int ldx) {
  const int Hs = q.H_max;
  const int64_t tot = (int64_t)ntile * kTileM * Hs;
  const int n_tiles = q.s.meta[1];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(e % Hs);
    const int64_t rr = e / Hs;
    const int r = (int)(rr % kTileM);
    const int t = tile0 + (int)(rr / kTileM);
    if (t >= n_tiles) continue;
    const int slot = q.s.tiles[3 * t], start = q.s.tiles[3 * t + 1], cnt = q.s.tiles[3 * t + 2];
    if (r >= cnt) continue;
    const DevObject &ob = q.objs[slot];
    if (h >= ob.H) continue;
    const int32_t ray = q.s.order[start + r];
    const int k = q.s.k[ray];
    const int LF = ob.L * ob.F;
    float *xo = q.s.X + ((int64_t)(t - tile0) * kTileM + r) * ldx + (size_t)h * LF;
    if (h >= 2 * k) {
      for (int j = 0; j < LF; ++j) xo[j] = 0.f;
      continue;
    }
    const float *P = q.s.pts + ((size_t)ray * Hs + h) * 3;
    const float3 p = make_float3(P[0], P[1], P[2]);
    for (int l = 0; l < ob.L; ++l) encode_level_any(ob, ob.tab32, p, l, xo + l * ob.F);
  }
}

// ---------------------------------------------------------------------------
// FP32 SIMT network: 128-row tiles, activations stay in shared memory
// between layers; decode in the epilogue.
// ---------------------------------------------------------------------------
constexpr int kMT = kTileM;  // rows per tile
constexpr int kKC = 32;      // K chunk

// out[N][kMT] = act(W[N][K] . in + b); in is global rows (Xg, stride ldx,
// rows_valid valid) or shared [K][kMT].
template <int CPT>
__device__ __forceinline__ void simt_layer(const float *__restrict__ Ain, const float *__restrict__ Xg, int64_t ldx,
                                           int rows_valid, int K, int N, const float *__restrict__ W,
                                           const float *__restrict__ bias, int act, bool apply_act, float *As,
                                           float *Ws, float *Aout) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // 16 column groups x 16 row groups of 8
  float acc[8][CPT];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
  for (int kc = 0; kc < K; kc += kKC) {
    const int kn = min(kKC, K - kc);
    __syncthreads();
    if (Xg) {
      for (int e = tid; e < kMT * kKC; e += blockDim.x) {
        const int r = e / kKC, kk = e % kKC;
        As[kk * kMT + r] = (r < rows_valid && kk < kn) ? Xg[(int64_t)r * ldx + kc + kk] : 0.f;
      }
    }
    for (int e = tid; e < kKC * N; e += blockDim.x) {
      const int nn = e / kKC, kk = e % kKC;
      Ws[kk * N + nn] = kk < kn ? W[(int64_t)nn * K + kc + kk] : 0.f;
    }
    __syncthreads();
    const float *A = Xg ? As : (Ain + (size_t)kc * kMT);
    for (int kk = 0; kk < kn; ++kk) {
      float a[8], b[CPT];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = A[kk * kMT + ty * 8 + i];
#pragma unroll
      for (int j = 0; j < CPT; ++j) b[j] = Ws[kk * N + tx * CPT + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int col = tx * CPT + j;
    const float bj = bias[col];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = acc[i][j] + bj;
      Aout[col * kMT + ty * 8 + i] = apply_act ? act_fn(v, act) : v;
    }
  }
  __syncthreads();
}

__device__ void simt_dispatch(int N, const float *Ain, const float *Xg, int64_t ldx, int rows_valid, int K,
                              const float *W, const float *bias, int act, bool apply_act, float *As, float *Ws,
                              float *Aout) {
  switch (N / 16) {
    case 1: simt_layer<1>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    case 2: simt_layer<2>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    case 3: simt_layer<3>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    case 4: simt_layer<4>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    case 8: simt_layer<8>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    case 16: simt_layer<16>(Ain, Xg, ldx, rows_valid, K, N, W, bias, act, apply_act, As, Ws, Aout); break;
    default: {
      // other multiples of 16: generic path, 1 column group at a time
      for (int n0 = 0; n0 < N; n0 += 16)
        simt_layer<1>(Ain, Xg, ldx, rows_valid, K, 16, W + (int64_t)n0 * K, bias + n0, act, apply_act, As, Ws,
                      Aout + (size_t)n0 * kMT);
    }
  }
}

// One tile's network from its input rows X (stride ldx, `rows` valid) into
// logits out[n_out_pad][kMT] (a shared buffer); returns that buffer.
__device__ float *simt_network(const DevObject &ob, const float *X, int64_t ldx, int rows, float *As, float *Ws,
                               float *act0, float *act1) {
  const int W = ob.width;
  const float *p = ob.mlp32;
  simt_dispatch(W, nullptr, X, ldx, rows, ob.n_in, p, p + (size_t)W * ob.n_in, ob.act, true, As, Ws, act0);
  p += (size_t)W * ob.n_in + W;
  float *cur = act0, *nxt = act1;
  for (int l = 1; l < ob.n_hidden; ++l) {
    simt_dispatch(W, cur, nullptr, 0, kMT, W, p, p + (size_t)W * W, ob.act, true, As, Ws, nxt);
    p += (size_t)W * W + W;
    float *tmp = cur; cur = nxt; nxt = tmp;
  }
  // output layer, padded to n_out_pad rows (zero weights) by the launcher's copy
  const float *Wo = ob.plain_out, *bo = ob.plain_out + (size_t)ob.n_out_pad * W;
  simt_dispatch(ob.n_out_pad, cur, nullptr, 0, kMT, W, Wo, bo, ob.act, false, As, Ws, nxt);
  return nxt;
}

__global__ void __launch_bounds__(256) mlp_fp32_kernel(QueryLaunch q, int tile0, int ntile, int ldx) {
  extern __shared__ __align__(16) float sm[];
  const int wmax = q.s.wmax;
  float *As = sm;
  float *Ws = As + kKC * kMT;
  float *act0 = Ws + kKC * wmax;
  float *act1 = act0 + (size_t)wmax * kMT;
  const int n_tiles = q.s.meta[1];
  for (int tt = blockIdx.x; tt < ntile; tt += gridDim.x) {
    const int t = tile0 + tt;
    if (t >= n_tiles) break;
    const int slot = q.s.tiles[3 * t], start = q.s.tiles[3 * t + 1], cnt = q.s.tiles[3 * t + 2];
    const DevObject &ob = q.objs[slot];
    float *Z = simt_network(ob, q.s.X + (int64_t)tt * kMT * ldx, ldx, cnt, As, Ws, act0, act1);
    if (threadIdx.x < cnt) {
      const int r = threadIdx.x;
      float z[64];
      for (int j = 0; j < ob.n_out; ++j) z[j] = Z[j * kMT + r];
      const int32_t ray = q.s.order[start + r];
      const float2 tt01 = reinterpret_cast<const float2 *>(q.s.t01)[ray];
      decode_store(q.hits, ray, z, ob.n_out, ob.n_mat, tt01.x, tt01.y, q.rays.tmin[ray], q.rays.tmax[ray]);
    }
    __syncthreads();
  }
}

// lsnif_mlp, FP32: X rows in, logits out.
__global__ void __launch_bounds__(256) mlp_fp32_rows_kernel(const DevObject *dobj, const float *X, int64_t n,
                                                            float *Zout, int wmax) {
  extern __shared__ __align__(16) float sm[];
  const DevObject &ob = *dobj;
  float *As = sm;
  float *Ws = As + kKC * kMT;
  float *act0 = Ws + kKC * wmax;
  float *act1 = act0 + (size_t)wmax * kMT;
  for (int64_t t0 = (int64_t)blockIdx.x * kMT; t0 < n; t0 += (int64_t)gridDim.x * kMT) {
    const int rv = (int)min((int64_t)kMT, n - t0);
    float *Z = simt_network(ob, X + t0 * ob.n_in, ob.n_in, rv, As, Ws, act0, act1);
    if (threadIdx.x < rv)
      for (int j = 0; j < ob.n_out; ++j) Zout[(t0 + threadIdx.x) * ob.n_out + j] = Z[j * kMT + threadIdx.x];
    __syncthreads();
  }
}

static size_t mlp_fp32_smem(int wmax) {
  return sizeof(float) * ((size_t)kKC * kMT + (size_t)kKC * wmax + 2 * (size_t)wmax * kMT);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

cudaError_t launch_trace(const QueryLaunch &q, int *launches) {
  cudaMemsetAsync(q.s.counts, 0, sizeof(int32_t) * q.n_slots * kBuckets, q.stream);
  const int nb = q.n_slots * kBuckets;
  const int smem_hist = nb <= 12288;
  const size_t smem = smem_hist ? nb * sizeof(int) : 0;
  if (q.trace_mode == 1) {
    cudaMemsetAsync(q.s.meta + 4, 0, sizeof(int32_t), q.stream);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (q.rays.n + 255) / 256;
    const int grid = (int)std::min<int64_t>(need, (int64_t)sms * 8);
    // long rounds: a lane whose ray ends waits for the warp's round to end,
    // so that the next refill starts many rays together (the start of a
    // ray -- unit-cube transform, slab test, first cell -- is the costly,
    // divergent part); 8, 32 and 64 cells per round took 0.76, 0.66 and
    // 0.61 ms on the 4M-ray torus query
    trace_pool_kernel<<<grid, 256, smem, q.stream>>>(q, smem_hist, 64, nullptr);
    *launches += 1;
    return cudaGetLastError();
  }
  if (q.trace_mode == 2) {
    const int key_bits = spatial_cell_bits(q.n_slots);
    const uint32_t last = (uint32_t)q.n_slots << key_bits;  // rays the traversal answers as misses
    const int64_t nbins = (int64_t)last + 1;
    const unsigned blocks = (unsigned)std::max<int64_t>((q.rays.n + 255) / 256, 1);
    cudaMemsetAsync(q.s.meta + 4, 0, sizeof(int32_t), q.stream);
    cudaError_t e = cudaMemsetAsync(q.s.bins, 0, (size_t)nbins * 4, q.stream);
    if (e != cudaSuccess) return e;
    presort_count_kernel<<<blocks, 256, 0, q.stream>>>(q, key_bits, last);
    e = launch_exclusive_scan(q.s.bins, nbins, q.s.bin_sums, q.stream);
    if (e != cudaSuccess) return e;
    presort_scatter_kernel<<<blocks, 256, 0, q.stream>>>(q);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>((q.rays.n + 255) / 256, (int64_t)sms * 8);
    trace_pool_kernel<<<grid, 256, smem, q.stream>>>(q, smem_hist, 64, q.s.order);
    *launches += 6;
    return cudaGetLastError();
  }
  const int grid = grid_for(q.rays.n, 256, 152 * 16);
  trace_kernel<<<grid, 256, smem, q.stream>>>(q, smem_hist);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_group(const QueryLaunch &q, int *launches) {
  if (q.group_mode == 1) {
    const int nblk = (int)((q.rays.n + kGroupBlock - 1) / kGroupBlock);
    group_count_kernel<<<nblk, 1024, 0, q.stream>>>(q, nblk);
    group_scan_kernel<<<1, 1024, 0, q.stream>>>(q, nblk);
    group_scatter_kernel<<<nblk, 1024, 0, q.stream>>>(q);
    *launches += 3;
    return cudaGetLastError();
  }
  if (q.group_mode == 3) {
    const int bits = spatial_cell_bits(q.n_slots);
    const int64_t nbins = (int64_t)q.n_slots << bits;
    const unsigned blocks = (unsigned)std::max<int64_t>((q.rays.n + 255) / 256, 1);
    scan_kernel<<<1, 1024, 0, q.stream>>>(q);
    cudaError_t e = cudaMemsetAsync(q.s.bins, 0, (size_t)nbins * 4, q.stream);
    if (e != cudaSuccess) return e;
    spatial_count_kernel<<<blocks, 256, 0, q.stream>>>(q, bits);
    e = launch_exclusive_scan(q.s.bins, nbins, q.s.bin_sums, q.stream);
    if (e != cudaSuccess) return e;
    spatial_scatter_kernel<<<blocks, 256, 0, q.stream>>>(q, bits);
    *launches += 6;
    return cudaGetLastError();
  }
  scan_kernel<<<1, 1024, 0, q.stream>>>(q);
  const int nb = q.n_slots * kBuckets;
  if (nb <= 4096) {
    const int64_t blocks = (q.rays.n + 1023) / 1024;
    scatter_block_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 1024, 2 * nb * sizeof(int), q.stream>>>(q, nb);
  } else {
    const int grid = grid_for(q.rays.n, 256, 152 * 16);
    scatter_kernel<<<grid, 256, 0, q.stream>>>(q);
  }
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(int32_t *v, int64_t n, int32_t *sums, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + 1023) / 1024;
  scan_block_kernel<<<(unsigned)nb, 1024, 0, st>>>(v, n, sums);
  scan_sums_kernel<<<1, 1024, 0, st>>>(sums, (int)nb);
  scan_add_kernel<<<(unsigned)nb, 1024, 0, st>>>(v, n, sums);
  return cudaGetLastError();
}

cudaError_t launch_plain_tail(const QueryLaunch &q, int ldx, int chunk_tiles, int *launches) {
  const size_t smem = mlp_fp32_smem(q.s.wmax);
  cudaError_t e = cudaFuncSetAttribute(mlp_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int t0 = 0; t0 < q.s.max_tiles; t0 += chunk_tiles) {
    const int nt = min(chunk_tiles, q.s.max_tiles - t0);
    const int64_t items = (int64_t)nt * kTileM * q.H_max;
    gather_fp32_kernel<<<grid_for(items, 256, 152 * 32), 256, 0, q.stream>>>(q, t0, nt, ldx);
    mlp_fp32_kernel<<<min(nt, 152 * 4), 256, smem, q.stream>>>(q, t0, nt, ldx);
    *launches += 2;
  }
  return cudaGetLastError();
}

// ---- stage entry points ----------------------------------------------------

__global__ void trace_only_kernel(const DevObject *dobj, RaysArg r, int32_t *kout, float *t01, float *pts,
                                  int32_t *vox, int *err) {
  const DevObject &ob = *dobj;
  const int H = ob.H, cap = H >> 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += (int64_t)gridDim.x * blockDim.x) {
    float3 o, d;
    int ea;
    float t0 = CUDART_NAN_F, t1 = CUDART_NAN_F;
    int k = 0;
    bool live = to_unit(ob, r.ox[i], r.oy[i], r.oz[i], r.dx[i], r.dy[i], r.dz[i], o, d) &&
                unit_slab(o, d, r.tmin[i], t0, t1, ea);
    if (live) {
      dda_walk(
          ob, o, d, t0, t1, ea, [&](uint32_t vid) { return occupied(ob.occ, vid); },
          [&](const Seg &sg) {
            float3 a = seg_point(o, d, sg.tin, sg.ain, sg.fin);
            float3 b = seg_point(o, d, sg.tout, sg.aout, sg.fout);
            if (pts) {
              float *w = pts + ((size_t)i * H + 2 * k) * 3;
              w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = b.x; w[4] = b.y; w[5] = b.z;
            }
            if (vox) vox[(size_t)i * cap + k] = (int32_t)sg.vid;
            ++k;
            return k < cap;
          });
    } else {
      t0 = t1 = CUDART_NAN_F;
    }
    if (vox)
      for (int j = k; j < cap; ++j) vox[(size_t)i * cap + j] = -1;
    if (kout) kout[i] = k;
    if (t01) { t01[2 * i] = t0; t01[2 * i + 1] = t1; }
  }
}

cudaError_t launch_trace_only(const DevObject *dobj, const RaysArg &rays, int32_t *k, float *t01, float *pts,
                              int32_t *vox, int *err, cudaStream_t st) {
  int grid = grid_for(rays.n, 256, 152 * 16);
  trace_only_kernel<<<grid, 256, 0, st>>>(dobj, rays, k, t01, pts, vox, err);
  return cudaGetLastError();
}

template <typename T, int F>
__global__ void encode_kernel(DevObject hob, const T *tab, const float *pts, int64_t n, float *feats) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float3 p = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    for (int l = 0; l < hob.L; ++l) {
      float f[F];
      encode_level<T, F>(tab + (size_t)l * (hob.mask + 1) * F, hob.mask, p, (float)hob.res[l], f);
      for (int j = 0; j < F; ++j) feats[(i * hob.L + l) * F + j] = f[j];
    }
  }
}

cudaError_t launch_encode(const DevObject *dobj, const DevObject &h, const float *pts, int64_t n, float *feats,
                          int precision, cudaStream_t st) {
  (void)dobj;
  int grid = grid_for(n, 256, 152 * 32);
  if (precision == LSNIF_FP32_PLAIN) {
    if (h.F == 2) encode_kernel<float, 2><<<grid, 256, 0, st>>>(h, h.tab32, pts, n, feats);
    else if (h.F == 4) encode_kernel<float, 4><<<grid, 256, 0, st>>>(h, h.tab32, pts, n, feats);
    else encode_kernel<float, 1><<<grid, 256, 0, st>>>(h, h.tab32, pts, n, feats);
  } else {
    const __half *t16 = reinterpret_cast<const __half *>(h.tab16);
    if (h.F == 2) encode_kernel<__half, 2><<<grid, 256, 0, st>>>(h, t16, pts, n, feats);
    else if (h.F == 4) encode_kernel<__half, 4><<<grid, 256, 0, st>>>(h, t16, pts, n, feats);
    else encode_kernel<__half, 1><<<grid, 256, 0, st>>>(h, t16, pts, n, feats);
  }
  return cudaGetLastError();
}

__global__ void corners_kernel(DevObject hob, const float *pts, int64_t n, uint32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float3 p = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    for (int l = 0; l < hob.L; ++l) {
      Cell c = lattice_cell(p, (float)hob.res[l]);
      for (int corner = 0; corner < 8; ++corner) {
        uint32_t x = c.cx + (corner & 1), y = c.cy + ((corner >> 1) & 1), z = c.cz + ((corner >> 2) & 1);
        out[(i * hob.L + l) * 8 + corner] = hash3(x, y, z) & hob.mask;
      }
    }
  }
}

cudaError_t launch_corners(const DevObject *dobj, const DevObject &h, const float *pts, int64_t n, uint32_t *out,
                           cudaStream_t st) {
  (void)dobj;
  int grid = grid_for(n, 256, 152 * 32);
  corners_kernel<<<grid, 256, 0, st>>>(h, pts, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_plain(const DevObject *dobj, const DevObject &h, const float *X, int64_t n, float *Z,
                             cudaStream_t st) {
  const int wmax = max(h.width, h.n_out_pad);
  const size_t smem = mlp_fp32_smem(wmax);
  cudaError_t e = cudaFuncSetAttribute(mlp_fp32_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_fp32_rows_kernel<<<grid_for(n, kMT, 152 * 4), 256, smem, st>>>(dobj, X, n, Z, wmax);
  return cudaGetLastError();
}

// ---- object preparation -----------------------------------------------------

__global__ void to_half_kernel(const float *src, __half *dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2half_rn(src[i]);
}

cudaError_t launch_tables_to_half(const float *src, uint16_t *dst, int64_t n, cudaStream_t st) {
  to_half_kernel<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(src, reinterpret_cast<__half *>(dst), n);
  return cudaGetLastError();
}

// BF16 (dst) and FP16 (dst16) weights in the tcgen05 no-swizzle K-major
// core-matrix layout: element (n, k) of a layer with K inputs sits at byte
//   ((n/8)*(K/8) + k/8)*128 + (n%8)*16 + (k%8)*2
// Rows past the real output count are zero. Biases follow as FP32 in both.
// FP16 weights saturate at +-65504.
__global__ void build_umma_kernel(DevObject h, uint8_t *dst, uint8_t *dst16, uint8_t *dst_lo, uint8_t *dst_w0c) {
  const float *p = h.mlp32;
  uint32_t off = 0;
  const uint32_t off1 = (uint32_t)h.width * h.n_in * 2;  // where the layers after the first start
  int n_layers = h.n_hidden + 1;
  for (int l = 0; l < n_layers; ++l) {
    int K = l == 0 ? h.n_in : h.width;
    int Nr = l < h.n_hidden ? h.width : h.n_out;
    int Np = l < h.n_hidden ? h.width : h.n_out_pad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Np * K;
         e += (int64_t)gridDim.x * blockDim.x) {
      int nn = (int)(e / K), kk = (int)(e % K);
      float v = nn < Nr ? p[(int64_t)nn * K + kk] : 0.f;
      size_t o = off + ((size_t)(nn / 8) * (K / 8) + kk / 8) * 128 + (nn % 8) * 16 + (kk % 8) * 2;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      *reinterpret_cast<__nv_bfloat16 *>(dst + o) = hi;
      *reinterpret_cast<__half *>(dst16 + o) = __float2half_rn(fminf(fmaxf(v, -65504.f), 65504.f));
      if (l > 0) *reinterpret_cast<__nv_bfloat16 *>(dst_lo + (o - off1)) = __float2bfloat16_rn(v - __bfloat162float(hi));
      if (l == 0) {  // chunk-major copy: chunk s = kk / CHK is one contiguous W x CHK slice
        const int chk = 2 * h.L * h.F, s = kk / chk, c = kk % chk;
        const size_t oc = (size_t)s * h.width * chk * 2 + ((size_t)(nn / 8) * (chk / 8) + c / 8) * 128 + (nn % 8) * 16 +
                          (c % 8) * 2;
        *reinterpret_cast<__half *>(dst_w0c + oc) = __float2half_rn(fminf(fmaxf(v, -65504.f), 65504.f));
      }
    }
    const float *b = p + (size_t)Nr * K;
    float *bd = reinterpret_cast<float *>(dst + h.umma_bias_off) + (size_t)l * h.width;
    float *bd16 = reinterpret_cast<float *>(dst16 + h.umma_bias_off) + (size_t)l * h.width;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Np; j += gridDim.x * blockDim.x)
      bd[j] = bd16[j] = j < Nr ? b[j] : 0.f;
    off += (uint32_t)Np * K * 2;
    p += (size_t)Nr * K + Nr;
  }
}

// FP32 output layer padded with zero rows to n_out_pad (plain SIMT path).
__global__ void build_plain_out_kernel(DevObject h, float *dst) {
  const float *p = h.mlp32;
  int fan_in = h.n_in;
  for (int l = 0; l < h.n_hidden; ++l) {
    p += (size_t)h.width * fan_in + h.width;
    fan_in = h.width;
  }
  const float *b = p + (size_t)h.n_out * h.width;
  const int tot = h.n_out_pad * h.width;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot + h.n_out_pad; i += gridDim.x * blockDim.x) {
    if (i < tot) {
      const int r = i / h.width;
      dst[i] = r < h.n_out ? p[i] : 0.f;
    } else {
      const int j = i - tot;
      dst[i] = j < h.n_out ? b[j] : 0.f;
    }
  }
}

cudaError_t launch_build_umma(const DevObject &h, cudaStream_t st) {
  build_umma_kernel<<<152, 256, 0, st>>>(h, const_cast<uint8_t *>(h.umma), const_cast<uint8_t *>(h.umma_h),
                                         const_cast<uint8_t *>(h.umma_lo), const_cast<uint8_t *>(h.w0_16c));
  build_plain_out_kernel<<<16, 256, 0, st>>>(h, const_cast<float *>(h.plain_out));
  return cudaGetLastError();
}

}  // namespace lsnif
