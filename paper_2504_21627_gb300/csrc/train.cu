// Training on the GPU (Sec. 5.2, 5.3): balanced training rays, ground-truth
// labels by ray casting, and one optimisation step of the whole object --
// forward with saved activations, the multi-head loss, backward through the
// network, scatter of the feature gradients into the hash tables, Adam.
// Gradients are accumulated in FP32 (as in the paper). The network's dense
// products run on the tensor cores (train_gemm.cu: two-term BF16 operands,
// FP32 accumulation), or, for reference, as the FP32 SIMT GEMM below.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "device.cuh"
#include "encode.cuh"

namespace lsnif {

namespace {

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---------------------------------------------------------------------------
// ground truth: nearest triangle hit, walking the occupancy grid and testing
// the triangles listed for each occupied voxel (Moller-Trumbore, FP32)
// ---------------------------------------------------------------------------
struct Hit {
  float t, u, v;
  int32_t tri;
};

__device__ __forceinline__ bool mt_hit(const DevObject &ob, int32_t tri, const float o[3], const float d[3],
                                       float tmin, float tmax, float &t, float &u, float &v) {
  const int32_t *ix = ob.tris + 3 * (int64_t)tri;
  const float *a = ob.verts + 3 * (int64_t)ix[0];
  const float *b = ob.verts + 3 * (int64_t)ix[1];
  const float *c = ob.verts + 3 * (int64_t)ix[2];
  float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  float e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  float s[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
  float p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
  float det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
  if (det == 0.f) return false;
  float inv = 1.f / det;
  u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
  if (u < 0.f || u > 1.f) return false;
  float q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
  v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
  if (v < 0.f || u + v > 1.f) return false;
  t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
  return t >= tmin && t <= tmax;
}

__device__ Hit cast_ray(const DevObject &ob, float ox, float oy, float oz, float dx, float dy, float dz, float tmin,
                        float tmax) {
  Hit best{CUDART_INF_F, 0.f, 0.f, -1};
  float3 o3, d3;
  float t0, t1;
  int ea;
  if (!to_unit(ob, ox, oy, oz, dx, dy, dz, o3, d3) || !unit_slab(o3, d3, tmin, t0, t1, ea)) return best;
  const float o[3] = {ox, oy, oz}, d[3] = {dx, dy, dz};
  dda_walk(
      ob, o3, d3, t0, t1, ea, [&](uint32_t vid) { return occupied(ob.occ, vid); },
      [&](const Seg &sg) {
        const int32_t b = ob.vox_start[sg.vid], e = ob.vox_start[sg.vid + 1];
        for (int32_t j = b; j < e; ++j) {
          const int32_t tri = ob.vox_tris[j];
          float t, u, v;
          if (mt_hit(ob, tri, o, d, tmin, tmax, t, u, v) && (t < best.t || (t == best.t && tri < best.tri))) {
            best = Hit{t, u, v, tri};
          }
        }
        // a hit inside this voxel's span cannot be beaten by later voxels
        const float slack = 1e-5f * fabsf(sg.tout) + 1e-7f;
        return !(best.tri >= 0 && best.t <= sg.tout + slack);
      });
  return best;
}

__device__ __forceinline__ void sphere_point(float u0, float u1, float &x, float &y, float &z) {
  z = 1.f - 2.f * u0;
  const float r = sqrtf(fmaxf(0.f, 1.f - z * z));
  float s, c;
  sincospif(2.f * u1, &s, &c);
  x = r * c;
  y = r * s;
}

// cosine-weighted direction about unit n (basis of Duff et al. 2017)
__device__ __forceinline__ void cosine_dir(float nx, float ny, float nz, float u0, float u1, float &dx, float &dy,
                                           float &dz) {
  const float r = sqrtf(u0);
  float s, c;
  sincospif(2.f * u1, &s, &c);
  const float lx = r * c, ly = r * s, lz = sqrtf(fmaxf(0.f, 1.f - u0));
  const float sg = nz >= 0.f ? 1.f : -1.f;
  const float a = -1.f / (sg + nz);
  const float bb = nx * ny * a;
  const float tx = 1.f + sg * nx * nx * a, ty = sg * bb, tz = -sg * nx;
  const float bx = bb, by = sg + ny * ny * a, bz = -ny;
  dx = lx * tx + ly * bx + lz * nx;
  dy = lx * ty + ly * by + lz * ny;
  dz = lx * tz + ly * bz + lz * nz;
}

__global__ void make_rays_kernel(const DevObject *dobj, const float *u, int64_t n, int64_t n_outside, float *out,
                                 uint8_t *surface) {
  const DevObject &ob = *dobj;
  float lo[3], hi[3], c[3];
  float diag2 = 0.f;
  for (int a = 0; a < 3; ++a) {
    lo[a] = ob.bmin[a];
    hi[a] = ob.bmin[a] + 1.f / ob.inv_ext[a];
    c[a] = 0.5f * (lo[a] + hi[a]);
    diag2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
  }
  const float diag = sqrtf(diag2), R = 1.05f * 0.5f * diag;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float *ui = u + i * LSNIF_TRAIN_UNIFORMS;
    auto outside = [&](const float *uu, float *o, float *d) {
      float x, y, z;
      sphere_point(uu[0], uu[1], x, y, z);
      o[0] = c[0] + R * x;
      o[1] = c[1] + R * y;
      o[2] = c[2] + R * z;
      float w[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
      const float inv = rsqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
      cosine_dir(w[0] * inv, w[1] * inv, w[2] * inv, uu[2], uu[3], d[0], d[1], d[2]);
    };
    float o[3], d[3];
    outside(ui, o, d);
    uint8_t surf = 0;
    if (i >= n_outside) {
      for (int a = 0; a < 8; ++a) {
        float oa[3], da[3];
        outside(ui + 4 + 4 * a, oa, da);
        Hit h = cast_ray(ob, oa[0], oa[1], oa[2], da[0], da[1], da[2], 0.f, CUDART_INF_F);
        if (h.tri < 0) continue;
        const int32_t *ix = ob.tris + 3 * (int64_t)h.tri;
        const float *A = ob.verts + 3 * (int64_t)ix[0], *B = ob.verts + 3 * (int64_t)ix[1],
                    *C = ob.verts + 3 * (int64_t)ix[2];
        float e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        float g[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const float gi = rsqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        g[0] *= gi; g[1] *= gi; g[2] *= gi;
        float side = g[0] * da[0] + g[1] * da[1] + g[2] * da[2];
        const float sgn = side > 0.f ? -1.f : 1.f;  // normal facing the incoming ray
        const float nf[3] = {sgn * g[0], sgn * g[1], sgn * g[2]};
        for (int k = 0; k < 3; ++k) o[k] = oa[k] + h.t * da[k] + 1e-4f * diag * nf[k];
        cosine_dir(nf[0], nf[1], nf[2], ui[36], ui[37], d[0], d[1], d[2]);
        surf = 1;
        break;
      }
    }
    for (int k = 0; k < 3; ++k) {
      out[k * n + i] = o[k];
      out[(3 + k) * n + i] = d[k];
    }
    out[6 * n + i] = 0.f;
    out[7 * n + i] = CUDART_INF_F;
    if (surface) surface[i] = surf;
  }
}

__global__ void label_kernel(const DevObject *dobj, RaysArg r, lsnif_labels L) {
  const DevObject &ob = *dobj;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float tmin = r.tmin[i], tmax = r.tmax[i];
    Hit h = cast_ray(ob, r.ox[i], r.oy[i], r.oz[i], r.dx[i], r.dy[i], r.dz[i], tmin, tmax);
    float3 o3, d3;
    float t0 = 0.f, t1 = 1.f;
    int ea;
    bool live = to_unit(ob, r.ox[i], r.oy[i], r.oz[i], r.dx[i], r.dy[i], r.dz[i], o3, d3) &&
                unit_slab(o3, d3, tmin, t0, t1, ea);
    int k = 0;
    if (live && L.k) {
      const int cap = ob.H >> 1;
      dda_walk(
          ob, o3, d3, t0, t1, ea, [&](uint32_t vid) { return occupied(ob.occ, vid); },
          [&](const Seg &) { return ++k < cap; });
    }
    const bool occ = h.tri >= 0;
    float n3[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
    int32_t mat = 0;
    if (occ) {
      const int32_t *ix = ob.tris + 3 * (int64_t)h.tri;
      const float w0 = 1.f - h.u - h.v;
      for (int a = 0; a < 3; ++a)
        n3[a] = w0 * ob.vnormals[3 * ix[0] + a] + h.u * ob.vnormals[3 * ix[1] + a] + h.v * ob.vnormals[3 * ix[2] + a];
      const float nn = sqrtf(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2]);
      if (nn > 0.f) for (int a = 0; a < 3; ++a) n3[a] /= nn;
      mat = ob.tri_mat[h.tri];
      for (int a = 0; a < 3; ++a) al[a] = ob.albedo[3 * mat + a];
    }
    if (L.occ) L.occ[i] = occ ? 1.f : 0.f;
    if (L.t_local) L.t_local[i] = (occ && live) ? (h.t - t0) / (t1 - t0) : 0.f;
    if (L.normal) for (int a = 0; a < 3; ++a) L.normal[3 * i + a] = n3[a];
    if (L.albedo) for (int a = 0; a < 3; ++a) L.albedo[3 * i + a] = al[a];
    if (L.mat) L.mat[i] = mat;
    if (L.t_hit) L.t_hit[i] = h.t;
    if (L.tri) L.tri[i] = h.tri;
    if (L.k) L.k[i] = k;
  }
}

// ---------------------------------------------------------------------------
// forward features of the batch (FP32 tables), one thread per (ray, point,
// level): consecutive threads write consecutive levels of a point, and the
// corner loads of all levels are in flight together. Rows of rays that meet
// no occupied voxel stay zero.
// ---------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void feature_level(const DevObject &ob, int l, const float3 &p, float *xo) {
  const float *tl = ob.tab32 + (size_t)l * (ob.mask + 1) * F;
  float f[F];
  if constexpr (F == 2) encode_level_f32x2(tl, ob.mask, p, (float)ob.res[l], f);
  else encode_level<float, F>(tl, ob.mask, p, (float)ob.res[l], f);
#pragma unroll
  for (int j = 0; j < F; ++j) xo[j] = f[j];
}

// (ray i, point h, level l) of work item e = (i H + h) L + l, with 32-bit
// divisions when every item index fits 32 bits (a 64-bit integer division
// costs several times the instructions of a 32-bit one)
__device__ __forceinline__ void split_item(int64_t e, bool narrow, int H, int L, int64_t &i, int &h, int &l) {
  if (narrow) {
    const uint32_t u = (uint32_t)e, ih = u / (uint32_t)L, i32 = ih / (uint32_t)H;
    l = (int)(u - ih * (uint32_t)L);
    h = (int)(ih - i32 * (uint32_t)H);
    i = i32;
  } else {
    const int64_t ih = e / L;
    l = (int)(e - ih * L);
    i = ih / H;
    h = (int)(ih - i * H);
  }
}

__global__ void train_features_kernel(const DevObject *dobj, int64_t B, const int32_t *k, const float *pts,
                                      float *X) {
  const DevObject &ob = *dobj;
  const int H = ob.H, L = ob.L, F = ob.F;
  const int64_t tot = B * H * L;
  const bool narrow = tot + (int64_t)gridDim.x * blockDim.x < (int64_t(1) << 32);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    int h, l;
    split_item(e, narrow, H, L, i, h, l);
    float *xo = X + i * ob.n_in + ((size_t)h * L + l) * F;
    if (h >= 2 * k[i]) {
      for (int j = 0; j < F; ++j) xo[j] = 0.f;
      continue;
    }
    const float *pp = pts + (i * H + h) * 3;
    const float3 p = make_float3(pp[0], pp[1], pp[2]);
    if (F == 2) feature_level<2>(ob, l, p, xo);
    else if (F == 4) feature_level<4>(ob, l, p, xo);
    else feature_level<1>(ob, l, p, xo);
  }
}

// Scatter dX (B x n_in) into the table gradients, live points only. An entry
// point bit-identical to the previous segment's exit point (consecutive
// occupied voxels share a face) has the same corners and weights: its
// gradient is added to the exit point's before one set of reductions.
__global__ void train_scatter_kernel(const DevObject *dobj, int64_t B, const int32_t *k, const float *pts,
                                     const float *dX, float *gtab) {
  const DevObject &ob = *dobj;
  const int H = ob.H, L = ob.L, F = ob.F;
  const int64_t tot = B * H * L;
  const bool narrow = tot + (int64_t)gridDim.x * blockDim.x < (int64_t(1) << 32);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    int h, l;
    split_item(e, narrow, H, L, i, h, l);
    const int n_pts = 2 * k[i];
    if (h >= n_pts) continue;
    const float *pp = pts + (i * H + h) * 3;
    const float3 p = make_float3(pp[0], pp[1], pp[2]);
    // an entry point (even h > 0) equal to the exit point before it is scattered by that point's thread
    if (h > 0 && (h & 1) == 0 && pp[-3] == p.x && pp[-2] == p.y && pp[-1] == p.z) continue;
    const float *g = dX + i * ob.n_in + ((size_t)h * L + l) * F;
    float gs[4] = {0.f, 0.f, 0.f, 0.f};
    for (int f = 0; f < F; ++f) gs[f] = g[f];
    if ((h & 1) == 1 && h + 1 < n_pts && pp[3] == p.x && pp[4] == p.y && pp[5] == p.z) {
      const float *g2 = g + (size_t)L * F;  // the next point's features, same level
      for (int f = 0; f < F; ++f) gs[f] += g2[f];
    }
    encode_level_backward(gtab + (size_t)l * (ob.mask + 1) * F, ob.mask, p, (float)ob.res[l], gs, F);
  }
}

// ---------------------------------------------------------------------------
// FP32 SIMT GEMM: C[M x N] = op(A)[M x K] . op(B)[K x N], row-major,
// op(A)[m][k] = tA ? A[k*lda+m] : A[m*lda+k], op(B)[k][n] = tB ? B[n*ldb+k] : B[k*ldb+n].
// mode 0: store; 1: atomicAdd (split K); 2: + bias[n], store pre and act(pre);
// 3: + bias[n], store; 4: multiply by act'(aux[m][n]) and store.
// ---------------------------------------------------------------------------
constexpr int GB = 64, GK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *A, int lda, int tA,
                                                   const float *Bm, int ldb, int tB, float *C, int ldc, int mode,
                                                   const float *bias, float *post, const float *aux, int act,
                                                   int k_split) {
  __shared__ float As[GK][GB + 4];
  __shared__ float Bs[GK][GB + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GB, n0 = blockIdx.x * GB;
  const int kz = blockIdx.z;
  const int kb = (int)((int64_t)K * kz / k_split), ke = (int)((int64_t)K * (kz + 1) / k_split);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += GK) {
    for (int e = threadIdx.x; e < GB * GK; e += 256) {
      int mm, kk;
      if (tA) { mm = e % GB; kk = e / GB; } else { kk = e % GK; mm = e / GK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < ke) v = tA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
      int nn, kk2;
      if (tB) { kk2 = e % GK; nn = e / GK; } else { nn = e % GB; kk2 = e / GB; }
      const int gn = n0 + nn, gk2 = k0 + kk2;
      float w = 0.f;
      if (gn < N && gk2 < ke) w = tB ? Bm[(int64_t)gn * ldb + gk2] : Bm[(int64_t)gk2 * ldb + gn];
      Bs[kk2][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      const int64_t o = (int64_t)gm * ldc + gn;
      float v = acc[i][j];
      if (mode == 0) C[o] = v;
      else if (mode == 1) atomicAdd(C + o, v);
      else if (mode == 2) { v += bias[gn]; C[o] = v; post[o] = act_fn(v, act); }
      else if (mode == 3) C[o] = v + bias[gn];
      else C[o] = v * act_grad(aux[o], act);
    }
  }
}

void gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, int tA, const float *B, int ldb, int tB,
          float *C, int ldc, int mode, const float *bias = nullptr, float *post = nullptr, const float *aux = nullptr,
          int act = 0, int k_split = 1) {
  dim3 grid((N + GB - 1) / GB, (M + GB - 1) / GB, k_split);
  gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, mode, bias, post, aux, act, k_split);
}

// column sums of G (rows x cols, cols <= 256) added into out (bias
// gradients). The block is a whole number of rows wide (blockDim = cols x
// rows per sweep), so a thread keeps one column and the block's reads of a
// sweep are one contiguous run; per-thread sums, then per-column sums of
// the block, then one atomic per column and block.
__global__ void colsum_kernel(const float *G, int64_t rows, int cols, float *out) {
  extern __shared__ float part[];
  const int per = blockDim.x / cols;
  const int c = threadIdx.x % cols, rr = threadIdx.x / cols;
  float acc = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * per + rr; r < rows; r += (int64_t)gridDim.x * per) acc += G[r * cols + c];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < cols) {
    float s = 0.f;
    for (int j = 0; j < per; ++j) s += part[j * cols + threadIdx.x];
    atomicAdd(out + threadIdx.x, s);
  }
}

// loss terms and dLoss/dZ for the batch mean over rays that reach the
// network; sums into acc[0..5] = total, occ, t, normal, albedo, mat and
// acc[6] = live count (computed beforehand)
__global__ void loss_kernel(const DevObject *dobj, int64_t B, const int32_t *k, const float *Z, lsnif_labels lab,
                            float *dZ, float *acc, const float *live_count) {
  const DevObject &ob = *dobj;
  const int n_out = ob.n_out;
  const float inv_live = 1.f / fmaxf(*live_count, 1.f);
  float s[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    const float *z = Z + i * n_out;
    float *g = dZ + i * n_out;
    if (k[i] == 0) {
      for (int j = 0; j < n_out; ++j) g[j] = 0.f;
      continue;
    }
    const float y = lab.occ[i];
    const float z0 = z[0];
    const float l_occ = fmaxf(z0, 0.f) - z0 * y + log1pf(expf(-fabsf(z0)));
    g[0] = (sigmoidf_(z0) - y) * inv_live;
    // remaining heads only where the reference is occluded
    const float s1 = sigmoidf_(z[1]);
    const float dt = s1 - lab.t_local[i];
    const float l_t = fabsf(dt);
    const float g1 = (dt > 0.f ? 1.f : (dt < 0.f ? -1.f : 0.f)) * s1 * (1.f - s1);
    const float zn[3] = {z[2], z[3], z[4]};
    const float *yn = lab.normal + 3 * i;
    const float nz = fmaxf(sqrtf(zn[0] * zn[0] + zn[1] * zn[1] + zn[2] * zn[2]), 1e-12f);
    const float dot = zn[0] * yn[0] + zn[1] * yn[1] + zn[2] * yn[2];
    const float l_n = 1.f - dot / nz;
    float gn[3];
    for (int a = 0; a < 3; ++a) gn[a] = -(yn[a] / nz - dot * zn[a] / (nz * nz * nz));
    float l_a = 0.f, ga[3];
    for (int c = 0; c < 3; ++c) {
      const float sa = sigmoidf_(z[5 + c]);
      const float den = sa * sa + 0.01f;
      const float df = sa - lab.albedo[3 * i + c];
      l_a += df * df / den;
      ga[c] = (2.f / 3.f) * df / den * sa * (1.f - sa);
    }
    l_a *= (1.f / 3.f);
    float mx = z[8];
    for (int m = 1; m < ob.n_mat; ++m) mx = fmaxf(mx, z[8 + m]);
    float se = 0.f;
    for (int m = 0; m < ob.n_mat; ++m) se += expf(z[8 + m] - mx);
    const int ym = lab.mat[i];
    const float l_m = mx + logf(se) - z[8 + ym];
    g[1] = y * g1 * inv_live;
    for (int a = 0; a < 3; ++a) g[2 + a] = y * gn[a] * inv_live;
    for (int c = 0; c < 3; ++c) g[5 + c] = y * ga[c] * inv_live;
    for (int m = 0; m < ob.n_mat; ++m) g[8 + m] = y * (expf(z[8 + m] - mx) / se - (m == ym ? 1.f : 0.f)) * inv_live;
    s[1] += l_occ;
    s[2] += y * l_t;
    s[3] += y * l_n;
    s[4] += y * l_a;
    s[5] += y * l_m;
  }
  s[0] = s[1] + s[2] + s[3] + s[4] + s[5];
  // warp sums, then block sums, then one atomic per block and term (six
  // addresses take every block's atomic, so fewer of them contend less)
  __shared__ float part[6][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < 6; ++j) {
    float v = s[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) part[j][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < 6; ++j) {
      float v = lane < nw ? part[j][lane] : 0.f;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) atomicAdd(acc + j, v * inv_live);
    }
  }
}

// k = k8 (the traversal's one-byte point counts), and the live-ray count
__global__ void widen_count_kernel(const uint8_t *k8, int64_t B, int32_t *k, float *count) {
  float c = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ki = k8[i];
    k[i] = ki;
    c += ki > 0 ? 1.f : 0.f;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(count, c);
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

cudaError_t launch_make_training_rays(const DevObject *dobj, const DevObject &h, const float *u, int64_t n,
                                      int64_t n_outside, float *rays_out, uint8_t *surface, cudaStream_t st) {
  if (!h.vox_start) return cudaErrorNotSupported;
  make_rays_kernel<<<grid_for(n, 128, 152 * 16), 128, 0, st>>>(dobj, u, n, n_outside, rays_out, surface);
  return cudaGetLastError();
}

cudaError_t launch_label_rays(const DevObject *dobj, const DevObject &h, const RaysArg &rays, const lsnif_labels &out,
                              cudaStream_t st) {
  if (!h.vox_start) return cudaErrorNotSupported;
  label_kernel<<<grid_for(rays.n, 128, 152 * 16), 128, 0, st>>>(dobj, rays, out);
  return cudaGetLastError();
}

cudaError_t launch_train_step(const DevObject *objs, int n_slots, const DevObject *dobj, const DevObject &h,
                              const RaysArg &rays, const lsnif_labels &lab, const lsnif_train_opts &opts,
                              int64_t step, TrainBuffers &tb, int64_t n_params_mlp, int *err, cudaStream_t st) {
  const bool tc = opts.products == LSNIF_TRAIN_TENSOR_CORES;
  cudaError_t ge = cudaSuccess;  // first failed product launch
  auto mm = [&](int M, int N, int K, const float *A, int lda, int tA, const float *Bm, int ldb, int tB, float *C,
                int ldc, int mode, const float *bias = nullptr, float *post = nullptr, const float *aux = nullptr,
                int act = 0, int k_split = 1) {
    if (tc) {
      const cudaError_t e2 = launch_tc_gemm(st, M, N, K, A, lda, tA, Bm, ldb, tB, C, ldc, mode, bias, post, aux, act,
                                            k_split, err);
      if (ge == cudaSuccess) ge = e2;
    } else {
      gemm(st, M, N, K, A, lda, tA, Bm, ldb, tB, C, ldc, mode, bias, post, aux, act, k_split);
    }
  };
  const int64_t B = rays.n;
  const int W = h.width, NI = h.n_in, NO = h.n_out, NH = h.n_hidden;
  const size_t ntab = ((size_t)h.L << h.log2T) * h.F;
  cudaMemsetAsync(tb.loss, 0, 8 * sizeof(float), st);
  cudaMemsetAsync(tb.grad_mlp, 0, sizeof(float) * n_params_mlp, st);
  cudaMemsetAsync(tb.grad_tab, 0, sizeof(float) * ntab, st);
  // a1-a5 for the batch: the query's persistent-lane traversal with empty
  // cube skipping (the voxels and boundary points of the voxel-by-voxel
  // walk, bit for bit), no results written
  QueryLaunch q{};
  q.objs = objs;
  q.n_slots = n_slots;
  q.H_max = h.H;
  q.rays = rays;
  q.s.pts = tb.pts;
  q.s.t01 = tb.t01;
  q.s.k = tb.k8;
  q.s.dup = tb.dup;
  q.s.slot = tb.slot;
  q.s.counts = tb.counts;
  q.s.meta = tb.meta;
  q.err = err;
  q.stream = st;
  q.trace_mode = 1;
  int launches = 0;
  cudaError_t e = launch_trace(q, &launches);
  if (e != cudaSuccess) return e;
  widen_count_kernel<<<grid_for(B, 256, 152 * 4), 256, 0, st>>>(tb.k8, B, tb.k, tb.loss + 6);
  train_features_kernel<<<grid_for(B * h.H * h.L, 256, 152 * 32), 256, 0, st>>>(dobj, B, tb.k, tb.pts, tb.feats);
  // forward: pre[l], acts[l] (B x W each), logits Z
  const float *p = h.mlp32;
  const float *Wl[LSNIF_MAX_HIDDEN + 1], *bl[LSNIF_MAX_HIDDEN + 1];
  int fan_in = NI;
  for (int l = 0; l <= NH; ++l) {
    const int fo = l < NH ? W : NO;
    Wl[l] = p;
    bl[l] = p + (size_t)fo * fan_in;
    p += (size_t)fo * fan_in + fo;
    fan_in = fo;
  }
  const float *in = tb.feats;
  int K = NI;
  for (int l = 0; l < NH; ++l) {
    float *pre = tb.pre + (size_t)l * B * W, *post = tb.acts + (size_t)l * B * W;
    mm((int)B, W, K, in, K, 0, Wl[l], K, 1, pre, W, 2, bl[l], post, nullptr, h.act);
    in = post;
    K = W;
  }
  mm((int)B, NO, W, in, W, 0, Wl[NH], W, 1, tb.Z, NO, 3, bl[NH]);
  loss_kernel<<<grid_for(B, 256, 152 * 8), 256, 0, st>>>(dobj, B, tb.k, tb.Z, lab, tb.dZ, tb.loss, tb.loss + 6);
  // backward through the network; gradient layout mirrors the packed weights
  float *gW[LSNIF_MAX_HIDDEN + 1], *gb[LSNIF_MAX_HIDDEN + 1];
  {
    float *q = tb.grad_mlp;
    int fi = NI;
    for (int l = 0; l <= NH; ++l) {
      const int fo = l < NH ? W : NO;
      gW[l] = q;
      gb[l] = q + (size_t)fo * fi;
      q += (size_t)fo * fi + fo;
      fi = fo;
    }
  }
  const int ks = (int)std::min<int64_t>(256, std::max<int64_t>(1, B / 1024));
  const float *d = tb.dZ;  // gradient w.r.t. the current layer's output (pre-activation)
  int dcols = NO;
  for (int l = NH; l >= 0; --l) {
    const int fi = l == 0 ? NI : W;
    const float *hin = l == 0 ? tb.feats : tb.acts + (size_t)(l - 1) * B * W;
    // dW = d^T . hin  (dcols x fi), split over the batch
    mm(dcols, fi, (int)B, d, dcols, 1, hin, fi, 0, gW[l], fi, 1, nullptr, nullptr, nullptr, 0, ks);
    {
      const int threads = dcols * std::max(1, 256 / dcols);
      colsum_kernel<<<152 * 8, threads, threads * sizeof(float), st>>>(d, B, dcols, gb[l]);
    }
    // gradient w.r.t. the layer input: d . W_l (B x fi); for hidden inputs
    // multiply by act'(pre of layer l-1)
    float *dn = (l % 2 == 0) ? tb.dA : tb.dB;
    if (l > 0)
      mm((int)B, fi, dcols, d, dcols, 0, Wl[l], fi, 0, dn, fi, 4, nullptr, nullptr, tb.pre + (size_t)(l - 1) * B * W,
         h.act);
    else
      mm((int)B, fi, dcols, d, dcols, 0, Wl[l], fi, 0, dn, fi, 0);
    d = dn;
    dcols = fi;
  }
  // d is dX (B x n_in): scatter into the table gradients
  train_scatter_kernel<<<grid_for(B * h.H * h.L, 256, 152 * 32), 256, 0, st>>>(dobj, B, tb.k, tb.pts, d, tb.grad_tab);
  if (opts.apply_update) {
    const double c1 = 1.0 - std::pow((double)opts.beta1, (double)step);
    const double c2 = 1.0 - std::pow((double)opts.beta2, (double)step);
    adam_kernel<<<grid_for(n_params_mlp, 256, 152 * 8), 256, 0, st>>>(const_cast<float *>(h.mlp32), tb.grad_mlp,
                                                                       tb.m_mlp, tb.v_mlp, n_params_mlp, opts.lr,
                                                                       opts.beta1, opts.beta2, opts.eps, (float)c1,
                                                                       (float)c2);
    adam_kernel<<<grid_for((int64_t)ntab, 256, 152 * 16), 256, 0, st>>>(const_cast<float *>(h.tab32), tb.grad_tab,
                                                                         tb.m_tab, tb.v_tab, (int64_t)ntab, opts.lr,
                                                                         opts.beta1, opts.beta2, opts.eps, (float)c1,
                                                                         (float)c2);
  }
  if (ge != cudaSuccess) return ge;
  return cudaGetLastError();
}

}  // namespace lsnif
