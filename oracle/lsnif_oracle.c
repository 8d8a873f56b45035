/*
 * lsnif_oracle.c -- plain, slow FP64 CPU oracle for the LSNIF per-ray query
 * (Fujieda, Kao, Harada: "LSNIF: Locally-Subdivided Neural Intersection
 * Function", PACMCGIT 8(1), 2025).
 *
 * TEST INFRASTRUCTURE. This is the correctness reference the CUDA path is
 * checked against. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it. It shares no code, header or table with the
 * product library and is never linked into it.
 *
 * Every routine is written to be checked against the paper by eye:
 *   - occupancy: separating-axis triangle/closed-box test (Akenine-Moller,
 *     "Fast 3D triangle-box overlap testing", 2001) for every voxel whose box
 *     meets the triangle's bounding box (Sec. 3.1, surface-only voxelization);
 *   - traversal: every occupied voxel is slab-tested against the ray, hits of
 *     positive length are sorted by entry distance -- the brute-force
 *     definition of what the incremental 3D-DDA produces (Sec. 3.1, Fig. 2);
 *   - points: entry and exit of each occupied voxel on its boundary, capped at
 *     H points, remaining slots zero (Sec. 3.1, Sec. 5.1);
 *   - encoding: eight-corner trilinear interpolation of hashed lattice
 *     features on every level (Sec. 3.2, after instant-NGP);
 *   - judge: nearest Moller-Trumbore hit over all triangles (Sec. 5.2 uses
 *     ray casting for ground truth).
 *
 * All floating point is double unless a function says otherwise. Compile
 * with -ffp-contract=off so no fused multiply-add changes a rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------
 * Bounding box (Sec. 3.1: the object's AABB is its local frame).
 * The box of FP32 vertices is exact in FP32. An axis thinner than 1/8 of
 * the diagonal is widened symmetrically to that thickness, rounded outward
 * to FP32. The unit-cube map multiplies an axis by 1/extent, so a very thin
 * axis would magnify the rounding of FP32 ray origins along it into whole
 * voxels; at 1/8 of the diagonal it magnifies them at most 8 times as much
 * as the diagonal does.
 * ---------------------------------------------------------------------- */
ORC_API void orc_bbox(const float *verts, int64_t nv, float bmin[3], float bmax[3])
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = verts[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double diag = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                       (hi[2] - lo[2]) * (hi[2] - lo[2]));
    double emin = diag / 8.0;
    if (emin == 0.0) emin = 1e-6;
    for (int a = 0; a < 3; ++a) {
        if (hi[a] - lo[a] < emin) {
            double c = 0.5 * (lo[a] + hi[a]);
            lo[a] = c - 0.5 * emin;
            hi[a] = c + 0.5 * emin;
        }
        float fl = (float)lo[a], fh = (float)hi[a];
        if ((double)fl > lo[a]) fl = nextafterf(fl, -INFINITY);
        if ((double)fh < hi[a]) fh = nextafterf(fh, INFINITY);
        bmin[a] = fl;
        bmax[a] = fh;
    }
}

/* ------------------------------------------------------------------------
 * Voxelization (Sec. 3.1): binary occupancy of the V^3 grid over the AABB;
 * a voxel is occupied when some triangle overlaps its closed box.
 * Coordinates are scaled so voxel (i,j,k) is the box [i,i+1]x[j,j+1]x[k,k+1]:
 *   u = ((v - bmin) * V) / (bmax - bmin)     (this exact expression order)
 * Output occ[(z*V + y)*V + x] in {0,1}.
 * ---------------------------------------------------------------------- */

/* Separating-axis test of a triangle against the closed axis-aligned cube of
 * half-size h centred at c. Touching counts as overlap. */
static int tri_box_overlap(const double c[3], double h, const double u0[3], const double u1[3],
                           const double u2[3])
{
    double v[3][3], e[3][3];
    for (int a = 0; a < 3; ++a) {
        v[0][a] = u0[a] - c[a];
        v[1][a] = u1[a] - c[a];
        v[2][a] = u2[a] - c[a];
    }
    for (int a = 0; a < 3; ++a) {
        e[0][a] = v[1][a] - v[0][a];
        e[1][a] = v[2][a] - v[1][a];
        e[2][a] = v[0][a] - v[2][a];
    }
    /* nine axes: box axis j cross triangle edge i */
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double ax[3] = {0, 0, 0};
            /* unit_j x e_i */
            double uj[3] = {0, 0, 0};
            uj[j] = 1.0;
            ax[0] = uj[1] * e[i][2] - uj[2] * e[i][1];
            ax[1] = uj[2] * e[i][0] - uj[0] * e[i][2];
            ax[2] = uj[0] * e[i][1] - uj[1] * e[i][0];
            double p0 = ax[0] * v[0][0] + ax[1] * v[0][1] + ax[2] * v[0][2];
            double p1 = ax[0] * v[1][0] + ax[1] * v[1][1] + ax[2] * v[1][2];
            double p2 = ax[0] * v[2][0] + ax[1] * v[2][1] + ax[2] * v[2][2];
            double mn = fmin(p0, fmin(p1, p2)), mx = fmax(p0, fmax(p1, p2));
            double r = h * (fabs(ax[0]) + fabs(ax[1]) + fabs(ax[2]));
            if (mn > r || mx < -r) return 0;
        }
    }
    /* three box face normals */
    for (int a = 0; a < 3; ++a) {
        double mn = fmin(v[0][a], fmin(v[1][a], v[2][a]));
        double mx = fmax(v[0][a], fmax(v[1][a], v[2][a]));
        if (mn > h || mx < -h) return 0;
    }
    /* triangle plane */
    double n[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                   e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    double vmin[3], vmax[3];
    for (int a = 0; a < 3; ++a) {
        if (n[a] > 0.0) {
            vmin[a] = -h - v[0][a];
            vmax[a] = h - v[0][a];
        } else {
            vmin[a] = h - v[0][a];
            vmax[a] = -h - v[0][a];
        }
    }
    double dmin = n[0] * vmin[0] + n[1] * vmin[1] + n[2] * vmin[2];
    double dmax = n[0] * vmax[0] + n[1] * vmax[1] + n[2] * vmax[2];
    if (dmin > 0.0) return 0;
    if (dmax >= 0.0) return 1;
    return 0;
}

ORC_API int orc_tri_box_overlap(const double c[3], double h, const double u0[3],
                                const double u1[3], const double u2[3])
{
    return tri_box_overlap(c, h, u0, u1, u2);
}

static void to_grid(const float *p, const float bmin[3], const float bmax[3], int V, double u[3])
{
    for (int a = 0; a < 3; ++a)
        u[a] = (((double)p[a] - (double)bmin[a]) * (double)V) / ((double)bmax[a] - (double)bmin[a]);
}

ORC_API void orc_voxelize(const float *verts, const int32_t *tris, int64_t nt, const float bmin[3],
                          const float bmax[3], int V, uint8_t *occ)
{
    memset(occ, 0, (size_t)V * V * V);
    for (int64_t t = 0; t < nt; ++t) {
        double u[3][3];
        for (int c = 0; c < 3; ++c) to_grid(verts + 3 * (int64_t)tris[3 * t + c], bmin, bmax, V, u[c]);
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            double mn = fmin(u[0][a], fmin(u[1][a], u[2][a]));
            double mx = fmax(u[0][a], fmax(u[1][a], u[2][a]));
            /* closed boxes [i, i+1] touching [mn, mx]: i from ceil(mn)-1 to floor(mx) */
            lo[a] = (int)ceil(mn) - 1;
            hi[a] = (int)floor(mx);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > V - 1) hi[a] = V - 1;
        }
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    size_t id = ((size_t)z * V + y) * V + x;
                    if (occ[id]) continue;
                    double c[3] = {x + 0.5, y + 0.5, z + 0.5};
                    if (tri_box_overlap(c, 0.5, u[0], u[1], u[2])) occ[id] = 1;
                }
    }
}

/* ------------------------------------------------------------------------
 * Level resolutions (Sec. 3.2, geometric progression as in instant-NGP):
 *   b = exp((ln Nmax - ln Nmin) / (L - 1)),  N_l = floor(Nmin * b^l + 0.5)
 * ---------------------------------------------------------------------- */
ORC_API void orc_level_res(int Nmin, int Nmax, int L, int32_t *out)
{
    if (L == 1) {
        out[0] = Nmin;
        return;
    }
    double b = exp((log((double)Nmax) - log((double)Nmin)) / (double)(L - 1));
    for (int l = 0; l < L; ++l) out[l] = (int32_t)floor((double)Nmin * pow(b, (double)l) + 0.5);
}

/* ------------------------------------------------------------------------
 * Ray -> unit cube, slab tests, occupied-voxel segments and boundary points
 * (Fig. 2; Sec. 3.1; Sec. 5.1 for the cap H).
 *
 * Ray record (8 floats): ox oy oz dx dy dz tmin tmax, object space.
 * Unit cube: o' = (o - bmin)/(bmax - bmin), d' = d/(bmax - bmin); t unchanged.
 * [t0, t1]: t_near/t_far of the cube, t0 = max(t_near, tmin). tmax does not
 * clip the traversal (it only bounds the reported hit).
 * ---------------------------------------------------------------------- */

/* Slab test against [lo, hi]^3 componentwise. Returns 0 when a zero
 * direction component leaves the origin outside its slab. Otherwise sets
 * tn/tf and the axes that produced them (the lowest axis on ties). */
static int slab(const double o[3], const double d[3], const double lo[3], const double hi[3],
                double *tn, int *an, double *tf, int *af)
{
    double tnear = -INFINITY, tfar = INFINITY;
    int anear = -1, afar = -1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - o[a]) / d[a];
        double tb = (hi[a] - o[a]) / d[a];
        if (ta > tb) {
            double s = ta;
            ta = tb;
            tb = s;
        }
        if (ta > tnear) {
            tnear = ta;
            anear = a;
        }
        if (tb < tfar) {
            tfar = tb;
            afar = a;
        }
    }
    *tn = tnear;
    *an = anear;
    *tf = tfar;
    *af = afar;
    return 1;
}

typedef struct {
    double tin, tout;
    int ain, aout; /* boundary axis of entry/exit, -1 = interior (clipped by t0) */
    int32_t vox;
    int ix[3];
} seg_t;

static int seg_cmp(const void *pa, const void *pb)
{
    const seg_t *a = (const seg_t *)pa, *b = (const seg_t *)pb;
    if (a->tin < b->tin) return -1;
    if (a->tin > b->tin) return 1;
    if (a->tout < b->tout) return -1;
    if (a->tout > b->tout) return 1;
    return (a->vox > b->vox) - (a->vox < b->vox);
}

/* Overlap of the segment [t0, t1] of the ray with box [lo,hi]: 1 when it has
 * positive length; tin/tout the clipped interval. */
static int box_overlap(const double o[3], const double d[3], const double lo[3], const double hi[3],
                       double t0, double t1, double *tin, double *tout, int *ain, int *aout)
{
    double tn, tf;
    int an, af;
    if (!slab(o, d, lo, hi, &tn, &an, &tf, &af)) return 0;
    double a = tn, b = tf;
    int ea = an, eb = af;
    if (a < t0) {
        a = t0;
        ea = -1;
    }
    if (b > t1) b = t1;
    *tin = a;
    *tout = b;
    *ain = ea;
    *aout = eb;
    return b > a;
}

/*
 * Per ray: the ordered occupied-voxel segments and the H boundary points.
 *   occ_list: n_occ voxel ids (z*V+y)*V+x of occupied voxels
 *   out_k[i]      number of kept segments (<= H/2)
 *   out_t01[2i]   t0, t1 (NaN when the ray misses the cube)
 *   out_pts[i*H*3 ...] points in unit-cube coordinates, zero beyond 2k
 *   out_vox[i*(H/2) ...] voxel ids of kept segments, -1 beyond k
 *   out_flag[i]   1 when the ordered list is not robust to a perturbation of
 *                 `eps` (unit-cube units) of the voxel boxes (near-face ray)
 * Entry/exit points lie on the box face they cross: that coordinate is set
 * to exactly face/V, the other two are o' + t d'. A segment that starts at
 * t0 inside a voxel keeps its computed entry point.
 */
static void one_ray_segments(const float *r, const float bmin[3], const float bmax[3], int V,
                             const int32_t *occ_list, int64_t n_occ, int H, double eps, seg_t *segs,
                             double *unc_tin, int32_t *out_k, double *out_t01, double *out_pts,
                             int32_t *out_vox, uint8_t *out_flag)
{
    int cap = H / 2;
    double o[3], d[3], tmin = r[6];
    int bad = 0;
    for (int a = 0; a < 3; ++a) {
        double ext = (double)bmax[a] - (double)bmin[a];
        o[a] = ((double)r[a] - (double)bmin[a]) / ext;
        d[a] = (double)r[3 + a] / ext;
        if (isnan(o[a]) || isnan(d[a]) || isinf(o[a]) || isinf(d[a])) bad = 1;
    }
    if (isnan(tmin)) bad = 1;
    if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) bad = 1;
    *out_k = 0;
    *out_flag = 0;
    out_t01[0] = NAN;
    out_t01[1] = NAN;
    for (int h = 0; h < 3 * H; ++h) out_pts[h] = 0.0;
    for (int h = 0; h < cap; ++h) out_vox[h] = -1;
    if (bad) return;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, tn, tf;
    int an, af;
    if (!slab(o, d, lo, hi, &tn, &an, &tf, &af)) return;
    double t0 = tn > tmin ? tn : tmin, t1 = tf;
    if (!(t1 > t0)) return;
    out_t01[0] = t0;
    out_t01[1] = t1;
    /* brute force: every occupied voxel */
    int64_t ns = 0, nu = 0;
    for (int64_t q = 0; q < n_occ; ++q) {
        int32_t id = occ_list[q];
        int ix[3] = {id % V, (id / V) % V, id / (V * V)};
        double blo[3], bhi[3], tin, tout;
        int ain, aout;
        for (int a = 0; a < 3; ++a) {
            blo[a] = (double)ix[a] / V;
            bhi[a] = (double)(ix[a] + 1) / V;
        }
        int hit = box_overlap(o, d, blo, bhi, t0, t1, &tin, &tout, &ain, &aout);
        /* robustness: the box shrunk and grown by eps on every side */
        double slo[3], shi[3], glo[3], ghi[3], a1, b1, gin, gout;
        int c1, c2;
        for (int a = 0; a < 3; ++a) {
            slo[a] = blo[a] + eps;
            shi[a] = bhi[a] - eps;
            glo[a] = blo[a] - eps;
            ghi[a] = bhi[a] + eps;
        }
        int in_shrunk = box_overlap(o, d, slo, shi, t0, t1, &a1, &b1, &c1, &c2);
        int in_grown = box_overlap(o, d, glo, ghi, t0, t1, &gin, &gout, &c1, &c2);
        if (in_grown && !in_shrunk) unc_tin[nu++] = gin;
        if (hit) {
            seg_t *g = &segs[ns++];
            g->tin = tin;
            g->tout = tout;
            g->ain = ain;
            g->aout = aout;
            g->vox = id;
            g->ix[0] = ix[0];
            g->ix[1] = ix[1];
            g->ix[2] = ix[2];
        }
    }
    qsort(segs, (size_t)ns, sizeof(seg_t), seg_cmp);
    int k = ns < cap ? (int)ns : cap;
    *out_k = k;
    for (int s = 0; s < k; ++s) {
        const seg_t *g = &segs[s];
        double *p0 = out_pts + (2 * s) * 3;
        double *p1 = p0 + 3;
        for (int a = 0; a < 3; ++a) {
            p0[a] = o[a] + g->tin * d[a];
            p1[a] = o[a] + g->tout * d[a];
        }
        if (g->ain >= 0) {
            int a = g->ain;
            p0[a] = (double)(d[a] > 0 ? g->ix[a] : g->ix[a] + 1) / V;
        }
        if (g->aout >= 0) {
            int a = g->aout;
            p1[a] = (double)(d[a] > 0 ? g->ix[a] + 1 : g->ix[a]) / V;
        }
        out_vox[s] = g->vox;
    }
    /* near-face ray: an uncertain voxel could enter the kept prefix */
    double t_last = (ns >= cap && cap > 0) ? segs[cap - 1].tout : INFINITY;
    for (int64_t q = 0; q < nu; ++q)
        if (unc_tin[q] <= t_last) *out_flag = 1;
}

ORC_API void orc_ray_segments(const float *rays, int64_t n, const float bmin[3], const float bmax[3],
                              int V, const int32_t *occ_list, int64_t n_occ, int H, double eps,
                              int32_t *out_k, double *out_t01, double *out_pts, int32_t *out_vox,
                              uint8_t *out_flag)
{
#pragma omp parallel
    {
        seg_t *segs = (seg_t *)malloc(sizeof(seg_t) * (size_t)(n_occ > 0 ? n_occ : 1));
        double *unc = (double *)malloc(sizeof(double) * (size_t)(n_occ > 0 ? n_occ : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i)
            one_ray_segments(rays + 8 * i, bmin, bmax, V, occ_list, n_occ, H, eps, segs, unc,
                             out_k + i, out_t01 + 2 * i, out_pts + (size_t)i * H * 3,
                             out_vox + (size_t)i * (H / 2), out_flag + i);
        free(segs);
        free(unc);
    }
}

/* ------------------------------------------------------------------------
 * Hash grid (Sec. 3.2; spatial hash of Teschner et al. as used by
 * instant-NGP): h = (x*1) xor (y*2654435761) xor (z*805459861) mod 2^32,
 * index = h & (T - 1).
 * ---------------------------------------------------------------------- */
ORC_API uint32_t orc_hash(int64_t x, int64_t y, int64_t z, int log2T)
{
    uint32_t hx = (uint32_t)x * 1u;
    uint32_t hy = (uint32_t)y * 2654435761u;
    uint32_t hz = (uint32_t)z * 805459861u;
    return (hx ^ hy ^ hz) & (uint32_t)((1ull << log2T) - 1ull);
}

/*
 * Eight-corner trilinear encoding of npts unit-cube points on every level.
 * tables: (L, T, F) doubles.  out: (npts, L, F).
 * Lattice coordinate x = p * N_l (vertices 0..N_l, no offset); cell
 * c = floor(x); weight w = x - c; corner (dx,dy,dz) has weight
 * prod(d ? w : 1-w) and index hash(c + d).
 * dbg_idx / dbg_w (optional, npts*L*8): corner indices and weights, corner
 * order dx + 2 dy + 4 dz.
 */
ORC_API void orc_encode(const double *pts, int64_t npts, const int32_t *res, int L, int F, int log2T,
                        const double *tables, double *out, uint32_t *dbg_idx, double *dbg_w)
{
    int64_t T = 1ll << log2T;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npts; ++i) {
        for (int l = 0; l < L; ++l) {
            double x[3], w[3];
            int64_t c[3];
            for (int a = 0; a < 3; ++a) {
                x[a] = pts[3 * i + a] * (double)res[l];
                c[a] = (int64_t)floor(x[a]);
                w[a] = x[a] - (double)c[a];
            }
            for (int f = 0; f < F; ++f) out[(i * L + l) * F + f] = 0.0;
            for (int corner = 0; corner < 8; ++corner) {
                int dx = corner & 1, dy = (corner >> 1) & 1, dz = (corner >> 2) & 1;
                double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) *
                            (dz ? w[2] : 1.0 - w[2]);
                uint32_t idx = orc_hash(c[0] + dx, c[1] + dy, c[2] + dz, log2T);
                if (dbg_idx) dbg_idx[(i * L + l) * 8 + corner] = idx;
                if (dbg_w) dbg_w[(i * L + l) * 8 + corner] = wt;
                for (int f = 0; f < F; ++f)
                    out[(i * L + l) * F + f] += wt * tables[((int64_t)l * T + idx) * F + f];
            }
        }
    }
}

/* Backward of orc_encode: grad_tables[l][idx][f] += w * dout[i][l][f]. */
ORC_API void orc_encode_backward(const double *pts, int64_t npts, const int32_t *res, int L, int F,
                                 int log2T, const double *dout, double *grad_tables)
{
    int64_t T = 1ll << log2T;
    for (int64_t i = 0; i < npts; ++i) {
        for (int l = 0; l < L; ++l) {
            double x[3], w[3];
            int64_t c[3];
            for (int a = 0; a < 3; ++a) {
                x[a] = pts[3 * i + a] * (double)res[l];
                c[a] = (int64_t)floor(x[a]);
                w[a] = x[a] - (double)c[a];
            }
            for (int corner = 0; corner < 8; ++corner) {
                int dx = corner & 1, dy = (corner >> 1) & 1, dz = (corner >> 2) & 1;
                double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) *
                            (dz ? w[2] : 1.0 - w[2]);
                uint32_t idx = orc_hash(c[0] + dx, c[1] + dy, c[2] + dz, log2T);
                for (int f = 0; f < F; ++f)
                    grad_tables[((int64_t)l * T + idx) * F + f] += wt * dout[(i * L + l) * F + f];
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * Geometric judge: nearest Moller-Trumbore hit over all triangles.
 * Accepts tmin <= t <= tmax, u >= 0, v >= 0, u + v <= 1 (closed triangle);
 * a zero determinant is a miss. t = INFINITY and tri = -1 on a miss; ties
 * keep the lowest index.
 * ---------------------------------------------------------------------- */
static void cast_one(const double o[3], const double d[3], double tmin, double tmax, const float *verts,
                     const int32_t *tris, int64_t nt, double *out_t, int32_t *out_tri, double *out_u,
                     double *out_v)
{
    double best = INFINITY, bu = 0, bv = 0;
    int32_t bt = -1;
    for (int64_t t = 0; t < nt; ++t) {
        const float *a = verts + 3 * (int64_t)tris[3 * t];
        const float *b = verts + 3 * (int64_t)tris[3 * t + 1];
        const float *c = verts + 3 * (int64_t)tris[3 * t + 2];
        double e1[3], e2[3], s[3], p[3], q[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = (double)b[k] - (double)a[k];
            e2[k] = (double)c[k] - (double)a[k];
            s[k] = o[k] - (double)a[k];
        }
        p[0] = d[1] * e2[2] - d[2] * e2[1];
        p[1] = d[2] * e2[0] - d[0] * e2[2];
        p[2] = d[0] * e2[1] - d[1] * e2[0];
        double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
        if (det == 0.0) continue;
        double inv = 1.0 / det;
        double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
        if (u < 0.0 || u > 1.0) continue;
        q[0] = s[1] * e1[2] - s[2] * e1[1];
        q[1] = s[2] * e1[0] - s[0] * e1[2];
        q[2] = s[0] * e1[1] - s[1] * e1[0];
        double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
        if (v < 0.0 || u + v > 1.0) continue;
        double tt = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
        if (tt < tmin || tt > tmax) continue;
        if (tt < best) {
            best = tt;
            bt = (int32_t)t;
            bu = u;
            bv = v;
        }
    }
    *out_t = best;
    *out_tri = bt;
    if (out_u) *out_u = bu;
    if (out_v) *out_v = bv;
}

/* rays: n x 8 floats (object space) */
ORC_API void orc_judge(const float *rays, int64_t n, const float *verts, const int32_t *tris,
                       int64_t nt, double *out_t, int32_t *out_tri, double *out_u, double *out_v)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        const float *r = rays + 8 * i;
        double o[3] = {r[0], r[1], r[2]}, d[3] = {r[3], r[4], r[5]};
        cast_one(o, d, r[6], r[7], verts, tris, nt, out_t + i, out_tri + i, out_u ? out_u + i : 0,
                 out_v ? out_v + i : 0);
    }
}

/* FP64 rays: o, d n x 3 doubles; every t >= 0 accepted */
ORC_API void orc_cast64(const double *o, const double *d, int64_t n, const float *verts, const int32_t *tris,
                        int64_t nt, double *out_t, int32_t *out_tri, double *out_u, double *out_v)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        cast_one(o + 3 * i, d + 3 * i, 0.0, INFINITY, verts, tris, nt, out_t + i, out_tri + i, out_u + i,
                 out_v + i);
}

/* Host threads of the parallel loops above (timing only; no result depends
 * on it: every loop writes each output from one iteration). Returns the
 * count in effect before the call; n <= 0 only queries it. */
ORC_API int orc_threads(int n)
{
#ifdef _OPENMP
    const int before = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return before;
#else
    (void)n;
    return 1;
#endif
}
