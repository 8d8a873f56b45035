/*
 * lsnif.h -- C ABI of a GB300-native (sm_103a) implementation of the LSNIF
 * neural ray-intersection query.
 *
 * LSNIF (Fujieda, Kao, Harada, "LSNIF: Locally-Subdivided Neural Intersection
 * Function", PACMCGIT 8(1), 2025) replaces the bottom-level BVH of one object
 * with a small per-object model (Sec. 3, Fig. 2): the ray is clipped to the
 * object's AABB, a 3D-DDA walks a binary V^3 occupancy grid, the ray's entry
 * and exit points of occupied voxels are encoded by a multiresolution sparse
 * hash grid, the concatenated features go through an MLP, and the MLP returns
 * occlusion, hit distance, shading normal, albedo and material index.
 * Objects are trained offline, stored, and loaded at run time (Sec. 3.3);
 * many objects are served by one dispatch grouped by object (Sec. 4).
 *
 * Conventions for every entry point:
 *  - The return value is a status code: LSNIF_OK (0) on success,
 *    LSNIF_PENDING (1) for "still running", a negative LSNIF_ERR_* code on
 *    failure. No C++ exception crosses this boundary. On failure,
 *    lsnif_last_error() returns a message for the calling thread and no
 *    output buffer is guaranteed to have been written.
 *  - "device pointer" means memory of the context's CUDA device
 *    (cudaMalloc, or a PyTorch CUDA tensor's data pointer); "host pointer"
 *    means ordinary process memory. Buffers passed in are owned by the
 *    caller and are not retained after the call returns, except for the
 *    serving calls (lsnif_submit), whose buffers must stay valid until
 *    lsnif_poll reports completion.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *    that take a stream enqueue their kernels on it and return without
 *    waiting unless stated otherwise; outputs are ready when the stream
 *    reaches that point.
 *  - A context is used by one host thread at a time (it is not internally
 *    locked); separate contexts are independent.
 *  - Rays are structure-of-arrays FP32 in the object's space (the mesh's
 *    coordinate frame): origin, direction (need not be unit), tmin, tmax.
 *    n = 0 is a no-op returning LSNIF_OK. A ray with a NaN component or an
 *    all-zero direction is reported as a miss, not an error.
 */
#ifndef LSNIF_H
#define LSNIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSNIF_API_VERSION 2

#if defined(__GNUC__)
#define LSNIF_API __attribute__((visibility("default")))
#else
#define LSNIF_API
#endif

/* ---- status codes ------------------------------------------------------ */
#define LSNIF_OK 0
#define LSNIF_PENDING 1
#define LSNIF_ERR_INVALID_ARG (-1)   /* a pointer, size or config field is invalid */
#define LSNIF_ERR_BAD_HANDLE (-2)    /* unknown object handle or ticket */
#define LSNIF_ERR_OUT_OF_MEMORY (-3) /* a device or host allocation failed */
#define LSNIF_ERR_OVER_BUDGET (-4)   /* the context's device-memory budget is exhausted */
#define LSNIF_ERR_CORRUPT (-5)       /* a serialized object failed validation */
#define LSNIF_ERR_TIMEOUT (-6)       /* lsnif_poll reached its time limit */
#define LSNIF_ERR_CUDA (-7)          /* a CUDA runtime call failed */
#define LSNIF_ERR_DEVICE_CHECK (-8)  /* a kernel reported a failed internal check or wait */
#define LSNIF_ERR_BUSY (-9)          /* the request queue is full */
#define LSNIF_ERR_UNSUPPORTED (-10)  /* configuration not supported by the requested path */

typedef struct lsnif_ctx lsnif_ctx; /* opaque; owns every object and all scratch memory */
typedef uint32_t lsnif_obj;         /* object handle; 0 is never a valid handle */

/* Arithmetic of the query. FP32_PLAIN: FP32 tables, FP32 SIMT network, one
 * kernel per stage with global intermediates. BF16_FUSED: FP16 table copies,
 * FP32 interpolation, BF16 tcgen05 tensor-core MLP with FP32 accumulation,
 * gather + every layer + decode in one kernel (Sec. 5: half precision,
 * fused layers). Traversal is FP32 in both. */
/* FP8_FUSED: as BF16_FUSED with E4M3 network operands (features, weights,
 * hidden activations) and per-layer power-of-two scales chosen from the
 * parameters (the input scale from the largest FP16 table value, each
 * weight scale from the layer's largest weight, each activation scale from
 * max_j ||W_j||_2 M + |b_j| with M the previous magnitude), rounding to
 * nearest even and saturating at 448; tcgen05 kind::f8f6f4, FP32
 * accumulation; the first layer's weights are streamed, so networks too
 * large for BF16 shared memory (F = 4, L = 16, 4 x 128) run. Needs F in
 * {2, 4}, width 64 or 128, L * F a multiple of 16. */
/* FP16_FUSED: BF16_FUSED's kernel with FP16 network operands instead of
 * BF16 (tcgen05 kind::f16 with both A and B FP16): features as gathered from
 * the FP16 tables, FP16 weights, hidden activations rounded to FP16 (nearest
 * even, saturating at +-65504), FP32 accumulation. Networks whose weights do
 * not fit shared memory (such as F = 4, L = 16, 4 x 128) run on a second
 * FP16 kernel that streams the first layer's weights chunk by chunk and the
 * later layers' layer by layer; its features are interpolated in FP32 from
 * the FP16 tables and rounded once to FP16. */
enum lsnif_precision { LSNIF_FP32_PLAIN = 0, LSNIF_BF16_FUSED = 1, LSNIF_FP8_FUSED = 2, LSNIF_FP16_FUSED = 3 };

/* Hidden-layer activation: ReLU, or leaky ReLU with slope 0.01 (Sec. 5.1). */
enum lsnif_activation { LSNIF_RELU = 0, LSNIF_LEAKY_RELU = 1 };

#define LSNIF_MAX_LEVELS 32
#define LSNIF_MAX_HIDDEN 8

/* Hyper-parameters of one object (Sec. 3.1, 3.2, 5.1). */
typedef struct lsnif_config {
    int32_t V;          /* voxels per axis of the occupancy grid (2..1024) */
    int32_t H;          /* cap on boundary points per ray, even (2..64); H/2 voxels */
    int32_t L;          /* hash-grid levels (1..LSNIF_MAX_LEVELS) */
    int32_t F;          /* features per level: 1, 2 or 4 */
    int32_t log2_T;     /* table entries per level = 2^log2_T (4..24) */
    int32_t N_min;      /* coarsest lattice resolution */
    int32_t N_max;      /* finest lattice resolution (>= N_min) */
    int32_t n_hidden;   /* hidden layers (1..LSNIF_MAX_HIDDEN) */
    int32_t width;      /* neurons per hidden layer (16..256, multiple of 16) */
    int32_t n_mat;      /* materials; the network has 8 + n_mat outputs (1..56) */
    int32_t activation; /* enum lsnif_activation */
    float table_init;   /* features start U(-table_init, table_init) (paper: 1e-4) */
    uint64_t seed;      /* seed of the built-in initialisation */
} lsnif_config;

/* A triangle mesh (host pointers, read during the call only). */
typedef struct lsnif_mesh {
    const float *verts;      /* nv x 3 positions */
    const int32_t *tris;     /* nt x 3 vertex indices */
    const float *vnormals;   /* nv x 3 unit shading normals, or NULL (training labels need them) */
    const int32_t *tri_mat;  /* nt material indices in [0, n_mat), or NULL (all 0) */
    const float *mat_albedo; /* n_mat x 3 RGB, or NULL (0.5 grey) */
    int64_t nv, nt;
} lsnif_mesh;

/* How lsnif_load_object builds an object. Exactly one source of geometry:
 * a serialized blob, or a mesh (voxelized on load, Sec. 3.1). Parameters
 * come from the blob, from `tables`/`mlp` when given, or from the built-in
 * seeded initialisation (tables uniform, weights Xavier-uniform, biases 0). */
typedef struct lsnif_object_desc {
    lsnif_config cfg;        /* ignored when blob != NULL */
    lsnif_mesh mesh;         /* used when blob == NULL */
    const float *tables;     /* host, L x 2^log2_T x F FP32, or NULL */
    const float *mlp;        /* host, packed FP32 [W0 (out x in, row-major), b0, W1, b1, ...], or NULL */
    int32_t keep_mesh;       /* nonzero: keep the mesh on the device for training labels */
    const void *blob;        /* host, from lsnif_save_object, or NULL */
    size_t blob_len;
    /* Face-count switch of the hybrid pipeline (Sec. 4): a mesh with fewer
     * than this many triangles is not turned into an LSNIF object but kept
     * as a mesh object -- its triangles and a BVH, answered exactly by every
     * query (lsnif_query_rays, lsnif_query_scene, lsnif_raster_gbuffer).
     * Only cfg.n_mat of the config is used then. 0: never. */
    int64_t bvh_below_faces;
} lsnif_object_desc;

/* Read-only facts about a loaded object. */
typedef struct lsnif_object_info {
    lsnif_config cfg;
    float bmin[3], bmax[3];              /* AABB (object space) */
    int32_t res[LSNIF_MAX_LEVELS];       /* lattice resolution per level */
    int64_t n_occupied;                  /* occupied voxels */
    int64_t n_params_mlp;                /* weights + biases */
    size_t device_bytes;                 /* device memory charged to the budget */
    size_t footprint_fp16_bytes;         /* paper's storage model: bits + FP16 tables + FP16 network */
    int32_t kind;                        /* 0 = LSNIF object, 1 = mesh object (triangles + BVH) */
    int64_t n_triangles;                 /* mesh objects: triangles */
    int64_t bvh_nodes;                   /* mesh objects: BVH nodes (32 bytes each) */
} lsnif_object_info;

/* Rays, structure of arrays, DEVICE pointers (host pointers for
 * lsnif_query_rays_host). obj: per-ray handle (NULL: every ray uses
 * single_obj). */
typedef struct lsnif_rays {
    const float *ox, *oy, *oz;
    const float *dx, *dy, *dz;
    const float *tmin, *tmax;
    const uint32_t *obj;
    lsnif_obj single_obj;
    int64_t n;
} lsnif_rays;

/* Per-ray results; every pointer may be NULL (not written). For rays that
 * meet no occupied voxel: hit 0, t +inf, normal 0, material -1, albedo 0,
 * logits NaN. Otherwise the decoded network outputs (Sec. 5.3): hit =
 * (occlusion logit > 0) and tmin <= t <= tmax; t = t0 + sigmoid(z1)(t1-t0)
 * over the ray's clipped AABB interval [t0, t1]; normal = z2..4 normalised;
 * albedo = sigmoid(z5..7); material = argmax z8.. (lowest index on ties).
 * logits: n x (8 + n_mat) raw network outputs, row-major. */
typedef struct lsnif_hits {
    uint8_t *hit;
    float *t;
    float *nx, *ny, *nz;
    int32_t *mat;
    float *ar, *ag, *ab;
    float *logits;
} lsnif_hits;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`. mem_budget_bytes caps the device
 * memory the context may hold (objects + scratch); 0 means no cap.
 * Errors: INVALID_ARG (out == NULL or bad device), CUDA, OUT_OF_MEMORY. */
LSNIF_API int lsnif_create(lsnif_ctx **out, int device, size_t mem_budget_bytes);

/* Destroy a context: waits for its queued work, frees every object and all
 * scratch memory. NULL is accepted. */
LSNIF_API int lsnif_destroy(lsnif_ctx *ctx);

/* Message of the most recent failing call on this thread ("" if none). The
 * string is owned by the library and valid until the next call. */
LSNIF_API const char *lsnif_last_error(void);

/* API version compiled into the library (LSNIF_API_VERSION). */
LSNIF_API int lsnif_version(void);

/* Wait for `stream` and report kernel-side failures since the last check:
 * DEVICE_CHECK when a kernel flagged an unknown object handle, a failed
 * internal bound check or a bounded wait that gave up (the flag is then
 * cleared); CUDA when the stream itself failed. Kernels never trap. */
LSNIF_API int lsnif_check(lsnif_ctx *ctx, void *stream);

/* ---- objects (Sec. 3.3: voxels, grid and weights stored, loaded at run time) */

/* Build an object from a mesh (FP64 separating-axis voxelization of the
 * mesh's AABB, Sec. 3.1) or from a serialized blob, upload it and return its
 * handle in *out. All desc pointers are host pointers read during the call.
 * Errors: INVALID_ARG (bad config or mesh), CORRUPT (bad blob),
 * OVER_BUDGET, OUT_OF_MEMORY, CUDA. */
LSNIF_API int lsnif_load_object(lsnif_ctx *ctx, const lsnif_object_desc *desc, lsnif_obj *out);

/* Serialize an object (config, AABB, occupancy, FP32 tables and network)
 * into buf. With buf == NULL or *inout_len too small, sets *inout_len to
 * the size needed and returns INVALID_ARG (buf != NULL) or OK (buf == NULL).
 * The blob round-trips bit-exactly through lsnif_load_object. */
LSNIF_API int lsnif_save_object(lsnif_ctx *ctx, lsnif_obj obj, void *buf, size_t *inout_len);

/* Free an object's device memory. Errors: BAD_HANDLE. */
LSNIF_API int lsnif_unload_object(lsnif_ctx *ctx, lsnif_obj obj);

/* Fill *out with facts about the object. Errors: BAD_HANDLE. */
LSNIF_API int lsnif_get_object_info(lsnif_ctx *ctx, lsnif_obj obj, lsnif_object_info *out);

/* Which array lsnif_read_params / lsnif_write_params move. */
enum lsnif_param {
    LSNIF_PARAM_OCCUPANCY = 0, /* ceil(V^3/32) uint32 words, bit i of word i>>5 = voxel i */
    LSNIF_PARAM_TABLES = 1,    /* L x T x F FP32 (master copy) */
    LSNIF_PARAM_MLP = 2,       /* packed FP32 network, layout of lsnif_object_desc.mlp */
    LSNIF_PARAM_GRAD_TABLES = 3, /* gradients of the last lsnif_train_step, FP32 */
    LSNIF_PARAM_GRAD_MLP = 4
};

/* Copy an object array to host memory (synchronous). bytes must equal the
 * array's size. Errors: BAD_HANDLE, INVALID_ARG (size), CUDA. */
LSNIF_API int lsnif_read_params(lsnif_ctx *ctx, lsnif_obj obj, int which, void *host_dst, size_t bytes);

/* Replace the tables or network (LSNIF_PARAM_TABLES / _MLP) from host
 * memory; refreshes the reduced-precision copies and resets the optimiser. */
LSNIF_API int lsnif_write_params(lsnif_ctx *ctx, lsnif_obj obj, int which, const void *host_src, size_t bytes);

/* ---- the query (Fig. 2; Sec. 3.1-3.3; Sec. 4 single dispatch grouped by object) */

/* Intersect rays with objects: AABB clip, 3D-DDA over the occupancy grid,
 * entry/exit points of the first H/2 occupied voxels, hash-grid encoding,
 * MLP, decode. Device pointers for rays and hits. With rays->obj, rays of
 * many objects go through one launch sequence grouped by object. Uses
 * context-owned scratch memory (grown on demand and charged to the budget).
 * Results do not depend on which other rays share the call.
 * Errors: INVALID_ARG, BAD_HANDLE (a ray names an unknown object: checked
 * on the device, reported as DEVICE_CHECK), UNSUPPORTED (a fused path --
 * BF16, FP16 or FP8 -- with a config it does not cover), OVER_BUDGET, CUDA.
 * precision: one of enum lsnif_precision. */
LSNIF_API int lsnif_query_rays(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                     void *stream);

/* lsnif_query_rays with HOST ray and hit buffers: copies the rays to the
 * device, runs the query and copies the results back, returning when they
 * are in host memory. Page-locked host buffers make the copies faster. */
LSNIF_API int lsnif_query_rays_host(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                          void *stream);

/* How lsnif_query_rays_host moves data (an integration choice; the paper has
 * no counterpart). STAGED (default): copies through device buffers in
 * chunks that overlap the queries; any host memory. DIRECT: when every
 * buffer given is page-locked host memory (cudaHostAlloc, cudaHostRegister,
 * PyTorch pinned tensors), the kernels read the rays and write the results
 * there through its mapped address, with no staging copies or staging
 * memory -- on GB300 host memory is reached over the coherent NVLink-C2C
 * link; otherwise the call stages as in STAGED. Results are the same bit for
 * bit. Errors: INVALID_ARG. */
enum lsnif_host_mode { LSNIF_HOST_STAGED = 0, LSNIF_HOST_DIRECT = 1 };
LSNIF_API int lsnif_set_host_mode(lsnif_ctx *ctx, int mode);

/* lsnif_query_rays for callers that cannot allocate device memory while they
 * run -- for example a renderer whose frame loop forbids cudaMalloc/cudaFree
 * because they can synchronise the whole device, or a plug-in inside a host
 * engine that owns every allocation. The paper has no counterpart; this is
 * an integration convenience of this library.
 *
 * Runs the BF16 fused query (precision LSNIF_BF16_FUSED) on DEVICE ray and
 * hit buffers like lsnif_query_rays -- the same kernels, with the context's
 * traversal and grouping choices (lsnif_set_trace_mode, lsnif_set_group_mode,
 * lsnif_autotune), so the results are those of lsnif_query_rays at
 * LSNIF_BF16_FUSED bit for bit -- but its scratch lives in one static
 * device array of 32 MiB compiled into the library (every GPU that loads the
 * library holds it until the process exits) and it calls no cudaMalloc,
 * cudaFree or other allocating routine. The first call on a device looks up
 * that array's device address (once per device); make that first call
 * before any stream capture. Every call shares the array and it keeps the
 * previous call's contents, so calls that overlap on the GPU (other
 * streams, other threads, other contexts of the process) race: serialise
 * them. A batch whose scratch does not fit (about 230 bytes per ray for H =
 * 18, i.e. some 140k rays; when trace mode 2 or group mode 2 is chosen their
 * counting sort takes 8 MiB of the array first, leaving room for about
 * 100k) is rejected with LSNIF_ERR_INVALID_ARG and a message giving the
 * sizes. Errors otherwise as lsnif_query_rays. */
LSNIF_API int lsnif_query_rays_noalloc(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, void *stream);

/* ---- instanced scenes (Sec. 4 wavefront integration, Sec. 6 instancing) -- */

/* One placement of an object in a scene: the affine map from world to
 * object coordinates, p_obj = A p_world + b, stored row-major as the 3 x 4
 * matrix [A | b]. A must be invertible (rotation, scale, shear). */
typedef struct lsnif_instance {
    lsnif_obj obj;
    float world_to_obj[12];
} lsnif_instance;

/* Query world-space rays (DEVICE buffers; rays->obj and rays->single_obj are
 * ignored) against n_inst instances (HOST array, read during the call).
 * Every (ray, instance) pair whose ray, mapped into the instance's object
 * frame (o' = A o + b, d' = A d; t, tmin and tmax unchanged), crosses the
 * object's box is queried there; the pairs of all instances go through one
 * launch sequence grouped by object (Sec. 4). Each ray keeps its nearest hit:
 * smallest t, the lowest instance index on equal t. Results (DEVICE, any
 * pointer in `hits` may be NULL; logits are not supported and must be NULL):
 * hit, t, world normal A^T n normalised, material, albedo; inst_hit[n]
 * (DEVICE, may be NULL) receives the instance index, -1 on a miss. A ray no
 * pair hits gets hit 0, t +inf, normal 0, material -1, albedo 0. The call
 * waits once for the pair count on `stream`; the rest is queued on `stream`.
 * Scratch (about 80 bytes per pair plus the query's) is held by the context.
 * Errors: INVALID_ARG (NULL arrays, n_inst < 1, logits given, a singular A),
 * BAD_HANDLE (an instance names an unknown object), OVER_BUDGET,
 * OUT_OF_MEMORY, UNSUPPORTED (BF16_FUSED over objects of different network
 * shapes), CUDA, DEVICE_CHECK. */
LSNIF_API int lsnif_query_scene(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_instance *inst, int n_inst,
                                lsnif_hits *hits, int32_t *inst_hit, int precision, void *stream);

/* ---- mesh objects ------------------------------------------------------- */

/* The BVH builder of mesh objects (see bvh_below_faces), on the host only
 * (no GPU, no context): binned-SAH binary BVH over nt triangles. nodes_out
 * (room for 2 nt - 1 nodes) receives *n_nodes nodes of 32 bytes: float lo[3],
 * int32 a, float hi[3], int32 n -- an internal node has n = 0 and children
 * a and a + 1; a leaf has n > 0 triangles at order_out[a .. a + n). order_out
 * (nt entries) maps stored positions to mesh triangles; *depth (may be NULL)
 * receives the deepest leaf's depth. For checking the structure. Errors:
 * INVALID_ARG (NULL pointers, empty mesh, index out of range). */
LSNIF_API int lsnif_bvh_build_host(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                   void *nodes_out, int64_t *n_nodes, int32_t *order_out, int32_t *depth);

/* The occupancy distance field the traversal skips empty space with, on the
 * host only (no GPU, no context): for every voxel of the V^3 bitset `occ`
 * (layout of lsnif_read_params' occupancy), the Chebyshev distance in voxels
 * to the nearest occupied voxel, capped at `cap` (0 = occupied), into out[V^3]
 * in the same voxel order. For checking the transform. Errors: INVALID_ARG. */
LSNIF_API int lsnif_occupancy_distance_host(const uint32_t *occ, int32_t V, int32_t cap, uint8_t *out);

/* ---- primary-ray G-buffer (Sec. 4, Fig. 4a) ----------------------------- */

/* Pinhole camera: the ray of pixel (px, py) (row py from the top) starts at
 * eye with direction forward + x right + y up, normalised, where x = (2 (px
 * + 1/2) / width - 1) tan_half_fov width / height and y = (1 - 2 (py +
 * 1/2) / height) tan_half_fov. forward, right, up must be orthonormal. */
typedef struct lsnif_camera {
    float eye[3], forward[3], right[3], up[3];
    float tan_half_fov;   /* tangent of half the vertical field of view */
    int32_t width, height;
} lsnif_camera;

/* G-buffer planes, width x height each, row-major (DEVICE; any pointer may
 * be NULL; nx, ny, nz all or none). */
typedef struct lsnif_gbuffer {
    uint8_t *hit;         /* 1 where a triangle is hit, else 0 (the lsnif_hits convention) */
    int32_t *shape;       /* instance index; -1 where no triangle is hit */
    int32_t *prim;        /* triangle index in the instance's mesh; -1 */
    float *u, *v;         /* barycentric coordinates: p = (1-u-v) a + u b + v c; 0 */
    float *dist;          /* camera distance (t of the unit-direction ray); +inf */
    float *nx, *ny, *nz;  /* shading normal: vertex normals interpolated at (u, v),
                             mapped to world by A^T and normalised; 0 */
} lsnif_gbuffer;

/* Rasterise the primary visibility of n_inst instances (HOST array, as for
 * lsnif_query_scene; their objects must have been loaded with keep_mesh) into
 * a G-buffer: for every pixel, the nearest triangle that the pixel-centre ray
 * hits (closed triangles, Moller-Trumbore in FP32 on the triangle mapped to
 * world space, distance >= 0); equal distances keep the lowest instance,
 * then the lowest triangle (Sec. 4: primary visibility by rasterisation, so
 * that LSNIF answers only the later rays). Asynchronous on `stream`.
 * Scratch (8 bytes per pixel + 4 per triangle over the instances) is owned
 * by the context and reused. Errors: INVALID_ARG (NULL arguments, image
 * outside 1..16384 a side, camera not orthonormal, singular transform, more
 * than 2^31 - 1 triangles), BAD_HANDLE, UNSUPPORTED (object without its
 * mesh), OUT_OF_MEMORY, CUDA. */
LSNIF_API int lsnif_raster_gbuffer(lsnif_ctx *ctx, const lsnif_camera *cam, const lsnif_instance *inst, int n_inst,
                                   lsnif_gbuffer *out, void *stream);

/* Next-bounce rays of a path tracer from query results (all DEVICE): for a
 * ray with hit != 0 and a non-zero normal, origin = o + t d + eps n_f and a
 * cosine-weighted direction about n_f, where n_f is the normal turned to
 * face the incoming ray; the direction is x t + y b + z n_f with (x, y) =
 * sqrt(u0) (cos 2 pi u1, sin 2 pi u1), z = sqrt(1 - u0), and (t, b) the
 * orthonormal basis of Duff et al. 2017 about n_f; tmin 0, tmax +inf. Other
 * rays become dead rays: zero origin and direction (a miss for the query).
 * u: n x 2 uniforms in [0, 1), row-major. out: 8 x n FP32, rows ox oy oz dx
 * dy dz tmin tmax (n = rays->n), aliasing nothing in rays, hits or u.
 * hits->hit, t, nx, ny, nz are required. Errors: INVALID_ARG (NULL pointers,
 * n < 0), CUDA. */
LSNIF_API int lsnif_bounce_rays(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_hits *hits, const float *u,
                                float eps, float *out, void *stream);

/* Stage outputs of the traversal (a1-a5 of the query) for one object, all
 * DEVICE pointers, any may be NULL: k[n] kept occupied voxels (<= H/2);
 * t01[2n] the clipped AABB interval (NaN on a miss); pts[n*H*3] boundary
 * points in unit-cube coordinates of the AABB, entry then exit per voxel,
 * the crossed coordinate exactly face/V, slots past 2k untouched;
 * vox[n*H/2] voxel ids (z*V+y)*V+x, -1 past k. */
typedef struct lsnif_trace_out {
    int32_t *k;
    float *t01;
    float *pts;
    int32_t *vox;
} lsnif_trace_out;

/* Run only the traversal kernel (Sec. 3.1) for rays->single_obj. */
LSNIF_API int lsnif_trace(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_trace_out *out, void *stream);

/* Hash-grid encoding of n unit-cube points (Sec. 3.2): pts DEVICE n x 3 FP32
 * -> feats DEVICE n x L x F FP32. precision FP32_PLAIN reads the FP32
 * tables; every other precision reads the FP16 copies (interpolation in FP32
 * either way). Zero-weight corners are skipped. */
LSNIF_API int lsnif_encode(lsnif_ctx *ctx, lsnif_obj obj, const float *pts, int64_t n, float *feats,
                 int precision, void *stream);

/* Table index of each of the 8 cell corners per point and level: DEVICE
 * out n x L x 8 uint32, corner order dx + 2 dy + 4 dz. The cell is the floor
 * of the exact product p * N_l of the FP32 point and the level resolution
 * (computed with an error-free FMA split, identical to an FP64 evaluation). */
LSNIF_API int lsnif_corner_indices(lsnif_ctx *ctx, lsnif_obj obj, const float *pts, int64_t n, uint32_t *out,
                         void *stream);

/* The object's network alone (Sec. 5.1) on n given input rows: X DEVICE
 * n x (H*L*F) FP32 -> Z DEVICE n x (8+n_mat) FP32 logits. BF16_FUSED and
 * FP16_FUSED run the tcgen05 tensor-core layers (inputs rounded to the
 * operand type); FP8_FUSED is not offered here. */
LSNIF_API int lsnif_mlp(lsnif_ctx *ctx, lsnif_obj obj, const float *X, int64_t n, float *Z, int precision,
              void *stream);

/* Graph mode (on = 1): lsnif_query_rays on a non-default stream captures each
 * distinct query -- same ray and hit buffers, ray count, precision, object
 * handle, fused-kernel variant and number of object slots -- into a CUDA
 * graph the first time and replays that graph afterwards (one launch instead
 * of the query's kernel sequence). Object parameters may change between
 * replays (kernels read them at run time). Graphs are dropped when the
 * scratch is reallocated or graph mode is switched off. Queries on the
 * legacy default stream, and profiled queries, run without graphs. */
LSNIF_API int lsnif_set_graph_mode(lsnif_ctx *ctx, int on);

/* ---- autotuning of the fused kernel's shape ----------------------------- */

/* Number of fused-kernel variants (gather threads per CTA x corner-load
 * levels in flight per gather item x gather style). */
LSNIF_API int lsnif_variant_count(void);

/* Shape of variant v: *threads = gather threads per CTA (the CTA also has
 * one MMA warp and four epilogue warps), *levels = levels of corner loads in
 * flight per gather item. Errors: INVALID_ARG for v out of range. */
LSNIF_API int lsnif_variant_shape(int v, int *threads, int *levels);

/* Use variant v for every later BF16 and FP16 fused query of the context. */
LSNIF_API int lsnif_set_variant(lsnif_ctx *ctx, int v);

/* The FP8 fused kernel's shapes (LSNIF_FP8_FUSED with F = 4; F = 2 always
 * runs variant 0): *threads = gather threads per CTA, *levels = hash levels
 * whose corner loads one gather item issues together. Fewer levels per
 * batch need fewer registers, which lets more gather warps share an SM.
 * Errors: INVALID_ARG for v out of range. All variants compute identical
 * results. */
LSNIF_API int lsnif_variant8_count(void);
LSNIF_API int lsnif_variant8_shape(int v, int *threads, int *levels);

/* Use FP8 variant v for every later LSNIF_FP8_FUSED query of the context. */
LSNIF_API int lsnif_set_variant8(lsnif_ctx *ctx, int v);

/* Traversal kernel for later queries: 0 = one ray per thread, voxel by
 * voxel; 1 = persistent lanes (a lane whose ray finished takes the next ray
 * from a global counter) that cross empty cubes of voxels in one step;
 * 2 = the same lanes, handed the rays in the order of a counting sort by
 * (object, Morton cell of the point where the ray enters the object's box,
 * direction octant), so that shuffled rays (secondary rays, rays mixed
 * across objects) walk neighbouring voxels together. All compute identical
 * results; LSNIF_ERR_INVALID_ARG for any other mode. */
LSNIF_API int lsnif_set_trace_mode(lsnif_ctx *ctx, int mode);

/* Time every fused-kernel variant on `rays` (DEVICE buffers, `reps` BF16
 * queries each after one warm-up, CUDA events on `stream`, synchronous), keep
 * the fastest, then the other traversal kernels and the other groupings,
 * keeping each if faster; then time every variant again with
 * FP16 queries and keep the fastest for LSNIF_FP16_FUSED (the FP16 kernel
 * holds no lo weights, so its shared memory and L1 differ). *chosen (may be
 * NULL) receives the BF16 variant index. Results of the queries are
 * discarded; all choices compute identical results. */
LSNIF_API int lsnif_autotune(lsnif_ctx *ctx, const lsnif_rays *rays, int reps, void *stream, int *chosen);

/* How live rays are grouped into 128-ray tiles: 0 = by object, then by
 * number of occupied voxels (descending); 1 = in the rays' own order within
 * each object: single-object queries keep the original order exactly,
 * multi-object queries (and instanced scenes) group by object only and keep
 * each warp's run of consecutive rays together (neighbouring primary rays
 * share voxels and lattice cells, which the gather's caches exploit);
 * 2 = by object, then by the Morton code of the cell (64 per axis of the
 * object's box, fewer when more than 8 objects are loaded: at most 2^21
 * object-cell pairs) that holds the ray's first boundary point, so that
 * tiles hold nearby points whatever order the rays come in (secondary rays,
 * rays shuffled across objects). All compute identical results;
 * LSNIF_ERR_INVALID_ARG for any other mode. */
LSNIF_API int lsnif_set_group_mode(lsnif_ctx *ctx, int mode);

/* The context's current fused-kernel variant of BF16 queries, traversal
 * kernel and grouping (lsnif_autotune sets all three). */
LSNIF_API int lsnif_get_tuning(lsnif_ctx *ctx, int *variant, int *trace_mode, int *group_mode);

/* ---- training (Sec. 5.2, 5.3) ------------------------------------------ */

/* Number of uniforms per training ray that lsnif_make_training_rays reads. */
#define LSNIF_TRAIN_UNIFORMS 40

/* Balanced training rays (Sec. 5.2) for an object loaded with keep_mesh:
 * rays [0, n_outside) start uniformly on the sphere of radius 1.05 x half
 * the AABB diagonal about its centre (u0, u1) with cosine-weighted
 * directions about the inward direction (u2, u3); rays [n_outside, n) cast
 * up to 8 such rays (u[4+4a .. 8+4a]) until one hits the mesh and start at
 * the hit, offset 1e-4 x diagonal along the geometric normal facing the
 * incoming ray, with a cosine-weighted direction about it (u36, u37); if no
 * attempt hits they keep the outside ray of u0..u3. u: DEVICE n x 40 FP32
 * uniforms in [0,1) (the caller draws them). rays_out: DEVICE 8 x n FP32
 * (ox,oy,oz,dx,dy,dz,tmin=0,tmax=inf rows). surface: DEVICE n bytes, 1 for
 * rays that start on the surface; may be NULL. */
LSNIF_API int lsnif_make_training_rays(lsnif_ctx *ctx, lsnif_obj obj, const float *u, int64_t n,
                             int64_t n_outside, float *rays_out, uint8_t *surface, void *stream);

/* Ground-truth labels by ray casting against the kept mesh (Sec. 5.2),
 * DEVICE outputs, any may be NULL: occ (0/1), t_local = (t_hit-t0)/(t1-t0)
 * over the clipped AABB interval (0 on a miss), normal (3n, barycentric
 * shading normal, not flipped), albedo (3n), mat, t_hit (+inf on a miss),
 * tri (-1 on a miss), k (kept occupied voxels of the traversal, so callers
 * can drop rays that never reach the network). */
typedef struct lsnif_labels {
    float *occ;
    float *t_local;
    float *normal;
    float *albedo;
    int32_t *mat;
    float *t_hit;
    int32_t *tri;
    int32_t *k;
} lsnif_labels;

LSNIF_API int lsnif_label_rays(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_labels *out, void *stream);

typedef struct lsnif_train_opts {
    float lr;            /* Adam learning rate (paper: 0.01) */
    float beta1, beta2;  /* Adam moments (0.9, 0.999) */
    float eps;           /* Adam epsilon (1e-8) */
    int32_t apply_update;/* 0: only compute the loss and gradients (kept for lsnif_read_params) */
    int32_t products;    /* the network's dense products: LSNIF_TRAIN_TENSOR_CORES (default) or
                            LSNIF_TRAIN_FP32_SIMT */
} lsnif_train_opts;

/* How the training step forms the network's dense products (forward, input
 * gradients, weight gradients). TENSOR_CORES: tcgen05 kind::f16 with BF16
 * operands in two-term form (hi = BF16(x), lo = BF16(x - hi); hi.hi + hi.lo
 * + lo.hi) and FP32 accumulation -- the paper's reduced-precision products
 * with FP32 gradient accumulation (Sec. 5), at FP32-level accuracy and range.
 * FP32_SIMT: FP32 fused multiply-adds on the CUDA cores (the reference). */
enum lsnif_train_products { LSNIF_TRAIN_TENSOR_CORES = 0, LSNIF_TRAIN_FP32_SIMT = 1 };

typedef struct lsnif_train_stats {
    float total, occ, t, normal, albedo, mat; /* batch-mean loss terms (Sec. 5.3) */
    int64_t step;                              /* optimiser steps taken so far */
} lsnif_train_stats;

/* One optimisation step of the whole object (network and tables jointly,
 * Sec. 5.2) on a batch: forward with saved activations, multi-head loss
 * (BCE; masked MAE, cosine, relative L2, cross-entropy; Sec. 5.3), backward
 * (network, then trilinear scatter of feature gradients into the tables),
 * Adam. rays: DEVICE batch (single object); labels: DEVICE occ, t_local,
 * normal, albedo, mat as produced by lsnif_label_rays. Rays that meet no
 * occupied voxel contribute nothing. stats (host, may be NULL) are written
 * after a stream synchronisation. The FP16/BF16 copies used by the fused
 * query are refreshed after each update. */
LSNIF_API int lsnif_train_step(lsnif_ctx *ctx, const lsnif_rays *rays, const lsnif_labels *labels,
                     const lsnif_train_opts *opts, lsnif_train_stats *stats, void *stream);

/* ---- serving: continuous batching (Sec. 4 dispatch, served as requests) -- */

typedef struct lsnif_req_stats {
    double submit_us, start_us, done_us; /* host clock, microseconds */
    double gpu_ms;                        /* device time of the request's work */
    int64_t n_rays;
} lsnif_req_stats;

/* Queue a query. rays/hits are DEVICE buffers that must stay valid until
 * lsnif_poll returns OK or an error for the ticket. `stream` is the stream on
 * which the caller produced (or last used) those buffers: the request runs
 * only after the work enqueued on `stream` up to this call, so initialising
 * the buffers there and submitting right away is safe. A request is admitted
 * to the device when one of the context's streams is free and its scratch
 * fits the memory budget; admitted requests run concurrently with those
 * already on the device. Errors: INVALID_ARG, BUSY (queue full),
 * OVER_BUDGET (the request alone can never fit the budget). */
LSNIF_API int lsnif_submit(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision, void *stream,
                           uint64_t *ticket);

/* Advance the queue and report a request: OK (done; *st filled if not
 * NULL), PENDING (not done and timeout_us == 0), TIMEOUT (not done within
 * timeout_us microseconds), BAD_HANDLE, or the request's own error. Never
 * blocks longer than timeout_us (plus one admission step). A failed device
 * check in a request's kernels (for example a ray naming an unknown object
 * handle) is reported as DEVICE_CHECK on that request's ticket only: each of
 * the context's serving streams has its own device error word, copied to
 * host memory behind the request's kernels, so no read blocks and other
 * requests are not charged. Each of the context's serving streams takes up
 * to two requests, the second in stream order behind the first when the
 * stream's scratch already fits it: an admitted request starts on the device
 * when its predecessor ends, without a host call. Requests still waiting in
 * the queue are admitted inside lsnif_submit and lsnif_poll. */
LSNIF_API int lsnif_poll(lsnif_ctx *ctx, uint64_t ticket, int64_t timeout_us, lsnif_req_stats *st);

/* Number of submitted requests not yet reported done by lsnif_poll. */
LSNIF_API int64_t lsnif_pending(lsnif_ctx *ctx);

/* ---- measurement ------------------------------------------------------- */

typedef struct lsnif_profile {
    float ms_trace;      /* traversal + compaction kernels */
    float ms_group;      /* grouping of live rays by object and point count */
    float ms_encode;     /* FP32 path: gather kernel */
    float ms_mlp;        /* FP32 path: network kernel; BF16 path: fused gather+network kernel */
    float ms_total;
    int64_t n_rays, n_live, n_points; /* rays, rays reaching the network, boundary points */
    int32_t launches;    /* kernels launched by the last query */
} lsnif_profile;

/* Turn per-stage CUDA-event timing of queries on (1) or off (0). */
LSNIF_API int lsnif_set_profiling(lsnif_ctx *ctx, int on);

/* Stage times and counts of the last query run with profiling on
 * (synchronises the stream it ran on). */
LSNIF_API int lsnif_last_profile(lsnif_ctx *ctx, lsnif_profile *out);

/* Measurement: the request ceiling of the hash-grid gather on this GPU. The
 * paper has no counterpart; it supplies the roof against which the fused
 * query's corner loads are reported. Runs `loads` (0: about 1.6e9)
 * independent 8-byte loads at uniformly random positions of object obj's
 * FP16 table copy (L x 2^log2_T x F x 2 bytes, the tables the fused query
 * gathers from), 16 in flight per thread and every SM fully occupied, after
 * an untimed warm-up launch, and writes the loads completed per second to
 * *requests_per_s (each load touches one 32-byte sector). Tables that fit
 * L2 (129 MB) give L2's random-request rate; larger ones HBM's. Timed with
 * CUDA events on `stream`; returns when done. Allocates 4 bytes for the
 * duration of the call. Errors: INVALID_ARG, BAD_HANDLE, UNSUPPORTED (a mesh
 * object, or a table of 2^32 or more 8-byte words), OVER_BUDGET, CUDA. */
LSNIF_API int lsnif_gather_rate(lsnif_ctx *ctx, lsnif_obj obj, int64_t loads, void *stream, double *requests_per_s);

/* Device memory the context currently holds (objects + scratch). */
LSNIF_API size_t lsnif_device_bytes(lsnif_ctx *ctx);

/* Host-side fault injection for tests: after `n` further successful device
 * allocations the next one fails as if cudaMalloc had (n < 0 disables). */
LSNIF_API int lsnif_debug_fail_alloc_after(lsnif_ctx *ctx, int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* LSNIF_H */
