"""Python binding of the LSNIF C ABI (include/lsnif.h).

Argument marshalling only: every step of the query, the training step and
the serving loop runs in the CUDA library `_lib/liblsnif.so`. PyTorch is used
for device memory and streams. There is no fallback: if the library is
missing or a GPU is absent, calls raise.

Names follow the C entry points (lsnif_create -> Context, lsnif_query_rays ->
Context.query_rays, ...).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblsnif.so")

OK, PENDING = 0, 1
ERR = {-1: "INVALID_ARG", -2: "BAD_HANDLE", -3: "OUT_OF_MEMORY", -4: "OVER_BUDGET", -5: "CORRUPT", -6: "TIMEOUT",
       -7: "CUDA", -8: "DEVICE_CHECK", -9: "BUSY", -10: "UNSUPPORTED"}
FP32_PLAIN, BF16_FUSED, FP8_FUSED, FP16_FUSED = 0, 1, 2, 3
PARAM_OCCUPANCY, PARAM_TABLES, PARAM_MLP, PARAM_GRAD_TABLES, PARAM_GRAD_MLP = 0, 1, 2, 3, 4
TRAIN_UNIFORMS = 40
TRAIN_TENSOR_CORES, TRAIN_FP32_SIMT = 0, 1
HOST_STAGED, HOST_DIRECT = 0, 1
MAX_LEVELS = 32


class LsnifError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


# ---- mirrors of the C structs ---------------------------------------------------

class Config(C.Structure):
    _fields_ = [("V", C.c_int32), ("H", C.c_int32), ("L", C.c_int32), ("F", C.c_int32), ("log2_T", C.c_int32),
                ("N_min", C.c_int32), ("N_max", C.c_int32), ("n_hidden", C.c_int32), ("width", C.c_int32),
                ("n_mat", C.c_int32), ("activation", C.c_int32), ("table_init", C.c_float), ("seed", C.c_uint64)]


class Mesh(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("tris", C.c_void_p), ("vnormals", C.c_void_p), ("tri_mat", C.c_void_p),
                ("mat_albedo", C.c_void_p), ("nv", C.c_int64), ("nt", C.c_int64)]


class ObjectDesc(C.Structure):
    _fields_ = [("cfg", Config), ("mesh", Mesh), ("tables", C.c_void_p), ("mlp", C.c_void_p),
                ("keep_mesh", C.c_int32), ("blob", C.c_void_p), ("blob_len", C.c_size_t),
                ("bvh_below_faces", C.c_int64)]


class ObjectInfo(C.Structure):
    _fields_ = [("cfg", Config), ("bmin", C.c_float * 3), ("bmax", C.c_float * 3),
                ("res", C.c_int32 * MAX_LEVELS), ("n_occupied", C.c_int64), ("n_params_mlp", C.c_int64),
                ("device_bytes", C.c_size_t), ("footprint_fp16_bytes", C.c_size_t), ("kind", C.c_int32),
                ("n_triangles", C.c_int64), ("bvh_nodes", C.c_int64)]


class Rays(C.Structure):
    _fields_ = [("ox", C.c_void_p), ("oy", C.c_void_p), ("oz", C.c_void_p), ("dx", C.c_void_p),
                ("dy", C.c_void_p), ("dz", C.c_void_p), ("tmin", C.c_void_p), ("tmax", C.c_void_p),
                ("obj", C.c_void_p), ("single_obj", C.c_uint32), ("n", C.c_int64)]


class Instance(C.Structure):
    _fields_ = [("obj", C.c_uint32), ("world_to_obj", C.c_float * 12)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("forward", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_fov", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class GBufferS(C.Structure):
    _fields_ = [("hit", C.c_void_p), ("shape", C.c_void_p), ("prim", C.c_void_p), ("u", C.c_void_p),
                ("v", C.c_void_p), ("dist", C.c_void_p), ("nx", C.c_void_p), ("ny", C.c_void_p),
                ("nz", C.c_void_p)]


class Hits(C.Structure):
    _fields_ = [("hit", C.c_void_p), ("t", C.c_void_p), ("nx", C.c_void_p), ("ny", C.c_void_p),
                ("nz", C.c_void_p), ("mat", C.c_void_p), ("ar", C.c_void_p), ("ag", C.c_void_p),
                ("ab", C.c_void_p), ("logits", C.c_void_p)]


class TraceOut(C.Structure):
    _fields_ = [("k", C.c_void_p), ("t01", C.c_void_p), ("pts", C.c_void_p), ("vox", C.c_void_p)]


class Labels(C.Structure):
    _fields_ = [("occ", C.c_void_p), ("t_local", C.c_void_p), ("normal", C.c_void_p), ("albedo", C.c_void_p),
                ("mat", C.c_void_p), ("t_hit", C.c_void_p), ("tri", C.c_void_p), ("k", C.c_void_p)]


class TrainOpts(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("apply_update", C.c_int32), ("products", C.c_int32)]


class TrainStats(C.Structure):
    _fields_ = [("total", C.c_float), ("occ", C.c_float), ("t", C.c_float), ("normal", C.c_float),
                ("albedo", C.c_float), ("mat", C.c_float), ("step", C.c_int64)]


class ReqStats(C.Structure):
    _fields_ = [("submit_us", C.c_double), ("start_us", C.c_double), ("done_us", C.c_double),
                ("gpu_ms", C.c_double), ("n_rays", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("ms_trace", C.c_float), ("ms_group", C.c_float), ("ms_encode", C.c_float), ("ms_mlp", C.c_float),
                ("ms_total", C.c_float), ("n_rays", C.c_int64), ("n_live", C.c_int64), ("n_points", C.c_int64),
                ("launches", C.c_int32)]


# every entry point of include/lsnif.h with its ctypes signature
_P, _I, _I64, _U32, _U64, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t
SIGNATURES = {
    "lsnif_create": (_I, [C.POINTER(_P), _I, _SZ]),
    "lsnif_destroy": (_I, [_P]),
    "lsnif_last_error": (C.c_char_p, []),
    "lsnif_version": (_I, []),
    "lsnif_check": (_I, [_P, _P]),
    "lsnif_load_object": (_I, [_P, C.POINTER(ObjectDesc), C.POINTER(_U32)]),
    "lsnif_save_object": (_I, [_P, _U32, _P, C.POINTER(_SZ)]),
    "lsnif_unload_object": (_I, [_P, _U32]),
    "lsnif_get_object_info": (_I, [_P, _U32, C.POINTER(ObjectInfo)]),
    "lsnif_read_params": (_I, [_P, _U32, _I, _P, _SZ]),
    "lsnif_write_params": (_I, [_P, _U32, _I, _P, _SZ]),
    "lsnif_query_rays": (_I, [_P, C.POINTER(Rays), C.POINTER(Hits), _I, _P]),
    "lsnif_query_rays_host": (_I, [_P, C.POINTER(Rays), C.POINTER(Hits), _I, _P]),
    "lsnif_query_rays_noalloc": (_I, [_P, C.POINTER(Rays), C.POINTER(Hits), _P]),
    "lsnif_query_scene": (_I, [_P, C.POINTER(Rays), C.POINTER(Instance), _I, C.POINTER(Hits), _P, _I, _P]),
    "lsnif_bounce_rays": (_I, [_P, C.POINTER(Rays), C.POINTER(Hits), _P, C.c_float, _P, _P]),
    "lsnif_raster_gbuffer": (_I, [_P, C.POINTER(Camera), C.POINTER(Instance), _I, C.POINTER(GBufferS), _P]),
    "lsnif_bvh_build_host": (_I, [_P, C.c_int64, _P, C.c_int64, _P, C.POINTER(C.c_int64), _P, C.POINTER(_I)]),
    "lsnif_occupancy_distance_host": (_I, [_P, _I, _I, _P]),
    "lsnif_trace": (_I, [_P, C.POINTER(Rays), C.POINTER(TraceOut), _P]),
    "lsnif_encode": (_I, [_P, _U32, _P, _I64, _P, _I, _P]),
    "lsnif_corner_indices": (_I, [_P, _U32, _P, _I64, _P, _P]),
    "lsnif_mlp": (_I, [_P, _U32, _P, _I64, _P, _I, _P]),
    "lsnif_set_graph_mode": (_I, [_P, _I]),
    "lsnif_variant_count": (_I, []),
    "lsnif_variant_shape": (_I, [_I, C.POINTER(_I), C.POINTER(_I)]),
    "lsnif_set_variant": (_I, [_P, _I]),
    "lsnif_variant8_count": (_I, []),
    "lsnif_variant8_shape": (_I, [_I, C.POINTER(_I), C.POINTER(_I)]),
    "lsnif_set_variant8": (_I, [_P, _I]),
    "lsnif_autotune": (_I, [_P, C.POINTER(Rays), _I, _P, C.POINTER(_I)]),
    "lsnif_set_trace_mode": (_I, [_P, _I]),
    "lsnif_get_tuning": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "lsnif_set_group_mode": (_I, [_P, _I]),
    "lsnif_make_training_rays": (_I, [_P, _U32, _P, _I64, _I64, _P, _P, _P]),
    "lsnif_label_rays": (_I, [_P, C.POINTER(Rays), C.POINTER(Labels), _P]),
    "lsnif_train_step": (_I, [_P, C.POINTER(Rays), C.POINTER(Labels), C.POINTER(TrainOpts), C.POINTER(TrainStats),
                              _P]),
    "lsnif_submit": (_I, [_P, C.POINTER(Rays), C.POINTER(Hits), _I, _P, C.POINTER(_U64)]),
    "lsnif_poll": (_I, [_P, _U64, _I64, C.POINTER(ReqStats)]),
    "lsnif_pending": (_I64, [_P]),
    "lsnif_set_profiling": (_I, [_P, _I]),
    "lsnif_last_profile": (_I, [_P, C.POINTER(Profile)]),
    "lsnif_gather_rate": (_I, [_P, _U32, _I64, _P, C.POINTER(C.c_double)]),
    "lsnif_set_host_mode": (_I, [_P, _I]),
    "lsnif_device_bytes": (_SZ, [_P]),
    "lsnif_debug_fail_alloc_after": (_I, [_P, _I64]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblsnif.so and attach signatures. Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"LSNIF CUDA library not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def last_error() -> str:
    return load_library().lsnif_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise LsnifError(rc, last_error())
    return rc


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to the library must be contiguous"
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


BVH_NODE = np.dtype([("lo", np.float32, 3), ("a", np.int32), ("hi", np.float32, 3), ("n", np.int32)])


def bvh_build_host(verts, tris):
    """The mesh objects' BVH builder run on the host (no GPU): returns
    (nodes as a BVH_NODE array, order, depth)."""
    lib = load_library()
    v = np.ascontiguousarray(verts, np.float32)
    t = np.ascontiguousarray(tris, np.int32)
    nt = t.shape[0]
    nodes = np.zeros(max(2 * nt - 1, 1), BVH_NODE)
    order = np.zeros(nt, np.int32)
    nn, depth = C.c_int64(), _I()
    _check(lib.lsnif_bvh_build_host(_ptr(v), v.shape[0], _ptr(t), nt, nodes.ctypes.data, C.byref(nn), _ptr(order),
                                    C.byref(depth)))
    return nodes[:nn.value], order, depth.value


def occupancy_distance_host(occ_words, V: int, cap: int) -> np.ndarray:
    """The traversal's occupancy distance field computed on the host (no
    GPU): uint8 array of V^3 in voxel order."""
    lib = load_library()
    w = np.ascontiguousarray(occ_words, np.uint32)
    out = np.zeros(V ** 3, np.uint8)
    _check(lib.lsnif_occupancy_distance_host(_ptr(w), V, cap, _ptr(out)))
    return out


def cfg_struct(cfg) -> Config:
    """An inputs.Config (or any object with the same fields) -> Config."""
    return Config(cfg.V, cfg.H, cfg.L, cfg.F, cfg.log2_T, cfg.N_min, cfg.N_max, cfg.n_hidden, cfg.width, cfg.n_mat,
                  cfg.activation, float(cfg.table_init), int(cfg.seed))


def rays_struct(rays, obj=None, single_obj: int = 0) -> Rays:
    """rays: (8, n) float32 contiguous tensor/array (ox oy oz dx dy dz tmin tmax rows)."""
    n = int(rays.shape[1])
    base = _ptr(rays)
    row = 4 * n
    return Rays(*[base + i * row for i in range(8)], _ptr(obj), int(single_obj), n)


@dataclass
class QueryResult:
    hit: object
    t: object
    normal: object     # (3, n)
    mat: object
    albedo: object     # (3, n)
    logits: object | None


@dataclass
class GBuffer:
    hit: object        # (h, w) uint8
    shape: object      # (h, w) int32 instance index, -1 background
    prim: object       # (h, w) int32 triangle index, -1 background
    u: object
    v: object
    dist: object       # (h, w) camera distance, inf background
    normal: object | None   # (3, h, w)


class Context:
    """An LSNIF context on one CUDA device (lsnif_create / lsnif_destroy)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib.lsnif_create(C.byref(h), device, budget_bytes))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.lsnif_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- objects -------------------------------------------------------------
    def load_object(self, mesh=None, cfg=None, tables=None, mlp=None, keep_mesh: bool = False,
                    blob: bytes | None = None, bvh_below_faces: int = 0) -> int:
        """bvh_below_faces: meshes with fewer triangles stay mesh objects
        (triangles + BVH, exact answers) instead of becoming LSNIF objects."""
        d = ObjectDesc()
        d.bvh_below_faces = int(bvh_below_faces)
        keep = []
        if blob is not None:
            buf = C.create_string_buffer(blob, len(blob))
            keep.append(buf)
            d.blob = C.cast(buf, C.c_void_p)
            d.blob_len = len(blob)
        else:
            d.cfg = cfg_struct(cfg)
            v = np.ascontiguousarray(mesh.verts, np.float32)
            t = np.ascontiguousarray(mesh.tris, np.int32)
            vn = np.ascontiguousarray(mesh.vnormals, np.float32)
            tm = np.ascontiguousarray(mesh.tri_mat, np.int32)
            al = np.ascontiguousarray(mesh.albedo, np.float32)
            keep += [v, t, vn, tm, al]
            d.mesh = Mesh(_ptr(v), _ptr(t), _ptr(vn), _ptr(tm), _ptr(al), v.shape[0], t.shape[0])
            if tables is not None:
                tb = np.ascontiguousarray(tables, np.float32)
                keep.append(tb)
                d.tables = _ptr(tb)
            if mlp is not None:
                mp = np.ascontiguousarray(mlp, np.float32)
                keep.append(mp)
                d.mlp = _ptr(mp)
            d.keep_mesh = 1 if keep_mesh else 0
        out = C.c_uint32()
        _check(self.lib.lsnif_load_object(self.h, C.byref(d), C.byref(out)))
        return out.value

    def load_mesh(self, mesh, n_mat: int | None = None) -> int:
        """A mesh object: the triangles and a BVH, answered exactly."""
        from types import SimpleNamespace
        cfg = SimpleNamespace(V=0, H=0, L=0, F=0, log2_T=0, N_min=0, N_max=0, n_hidden=0, width=0,
                              n_mat=int(mesh.n_mat if n_mat is None else n_mat), activation=0, table_init=0.0,
                              seed=0)
        return self.load_object(mesh, cfg, bvh_below_faces=int(mesh.tris.shape[0]) + 1)

    def unload_object(self, obj: int):
        _check(self.lib.lsnif_unload_object(self.h, obj))

    def save_object(self, obj: int) -> bytes:
        n = C.c_size_t(0)
        _check(self.lib.lsnif_save_object(self.h, obj, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.lib.lsnif_save_object(self.h, obj, C.cast(buf, C.c_void_p), C.byref(n)))
        return buf.raw[: n.value]

    def object_info(self, obj: int) -> ObjectInfo:
        info = ObjectInfo()
        _check(self.lib.lsnif_get_object_info(self.h, obj, C.byref(info)))
        return info

    def read_params(self, obj: int, which: int) -> np.ndarray:
        info = self.object_info(obj)
        c = info.cfg
        if which == PARAM_OCCUPANCY:
            arr = np.zeros((c.V ** 3 + 31) // 32, np.uint32)
        elif which in (PARAM_TABLES, PARAM_GRAD_TABLES):
            arr = np.zeros((c.L, 1 << c.log2_T, c.F), np.float32)
        else:
            arr = np.zeros(info.n_params_mlp, np.float32)
        _check(self.lib.lsnif_read_params(self.h, obj, which, _ptr(arr), arr.nbytes))
        return arr

    def write_params(self, obj: int, which: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, np.float32)
        _check(self.lib.lsnif_write_params(self.h, obj, which, _ptr(a), a.nbytes))

    # ---- query -------------------------------------------------------------------
    def _alloc_hits(self, n: int, n_out: int, want_logits: bool, device: bool = True):
        import torch
        kw = dict(device=f"cuda:{self.device}") if device else dict(pin_memory=True)
        hit = torch.zeros(n, dtype=torch.uint8, **kw)
        t = torch.zeros(n, dtype=torch.float32, **kw)
        nrm = torch.zeros((3, n), dtype=torch.float32, **kw)
        mat = torch.zeros(n, dtype=torch.int32, **kw)
        alb = torch.zeros((3, n), dtype=torch.float32, **kw)
        lg = torch.zeros((n, n_out), dtype=torch.float32, **kw) if want_logits else None
        return QueryResult(hit, t, nrm, mat, alb, lg)

    @staticmethod
    def hits_struct(r: QueryResult) -> Hits:
        n = r.t.shape[0]
        nrm, alb = _ptr(r.normal), _ptr(r.albedo)
        return Hits(_ptr(r.hit), _ptr(r.t), nrm, nrm and nrm + 4 * n, nrm and nrm + 8 * n,
                    _ptr(r.mat), alb, alb and alb + 4 * n, alb and alb + 8 * n, _ptr(r.logits))

    def query_rays(self, rays, obj: int = 0, obj_per_ray=None, precision: int = BF16_FUSED,
                   logits: bool = False, out: QueryResult | None = None, stream=None) -> QueryResult:
        """rays: (8, n) float32 CUDA tensor; results are CUDA tensors."""
        n = int(rays.shape[1])
        n_out = 8 + self.object_info(obj).cfg.n_mat if (logits and obj) else 0
        res = out if out is not None else self._alloc_hits(n, n_out, logits)
        rs = rays_struct(rays, obj_per_ray, obj)
        hs = self.hits_struct(res)
        _check(self.lib.lsnif_query_rays(self.h, C.byref(rs), C.byref(hs), precision, _stream(stream)))
        return res

    def query_rays_host(self, rays, obj: int = 0, obj_per_ray=None, precision: int = BF16_FUSED,
                        out: QueryResult | None = None, stream=None) -> QueryResult:
        """rays: (8, n) float32 host tensor (pinned is faster); results in host tensors."""
        n = int(rays.shape[1])
        res = out if out is not None else self._alloc_hits(n, 0, False, device=False)
        rs = rays_struct(rays, obj_per_ray, obj)
        hs = self.hits_struct(res)
        _check(self.lib.lsnif_query_rays_host(self.h, C.byref(rs), C.byref(hs), precision, _stream(stream)))
        return res

    def query_rays_noalloc(self, rays, out: QueryResult, obj: int = 0, obj_per_ray=None, stream=None):
        """BF16 fused query that allocates nothing (its scratch is a static
        device array); `out` must be preallocated (see lsnif.h)."""
        rs = rays_struct(rays, obj_per_ray, obj)
        hs = self.hits_struct(out)
        _check(self.lib.lsnif_query_rays_noalloc(self.h, C.byref(rs), C.byref(hs), _stream(stream)))
        return out

    def query_scene(self, rays, instances, precision: int = BF16_FUSED, stream=None):
        """World rays (8, n) CUDA tensor against instances [(handle, A (3x3),
        b (3,)), ...] with p_obj = A p + b. Returns (QueryResult, instance
        index per ray, -1 on a miss)."""
        import torch
        n = int(rays.shape[1])
        res = self._alloc_hits(n, 0, False)
        inst = torch.full((n,), -1, dtype=torch.int32, device=rays.device)
        arr = self._instances(instances)
        rs = rays_struct(rays)
        hs = self.hits_struct(res)
        _check(self.lib.lsnif_query_scene(self.h, C.byref(rs), arr, len(instances), C.byref(hs), _ptr(inst),
                                          precision, _stream(stream)))
        return res, inst

    @staticmethod
    def _instances(instances):
        arr = (Instance * len(instances))()
        for k, (h, A, b) in enumerate(instances):
            m = np.concatenate([np.asarray(A, np.float64), np.asarray(b, np.float64)[:, None]], 1)
            arr[k].obj = int(h)
            arr[k].world_to_obj[:] = [float(x) for x in m.astype(np.float32).reshape(-1)]
        return arr

    def raster_gbuffer(self, eye, forward, right, up, tan_half_fov: float, width: int, height: int, instances,
                       normals: bool = True, out: GBuffer | None = None, stream=None) -> GBuffer:
        """Primary-ray G-buffer of instances [(handle, A, b), ...] (objects
        loaded with keep_mesh) seen by a pinhole camera; CUDA tensors of
        height x width (normal: 3 x height x width)."""
        import torch
        if out is None:
            kw = dict(device=f"cuda:{self.device}")
            n = (height, width)
            out = GBuffer(torch.zeros(n, dtype=torch.uint8, **kw), torch.zeros(n, dtype=torch.int32, **kw),
                          torch.zeros(n, dtype=torch.int32, **kw), torch.zeros(n, dtype=torch.float32, **kw),
                          torch.zeros(n, dtype=torch.float32, **kw), torch.zeros(n, dtype=torch.float32, **kw),
                          torch.zeros((3,) + n, dtype=torch.float32, **kw) if normals else None)
        cam = Camera()
        cam.eye[:] = [float(x) for x in np.asarray(eye, np.float32)]
        cam.forward[:] = [float(x) for x in np.asarray(forward, np.float32)]
        cam.right[:] = [float(x) for x in np.asarray(right, np.float32)]
        cam.up[:] = [float(x) for x in np.asarray(up, np.float32)]
        cam.tan_half_fov = float(np.float32(tan_half_fov))
        cam.width, cam.height = int(width), int(height)
        npx = width * height
        nrm = _ptr(out.normal) if out.normal is not None else None
        g = GBufferS(_ptr(out.hit), _ptr(out.shape), _ptr(out.prim), _ptr(out.u), _ptr(out.v), _ptr(out.dist),
                     nrm, nrm + 4 * npx if nrm else None, nrm + 8 * npx if nrm else None)
        arr = self._instances(instances)
        _check(self.lib.lsnif_raster_gbuffer(self.h, C.byref(cam), arr, len(instances), C.byref(g),
                                             _stream(stream)))
        return out

    def bounce_rays(self, rays, res: QueryResult, u, eps: float, stream=None):
        """Next-bounce rays (8, n) from world rays and their query results;
        u: (n, 2) uniforms, all CUDA tensors."""
        import torch
        n = int(rays.shape[1])
        out = torch.empty((8, n), dtype=torch.float32, device=rays.device)
        rs = rays_struct(rays)
        hs = self.hits_struct(res)
        _check(self.lib.lsnif_bounce_rays(self.h, C.byref(rs), C.byref(hs), _ptr(u), float(eps), _ptr(out),
                                          _stream(stream)))
        return out

    def trace(self, rays, obj: int, stream=None):
        import torch
        info = self.object_info(obj)
        n, H = int(rays.shape[1]), info.cfg.H
        dev = rays.device
        k = torch.zeros(n, dtype=torch.int32, device=dev)
        t01 = torch.zeros((n, 2), dtype=torch.float32, device=dev)
        pts = torch.zeros((n, H, 3), dtype=torch.float32, device=dev)
        vox = torch.zeros((n, H // 2), dtype=torch.int32, device=dev)
        to = TraceOut(_ptr(k), _ptr(t01), _ptr(pts), _ptr(vox))
        rs = rays_struct(rays, None, obj)
        _check(self.lib.lsnif_trace(self.h, C.byref(rs), C.byref(to), _stream(stream)))
        return k, t01, pts, vox

    def encode(self, obj: int, pts, precision: int = FP32_PLAIN, stream=None):
        import torch
        c = self.object_info(obj).cfg
        n = int(pts.shape[0])
        feats = torch.zeros((n, c.L, c.F), dtype=torch.float32, device=pts.device)
        _check(self.lib.lsnif_encode(self.h, obj, _ptr(pts), n, _ptr(feats), precision, _stream(stream)))
        return feats

    def corner_indices(self, obj: int, pts, stream=None):
        import torch
        c = self.object_info(obj).cfg
        n = int(pts.shape[0])
        out = torch.zeros((n, c.L, 8), dtype=torch.int32, device=pts.device)
        _check(self.lib.lsnif_corner_indices(self.h, obj, _ptr(pts), n, _ptr(out), _stream(stream)))
        return out

    def mlp(self, obj: int, X, precision: int = FP32_PLAIN, stream=None):
        import torch
        c = self.object_info(obj).cfg
        n = int(X.shape[0])
        Z = torch.zeros((n, 8 + c.n_mat), dtype=torch.float32, device=X.device)
        _check(self.lib.lsnif_mlp(self.h, obj, _ptr(X), n, _ptr(Z), precision, _stream(stream)))
        return Z

    # ---- autotuning -------------------------------------------------------------
    @staticmethod
    def variants() -> list[tuple[int, int]]:
        lib = load_library()
        out = []
        for v in range(lib.lsnif_variant_count()):
            t, l = C.c_int(), C.c_int()
            _check(lib.lsnif_variant_shape(v, C.byref(t), C.byref(l)))
            out.append((t.value, l.value))
        return out

    @staticmethod
    def variants8() -> list[tuple[int, int]]:
        lib = load_library()
        out = []
        for v in range(lib.lsnif_variant8_count()):
            t, l = C.c_int(), C.c_int()
            _check(lib.lsnif_variant8_shape(v, C.byref(t), C.byref(l)))
            out.append((t.value, l.value))
        return out

    def set_variant8(self, v: int):
        _check(self.lib.lsnif_set_variant8(self.h, v))

    def set_graph_mode(self, on: bool):
        _check(self.lib.lsnif_set_graph_mode(self.h, 1 if on else 0))

    def set_variant(self, v: int):
        _check(self.lib.lsnif_set_variant(self.h, v))

    def set_trace_mode(self, mode: int):
        _check(self.lib.lsnif_set_trace_mode(self.h, mode))

    def set_group_mode(self, mode: int):
        _check(self.lib.lsnif_set_group_mode(self.h, mode))

    def tuning(self) -> tuple[int, int, int]:
        """(fused-kernel variant, traversal kernel, grouping)"""
        v, t, g = C.c_int(), C.c_int(), C.c_int()
        _check(self.lib.lsnif_get_tuning(self.h, C.byref(v), C.byref(t), C.byref(g)))
        return v.value, t.value, g.value

    def autotune(self, rays, obj: int = 0, obj_per_ray=None, reps: int = 3, stream=None) -> int:
        rs = rays_struct(rays, obj_per_ray, obj)
        ch = C.c_int(-1)
        _check(self.lib.lsnif_autotune(self.h, C.byref(rs), reps, _stream(stream), C.byref(ch)))
        return ch.value

    # ---- training --------------------------------------------------------------
    def make_training_rays(self, obj: int, u, n_outside: int, stream=None):
        import torch
        n = int(u.shape[0])
        rays = torch.zeros((8, n), dtype=torch.float32, device=u.device)
        surf = torch.zeros(n, dtype=torch.uint8, device=u.device)
        _check(self.lib.lsnif_make_training_rays(self.h, obj, _ptr(u), n, n_outside, _ptr(rays), _ptr(surf),
                                                 _stream(stream)))
        return rays, surf

    def label_rays(self, rays, obj: int, stream=None) -> dict:
        import torch
        n = int(rays.shape[1])
        dev = rays.device
        lab = dict(occ=torch.zeros(n, device=dev), t_local=torch.zeros(n, device=dev),
                   normal=torch.zeros((n, 3), device=dev), albedo=torch.zeros((n, 3), device=dev),
                   mat=torch.zeros(n, dtype=torch.int32, device=dev), t_hit=torch.zeros(n, device=dev),
                   tri=torch.zeros(n, dtype=torch.int32, device=dev), k=torch.zeros(n, dtype=torch.int32, device=dev))
        ls = self.labels_struct(lab)
        rs = rays_struct(rays, None, obj)
        _check(self.lib.lsnif_label_rays(self.h, C.byref(rs), C.byref(ls), _stream(stream)))
        return lab

    @staticmethod
    def labels_struct(lab: dict) -> Labels:
        return Labels(*[_ptr(lab.get(k)) for k in ("occ", "t_local", "normal", "albedo", "mat", "t_hit", "tri", "k")])

    def train_step(self, rays, lab: dict, obj: int, lr: float = 0.01, apply_update: bool = True,
                   stats: bool = True, stream=None, products: int = 0) -> TrainStats | None:
        """products: TRAIN_TENSOR_CORES (0) or TRAIN_FP32_SIMT (1)."""
        rs = rays_struct(rays, None, obj)
        ls = self.labels_struct(lab)
        opts = TrainOpts(lr, 0.9, 0.999, 1e-8, 1 if apply_update else 0, products)
        st = TrainStats()
        _check(self.lib.lsnif_train_step(self.h, C.byref(rs), C.byref(ls), C.byref(opts),
                                         C.byref(st) if stats else None, _stream(stream)))
        return st if stats else None

    # ---- serving -----------------------------------------------------------------
    def submit(self, rays, res: QueryResult, obj: int = 0, obj_per_ray=None, precision: int = BF16_FUSED,
               stream=None) -> int:
        """Queue a query; it runs after the work already enqueued on `stream`
        (default: the current stream), where the buffers were produced."""
        rs = rays_struct(rays, obj_per_ray, obj)
        hs = self.hits_struct(res)
        tk = C.c_uint64()
        _check(self.lib.lsnif_submit(self.h, C.byref(rs), C.byref(hs), precision, _stream(stream), C.byref(tk)))
        return tk.value

    def poll(self, ticket: int, timeout_us: int = 0):
        st = ReqStats()
        rc = self.lib.lsnif_poll(self.h, ticket, timeout_us, C.byref(st))
        if rc == PENDING:
            return None
        _check(rc)
        return st

    def pending(self) -> int:
        return int(self.lib.lsnif_pending(self.h))

    # ---- measurement / checks ---------------------------------------------------
    def set_profiling(self, on: bool):
        _check(self.lib.lsnif_set_profiling(self.h, 1 if on else 0))

    def last_profile(self) -> Profile:
        p = Profile()
        _check(self.lib.lsnif_last_profile(self.h, C.byref(p)))
        return p

    def set_host_mode(self, mode: int):
        """HOST_STAGED (0) or HOST_DIRECT (1) for query_rays_host (see lsnif_set_host_mode)."""
        _check(self.lib.lsnif_set_host_mode(self.h, mode))

    def gather_rate(self, obj: int, loads: int = 0, stream=None) -> float:
        """Random 8-byte loads per second over the object's FP16 tables (the
        gather's request ceiling; see lsnif_gather_rate)."""
        r = C.c_double()
        _check(self.lib.lsnif_gather_rate(self.h, obj, loads, _stream(stream), C.byref(r)))
        return r.value

    def check(self, stream=None):
        _check(self.lib.lsnif_check(self.h, _stream(stream)))

    def device_bytes(self) -> int:
        return int(self.lib.lsnif_device_bytes(self.h))

    def debug_fail_alloc_after(self, n: int):
        _check(self.lib.lsnif_debug_fail_alloc_after(self.h, n))
