"""FP64 oracle for the LSNIF per-ray query and its training step.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It never imports the
product package's CUDA binding and shares no code with it; the two meet only
in the seeded inputs of ``paper_2504_21627_gb300.inputs``.

The heavy geometric loops live in ``lsnif_oracle.c`` (loaded through ctypes);
the network, decode, losses, backward pass and Adam are plain float64 numpy.
Each function names the passage of the paper (Fujieda et al., LSNIF, 2025)
that it restates.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test to a
closed form, a brute-force alternative, a library routine or a value printed
in the paper. Nothing in this module is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

#: distance (unit-cube units) within which a voxel face makes a ray "near-face"
NEAR_FACE_EPS = 1e-5


def build(force: bool = False) -> str:
    """Compile lsnif_oracle.c into oracle/_build/liboracle.so with gcc."""
    src = os.path.join(_HERE, "lsnif_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fvisibility=hidden", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_bbox.argtypes = [P, i64, P, P]
        L.orc_voxelize.argtypes = [P, P, i64, P, P, i32, P]
        L.orc_tri_box_overlap.argtypes = [P, dbl, P, P, P]
        L.orc_tri_box_overlap.restype = i32
        L.orc_level_res.argtypes = [i32, i32, i32, P]
        L.orc_ray_segments.argtypes = [P, i64, P, P, i32, P, i64, i32, dbl, P, P, P, P, P]
        L.orc_hash.argtypes = [i64, i64, i64, i32]
        L.orc_hash.restype = ctypes.c_uint32
        L.orc_encode.argtypes = [P, i64, P, i32, i32, i32, P, P, P, P]
        L.orc_encode_backward.argtypes = [P, i64, P, i32, i32, i32, P, P]
        L.orc_judge.argtypes = [P, i64, P, P, i64, P, P, P, P]
        L.orc_cast64.argtypes = [P, P, i64, P, P, i64, P, P, P, P]
        L.orc_threads.argtypes = [i32]
        L.orc_threads.restype = i32
        _lib = L
    return _lib


def threads(n: int = 0) -> int:
    """Host threads of the C loops (n > 0 sets them); returns the previous
    count. Timing only: every output comes from one loop iteration."""
    return int(lib().orc_threads(n))


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# geometry: bbox, voxelization, level resolutions
# --------------------------------------------------------------------------

def bbox(verts: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Object AABB (Sec. 3.1 local frame), FP32, thin axes widened."""
    v = _c(verts, np.float32)
    lo = np.zeros(3, np.float32)
    hi = np.zeros(3, np.float32)
    lib().orc_bbox(_p(v), v.shape[0], _p(lo), _p(hi))
    return lo, hi


def voxelize(verts, tris, bmin, bmax, V: int) -> np.ndarray:
    """Surface-only binary occupancy (Sec. 3.1), uint8 [V^3], index (z*V+y)*V+x."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    occ = np.zeros(V * V * V, np.uint8)
    lib().orc_voxelize(_p(v), _p(t), t.shape[0], _p(_c(bmin, np.float32)), _p(_c(bmax, np.float32)),
                       V, _p(occ))
    return occ


def tri_box_overlap(center, half, u0, u1, u2) -> bool:
    return bool(lib().orc_tri_box_overlap(_p(_c(center, np.float64)), float(half), _p(_c(u0, np.float64)),
                                          _p(_c(u1, np.float64)), _p(_c(u2, np.float64))))


def level_res(N_min: int, N_max: int, L: int) -> np.ndarray:
    """Per-level lattice resolution, geometric from N_min to N_max (Sec. 3.2)."""
    out = np.zeros(L, np.int32)
    lib().orc_level_res(N_min, N_max, L, _p(out))
    return out


def occupancy_bits(occ: np.ndarray) -> np.ndarray:
    """uint8 occupancy -> packed little-endian uint32 words (bit i of word i>>5)."""
    n = occ.size
    words = np.zeros((n + 31) // 32, np.uint32)
    idx = np.nonzero(occ)[0]
    np.bitwise_or.at(words, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return words


# --------------------------------------------------------------------------
# the object as the oracle sees it
# --------------------------------------------------------------------------

@dataclass
class OracleObject:
    cfg: object              # inputs.Config
    bmin: np.ndarray
    bmax: np.ndarray
    occ: np.ndarray          # uint8 [V^3]
    res: np.ndarray          # int32 [L]
    tables: np.ndarray       # float64 (L, T, F)
    weights: list            # [(W (out,in) f64, b f64)]

    @property
    def occ_list(self) -> np.ndarray:
        return np.nonzero(self.occ)[0].astype(np.int32)


def build_object(mesh, cfg, params) -> OracleObject:
    lo, hi = bbox(mesh.verts)
    occ = voxelize(mesh.verts, mesh.tris, lo, hi, cfg.V)
    return OracleObject(cfg, lo, hi, occ, level_res(cfg.N_min, cfg.N_max, cfg.L),
                        params.tables.astype(np.float64),
                        [(W.astype(np.float64), b.astype(np.float64)) for W, b in params.weights])


# --------------------------------------------------------------------------
# traversal and points (Fig. 2, Sec. 3.1, Sec. 5.1)
# --------------------------------------------------------------------------

@dataclass
class Segments:
    k: np.ndarray        # int32 (n,) kept occupied voxels
    t01: np.ndarray      # float64 (n, 2) clipped cube interval, NaN on a miss
    pts: np.ndarray      # float64 (n, H, 3) unit-cube points, zero beyond 2k
    vox: np.ndarray      # int32 (n, H/2) voxel ids, -1 beyond k
    near: np.ndarray     # bool (n,) near-face rays


def ray_segments(obj: OracleObject, rays: np.ndarray, eps: float = NEAR_FACE_EPS) -> Segments:
    """Occupied-voxel segments and their boundary points, by brute force."""
    r = _c(np.asarray(rays, np.float32).T, np.float32)  # (n, 8)
    n = r.shape[0]
    H = obj.cfg.H
    ol = _c(obj.occ_list, np.int32)
    k = np.zeros(n, np.int32)
    t01 = np.zeros((n, 2))
    pts = np.zeros((n, H, 3))
    vox = np.zeros((n, H // 2), np.int32)
    flag = np.zeros(n, np.uint8)
    lib().orc_ray_segments(_p(r), n, _p(obj.bmin), _p(obj.bmax), obj.cfg.V, _p(ol), ol.size, H, eps,
                           _p(k), _p(t01), _p(pts), _p(vox), _p(flag))
    return Segments(k, t01, pts, vox, flag.astype(bool))


# --------------------------------------------------------------------------
# sparse hash-grid encoding (Sec. 3.2)
# --------------------------------------------------------------------------

def hash_index(x: int, y: int, z: int, log2_T: int) -> int:
    return int(lib().orc_hash(int(x), int(y), int(z), int(log2_T)))


def encode(pts: np.ndarray, res, F: int, log2_T: int, tables: np.ndarray, debug: bool = False):
    """Trilinear hash-grid features of points (npts, 3) -> (npts, L, F)."""
    p = _c(pts, np.float64).reshape(-1, 3)
    res = _c(res, np.int32)
    L = res.size
    tab = _c(tables, np.float64)
    out = np.zeros((p.shape[0], L, F))
    if debug:
        idx = np.zeros((p.shape[0], L, 8), np.uint32)
        w = np.zeros((p.shape[0], L, 8))
        lib().orc_encode(_p(p), p.shape[0], _p(res), L, F, log2_T, _p(tab), _p(out), _p(idx), _p(w))
        return out, idx, w
    lib().orc_encode(_p(p), p.shape[0], _p(res), L, F, log2_T, _p(tab), _p(out), None, None)
    return out


def encode_backward(pts: np.ndarray, res, F: int, log2_T: int, dout: np.ndarray,
                    grad_tables: np.ndarray) -> None:
    p = _c(pts, np.float64).reshape(-1, 3)
    res = _c(res, np.int32)
    d = _c(dout, np.float64)
    assert grad_tables.dtype == np.float64 and grad_tables.flags["C_CONTIGUOUS"]
    lib().orc_encode_backward(_p(p), p.shape[0], _p(res), res.size, F, log2_T, _p(d), _p(grad_tables))


def features(obj: OracleObject, seg: Segments, tables: np.ndarray | None = None) -> np.ndarray:
    """Concatenated network input (Sec. 3.2): for slot h < 2k the L*F features
    of point h, zeros for empty slots (Sec. 5.1). Shape (n, H*L*F)."""
    cfg = obj.cfg
    tab = obj.tables if tables is None else tables
    n, H = seg.k.size, cfg.H
    live = np.arange(H)[None, :] < 2 * seg.k[:, None]          # (n, H)
    X = np.zeros((n, H, cfg.L, cfg.F))
    if live.any():
        X[live] = encode(seg.pts[live], obj.res, cfg.F, cfg.log2_T, tab)
    return X.reshape(n, H * cfg.L * cfg.F)


# --------------------------------------------------------------------------
# reduced-precision emulation (used to compare the BF16 path decision for
# decision; the network's own arithmetic stays float64)
# --------------------------------------------------------------------------

def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) via float32."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    nan = np.isnan(f)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def split_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two-term bfloat16 form of x: hi = BF16(x), lo = BF16(x - hi), so that
    hi + lo carries about 16 significant bits of x (each rounding as in
    round_bf16, through float32)."""
    x = np.asarray(x, np.float64)
    hi = round_bf16(x)
    return hi, round_bf16(x - hi)


def round_fp16(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


FP16_MAX = 65504.0


def round_fp16_sat(x: np.ndarray) -> np.ndarray:
    """Round to the nearest IEEE binary16 value (ties to even) through
    float32, saturating at +-65504 instead of overflowing to infinity."""
    return round_fp16(np.clip(np.asarray(x, np.float64), -FP16_MAX, FP16_MAX))


E4M3_MAX = 448.0


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """Round to the nearest FP8 E4M3 value (1 sign, 4 exponent bits with bias
    7, 3 mantissa bits; normals down to 2^-6, subnormals in steps of 2^-9,
    largest finite 448), ties to even, saturating: |x| > 448 gives +-448."""
    x = np.asarray(x, np.float64)
    _, e = np.frexp(x)                        # x = m 2^e, 0.5 <= |m| < 1
    q = np.ldexp(1.0, np.maximum(e - 1, -6) - 3)   # spacing of the binade (subnormal spacing below 2^-6)
    r = np.round(x / q) * q                   # np.round: half to even
    return np.clip(np.where(x == 0, 0.0, r), -E4M3_MAX, E4M3_MAX)


def pow2_scale(m: float) -> float:
    """The power of two s with 448 / 2 < s m <= 448 (1 when m is 0): the scale
    that brings a magnitude m to the top binade of E4M3."""
    if not m > 0:
        return 1.0
    _, e = math.frexp(E4M3_MAX / m)           # 448 / m = f 2^e, 0.5 <= f < 1
    return math.ldexp(1.0, e - 1)


def fp8_scales(tables_fp16_max: float, weights) -> tuple[list, list]:
    """Per-layer power-of-two scales of the FP8 network: input scales s_l
    (s_0 from the largest FP16 table value, which bounds every interpolated
    feature; s_{l+1} from the magnitude estimate M_{l+1} = max_j
    (||W_l[j]||_2 M_l + |b_l[j]|), with M_0 the table maximum) and weight
    scales w_l (from max |W_l|). Values beyond the E4M3 range saturate."""
    s, w = [], []
    M = float(tables_fp16_max)
    for W, b in weights:
        W = np.asarray(W, np.float64)
        b = np.asarray(b, np.float64)
        s.append(pow2_scale(M))
        w.append(pow2_scale(float(np.max(np.abs(W))) if W.size else 0.0))
        M = float(np.max(np.sqrt(np.sum(W * W, axis=1)) * M + np.abs(b)))
    return s, w


# --------------------------------------------------------------------------
# network (Sec. 5.1) and decode (Sec. 5.1, Sec. 5.3)
# --------------------------------------------------------------------------

def activation(x: np.ndarray, kind: int) -> np.ndarray:
    return np.maximum(x, 0.0) if kind == 0 else np.where(x > 0, x, 0.01 * x)


def activation_grad(pre: np.ndarray, kind: int) -> np.ndarray:
    return (pre > 0).astype(np.float64) if kind == 0 else np.where(pre > 0, 1.0, 0.01)


def mlp_forward(X: np.ndarray, weights, act: int = 0, precision: str = "f64", keep: bool = False,
                fp8=None):
    """Dense layers, hidden activation `act`, linear output; sums in float64.

    precision='bf16_plain': every matmul operand (inputs, weights, hidden
    activations) is rounded once to bfloat16. precision='bf16': the first
    layer is the same, and every later layer takes its input activations
    and its weights in the two-term form of split_bf16 and forms
    hi_a.hi_w + hi_a.lo_w + lo_a.hi_w (the lo_a.lo_w product, about 2^-16
    of the rest, is left out). precision='fp16' rounds every operand once
    to binary16 with saturation. precision='fp8' (fp8 = (s, w) from
    fp8_scales): every layer multiplies round_e4m3(s_l h) by
    round_e4m3(w_l W_l) and divides the sum by s_l w_l before the bias."""
    h = np.asarray(X, np.float64)
    rnd = {"bf16": round_bf16, "bf16_plain": round_bf16, "fp16": round_fp16_sat}.get(precision)
    if rnd is not None:
        h = rnd(h)
    cache = []
    for i, (W, b) in enumerate(weights):
        bq = np.asarray(b, np.float64)
        W = np.asarray(W, np.float64)
        if precision == "fp8":
            s, w = fp8[0][i], fp8[1][i]
            z = (round_e4m3(h * s) @ round_e4m3(W * w).T) / (s * w) + bq
        elif precision == "bf16" and i > 0:
            h_hi, h_lo = h
            W_hi, W_lo = split_bf16(W)
            z = h_hi @ W_hi.T + h_hi @ W_lo.T + h_lo @ W_hi.T + bq
            h = h_hi + h_lo
        else:
            Wq = rnd(W) if rnd is not None else W
            z = h @ Wq.T + bq
        cache.append((h, z))
        if i < len(weights) - 1:
            h = activation(z, act)
            if precision == "bf16":
                h = split_bf16(h)
            elif rnd is not None:
                h = rnd(h)
        else:
            h = z
    return (h, cache) if keep else h


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * np.asarray(x, np.float64)))


@dataclass
class Hits:
    hit: np.ndarray      # bool
    t: np.ndarray
    normal: np.ndarray   # (n, 3)
    mat: np.ndarray      # int32
    albedo: np.ndarray   # (n, 3)
    logits: np.ndarray   # (n, 8 + n_mat), NaN rows for rays that skip the network
    live: np.ndarray     # bool: ray reached the network (k > 0)


def decode(Z: np.ndarray, t01: np.ndarray, tmin: np.ndarray, tmax: np.ndarray) -> dict:
    """Output layout [occ, t, nx, ny, nz, r, g, b, mat_0..]. Occlusion = z0 > 0
    (sigmoid >= 0.5 threshold, Sec. 5.3); hit distance local to the AABB
    interval, t = t0 + sigmoid(z1)(t1 - t0); normal = z[2:5] normalised (zero
    stays zero); albedo = sigmoid; material = argmax (lowest index on ties);
    a hit also needs tmin <= t <= tmax."""
    occ = Z[:, 0] > 0
    t = t01[:, 0] + sigmoid(Z[:, 1]) * (t01[:, 1] - t01[:, 0])
    nz = Z[:, 2:5]
    nn = np.linalg.norm(nz, axis=1, keepdims=True)
    normal = np.where(nn > 0, nz / np.where(nn > 0, nn, 1.0), 0.0)
    albedo = sigmoid(Z[:, 5:8])
    mat = np.argmax(Z[:, 8:], axis=1).astype(np.int32)
    hit = occ & (t >= tmin) & (t <= tmax)
    return dict(hit=hit, t=t, normal=normal, albedo=albedo, mat=mat)


def query(obj: OracleObject, rays: np.ndarray, precision: str = "f64", seg: Segments | None = None):
    """The per-ray query of Fig. 2 end to end. Rays that meet no occupied
    voxel never reach the network: hit 0, t inf, normal 0, mat -1."""
    cfg = obj.cfg
    seg = ray_segments(obj, rays) if seg is None else seg
    n = seg.k.size
    live = seg.k > 0
    tables = round_fp16(obj.tables) if precision in ("bf16", "bf16_plain", "fp16", "fp8") else obj.tables
    fp8 = fp8_scales(float(np.max(np.abs(tables))), obj.weights) if precision == "fp8" else None
    out = Hits(np.zeros(n, bool), np.full(n, np.inf), np.zeros((n, 3)), np.full(n, -1, np.int32),
               np.zeros((n, 3)), np.full((n, cfg.n_out), np.nan), live)
    if live.any():
        sub = Segments(seg.k[live], seg.t01[live], seg.pts[live], seg.vox[live], seg.near[live])
        X = features(obj, sub, tables)
        Z = mlp_forward(X, obj.weights, cfg.activation, precision, fp8=fp8)
        rr = np.asarray(rays, np.float64)[:, live]
        dec = decode(Z, sub.t01, rr[6], rr[7])
        out.hit[live] = dec["hit"]
        out.t[live] = dec["t"]
        out.normal[live] = dec["normal"]
        out.mat[live] = dec["mat"]
        out.albedo[live] = dec["albedo"]
        out.logits[live] = Z
    return out, seg


# --------------------------------------------------------------------------
# instanced scenes: world rays against transformed objects (Sec. 4, Sec. 6)
# --------------------------------------------------------------------------

@dataclass
class Instance:
    obj: int           # index into the list of objects
    A: np.ndarray      # (3, 3) world -> object linear part
    b: np.ndarray      # (3,) translation: p_obj = A p_world + b


def to_object_frame(rays: np.ndarray, inst: Instance) -> np.ndarray:
    """World rays in an instance's object frame, FP64: o' = A o + b, d' = A d.
    The ray parameter t is unchanged, so tmin and tmax carry over."""
    r = np.asarray(rays, np.float64)
    out = np.empty_like(r)
    out[0:3] = inst.A @ r[0:3] + inst.b[:, None]
    out[3:6] = inst.A @ r[3:6]
    out[6:8] = r[6:8]
    return out


def pixel_rays(eye, forward, right, up, tan_half_fov: float, width: int, height: int):
    """Primary rays of a pinhole camera through the pixel centres, row-major
    (y outer), in FP64: d = forward + x tan a right + y tan up with x = 2 (px
    + 1/2) / width - 1, y = 1 - 2 (py + 1/2) / height, a = width / height,
    normalised (so t is the distance from the eye). The camera vectors are
    taken as given (FP32 values widened to FP64)."""
    e, f, r, u = (np.asarray(v, np.float64) for v in (eye, forward, right, up))
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    x = (2.0 * (px.reshape(-1) + 0.5) / width - 1.0) * tan_half_fov * (width / height)
    y = (1.0 - 2.0 * (py.reshape(-1) + 0.5) / height) * tan_half_fov
    d = f[None, :] + x[:, None] * r[None, :] + y[:, None] * u[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.broadcast_to(e, d.shape).copy(), d


def gbuffer(meshes, instances, eye, forward, right, up, tan_half_fov: float, width: int, height: int) -> dict:
    """The primary-ray G-buffer of the hybrid pipeline (Sec. 4, Fig. 4a):
    for every pixel, the nearest triangle that the ray through the pixel
    centre hits over all instances -- shape index (the instance), primitive
    index (the triangle), barycentric coordinates (u, v) of the hit (p = (1
    - u - v) a + u b + v c) and camera distance. Each instance's triangles
    are met in its object frame (the ray mapped by o' = A o + b, d' = A d;
    t unchanged), by brute force over every triangle. Ties: the lowest
    instance, then the lowest triangle. A pixel with no hit: shape -1,
    prim -1, u = v = 0, distance +inf."""
    o, d = pixel_rays(eye, forward, right, up, tan_half_fov, width, height)
    n = o.shape[0]
    out = dict(shape=np.full(n, -1, np.int32), prim=np.full(n, -1, np.int32), u=np.zeros(n), v=np.zeros(n),
               dist=np.full(n, np.inf), normal=np.zeros((n, 3)))
    for k, inst in enumerate(instances):
        mesh = meshes[inst.obj]
        oo = _c(o @ inst.A.T + inst.b[None, :], np.float64)
        dd = _c(d @ inst.A.T, np.float64)
        t = np.zeros(n)
        tri = np.zeros(n, np.int32)
        uu = np.zeros(n)
        vv = np.zeros(n)
        lib().orc_cast64(_p(oo), _p(dd), n, _p(_c(mesh.verts, np.float32)), _p(_c(mesh.tris, np.int32)), mesh.nt,
                         _p(t), _p(tri), _p(uu), _p(vv))
        take = (tri >= 0) & (t < out["dist"])
        out["shape"][take] = k
        out["prim"][take] = tri[take]
        out["u"][take] = uu[take]
        out["v"][take] = vv[take]
        out["dist"][take] = t[take]
    # shading normal of the winner: its vertex normals interpolated at (u, v)
    # (Sec. 5.3 convention), mapped to world by A^T and normalised
    for k, inst in enumerate(instances):
        m = out["shape"] == k
        if not m.any():
            continue
        mesh = meshes[inst.obj]
        tri = mesh.tris[out["prim"][m]]
        vn = mesh.vnormals.astype(np.float64)
        u, v = out["u"][m], out["v"][m]
        nrm = (1 - u - v)[:, None] * vn[tri[:, 0]] + u[:, None] * vn[tri[:, 1]] + v[:, None] * vn[tri[:, 2]]
        nrm = nrm @ inst.A
        ln = np.linalg.norm(nrm, axis=1, keepdims=True)
        out["normal"][m] = nrm / np.where(ln > 0, ln, 1.0)
    return out


def ray_triangle(mesh, inst, tri: np.ndarray, o: np.ndarray, d: np.ndarray):
    """(t, u, v) of rays (o, d; n x 3, world) against triangles `tri` of an
    instance's mesh, one per ray, WITHOUT the inside test: the Moller-Trumbore
    solution of o' + t d' = (1 - u - v) a + u b + v c in the object frame.
    For judging pixels that lie on a triangle's edge within rounding."""
    oo = o @ inst.A.T + inst.b[None, :]
    dd = d @ inst.A.T
    v3 = mesh.verts.astype(np.float64)
    a, b, c = (v3[mesh.tris[tri, j]] for j in range(3))
    e1, e2, s = b - a, c - a, oo - a
    p = np.cross(dd, e2)
    det = np.einsum("ij,ij->i", e1, p)
    q = np.cross(s, e1)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.einsum("ij,ij->i", s, p) / det
        v = np.einsum("ij,ij->i", dd, q) / det
        t = np.einsum("ij,ij->i", e2, q) / det
    return t, u, v


@dataclass
class MeshObject:
    """A scene object kept as triangles (the hybrid pipeline's non-LSNIF
    objects, Sec. 4): queries are answered exactly."""
    mesh: object
    bmin: np.ndarray
    bmax: np.ndarray


def mesh_object(mesh) -> MeshObject:
    lo, hi = bbox(mesh.verts)
    return MeshObject(mesh, lo, hi)


def mesh_query(mobj: MeshObject, rays: np.ndarray):
    """Exact answer for a mesh object: the nearest triangle by brute force
    (the judge, tmin <= t <= tmax, lowest index on ties), its shading normal
    (vertex normals interpolated at the hit, Sec. 5.3 convention),
    material and the material's albedo. Returns (Hits, Segments) shaped like
    query()'s, with no network outputs and no near-face rays."""
    mesh = mobj.mesh
    j = judge(mesh, rays)
    n = j.t.size
    hit = j.tri >= 0
    h = Hits(hit.copy(), np.where(hit, j.t, np.inf), shading_normal(mesh, j), np.full(n, -1, np.int32),
             np.zeros((n, 3)), np.full((n, 0), np.nan), np.zeros(n, bool))
    h.mat[hit] = mesh.tri_mat[j.tri[hit]]
    h.albedo[hit] = mesh.albedo[h.mat[hit]].astype(np.float64)
    seg = Segments(np.zeros(n, np.int32), np.full((n, 2), np.nan), np.zeros((n, 0, 3)), np.zeros((n, 0), np.int32),
                   np.zeros(n, bool))
    return h, seg


def scene_query(objs, instances, rays: np.ndarray, precision: str = "f64") -> dict:
    """The wavefront integration of Sec. 4 over instanced objects (Sec. 6):
    every (ray, instance) pair is queried in the instance's object frame (the
    query takes FP32 rays, so the mapped rays are rounded to FP32); each ray
    keeps its nearest hit -- smallest t, the lowest instance index on equal
    t. The normal returns to world space as A^T n, normalised (normals map
    with the inverse transpose of the object-to-world map, which is A^T). A
    ray no pair hits gets the miss values: hit 0, t inf, normal 0, mat -1,
    albedo 0, instance -1. `near` marks rays with a near-face pair. Objects
    may be LSNIF objects or mesh objects (answered exactly, mesh_query)."""
    r = np.asarray(rays, np.float64)
    n = r.shape[1]
    res = dict(hit=np.zeros(n, bool), t=np.full(n, np.inf), normal=np.zeros((n, 3)),
               mat=np.full(n, -1, np.int32), albedo=np.zeros((n, 3)), inst=np.full(n, -1, np.int32),
               near=np.zeros(n, bool))
    for i, inst in enumerate(instances):
        local = to_object_frame(r, inst).astype(np.float32)
        ob = objs[inst.obj]
        h, seg = mesh_query(ob, local) if isinstance(ob, MeshObject) else query(ob, local, precision)
        res["near"] |= seg.near
        take = h.hit & (h.t < res["t"])
        if not take.any():
            continue
        nw = h.normal[take] @ inst.A          # rows are (A^T n)^T
        ln = np.linalg.norm(nw, axis=1, keepdims=True)
        res["normal"][take] = np.where(ln > 0, nw / np.where(ln > 0, ln, 1.0), 0.0)
        res["hit"][take] = True
        res["t"][take] = h.t[take]
        res["mat"][take] = h.mat[take]
        res["albedo"][take] = h.albedo[take]
        res["inst"][take] = i
    return res


def bounce_rays(rays: np.ndarray, hit: np.ndarray, t: np.ndarray, normal: np.ndarray, u: np.ndarray,
                eps: float) -> np.ndarray:
    """Next-bounce rays of a path tracer from the query's hits: origin at the
    hit point o + t d moved by eps along the normal turned to face the
    incoming ray, direction cosine-weighted about that normal (u: n x 2
    uniforms), tmin 0, tmax inf. Rays without a hit, or with a zero normal,
    become dead rays (zero direction: a miss for the query)."""
    r = np.asarray(rays, np.float64)
    n = r.shape[1]
    out = np.zeros((8, n))
    out[7] = np.inf
    nn = np.asarray(normal, np.float64)
    live = np.asarray(hit, bool) & (np.linalg.norm(nn, axis=1) > 0)
    if not live.any():
        return out
    o, d = r[0:3, live].T, r[3:6, live].T
    nl = nn[live]
    nl = nl / np.linalg.norm(nl, axis=1, keepdims=True)
    facing = np.where(np.einsum("ij,ij->i", nl, d) > 0, -1.0, 1.0)
    nf = nl * facing[:, None]
    p = o + t[live, None] * d + eps * nf
    dirs = cosine_dir(nf, u[live, 0], u[live, 1])
    out[0:3, live] = p.T
    out[3:6, live] = dirs.T
    out[6, live] = 0.0
    return out


# --------------------------------------------------------------------------
# geometric judge (Sec. 5.2 ground truth by ray casting)
# --------------------------------------------------------------------------

@dataclass
class Judge:
    t: np.ndarray        # inf on a miss
    tri: np.ndarray      # -1 on a miss
    u: np.ndarray
    v: np.ndarray


def judge(mesh, rays: np.ndarray) -> Judge:
    r = _c(np.asarray(rays, np.float32).T, np.float32)
    n = r.shape[0]
    t = np.zeros(n)
    tri = np.zeros(n, np.int32)
    u = np.zeros(n)
    v = np.zeros(n)
    lib().orc_judge(_p(r), n, _p(_c(mesh.verts, np.float32)), _p(_c(mesh.tris, np.int32)), mesh.nt,
                    _p(t), _p(tri), _p(u), _p(v))
    return Judge(t, tri, u, v)


def shading_normal(mesh, j: Judge) -> np.ndarray:
    """Barycentric interpolation of vertex normals, normalised (Sec. 5.3)."""
    out = np.zeros((j.t.size, 3))
    m = j.tri >= 0
    tri = mesh.tris[j.tri[m]]
    vn = mesh.vnormals.astype(np.float64)
    w0 = 1.0 - j.u[m] - j.v[m]
    nrm = w0[:, None] * vn[tri[:, 0]] + j.u[m, None] * vn[tri[:, 1]] + j.v[m, None] * vn[tri[:, 2]]
    ln = np.linalg.norm(nrm, axis=1, keepdims=True)
    out[m] = nrm / np.where(ln > 0, ln, 1.0)
    return out


# --------------------------------------------------------------------------
# training data (Sec. 5.2): balanced outside / surface rays
# --------------------------------------------------------------------------

def onb(n: np.ndarray):
    """Orthonormal basis (t, b) about unit n, Duff et al. 2017 ("Building an
    Orthonormal Basis, Revisited")."""
    s = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (s + n[:, 2])
    bb = n[:, 0] * n[:, 1] * a
    t = np.stack([1.0 + s * n[:, 0] ** 2 * a, s * bb, -s * n[:, 0]], 1)
    b = np.stack([bb, s + n[:, 1] ** 2 * a, -n[:, 1]], 1)
    return t, b


def sphere_point(u0, u1):
    z = 1.0 - 2.0 * u0
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = 2.0 * np.pi * u1
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)


def cosine_dir(n, u0, u1):
    """Cosine-weighted direction about unit axis n: sqrt(u0) disk radius,
    2 pi u1 angle, lifted to the hemisphere."""
    r = np.sqrt(u0)
    ph = 2.0 * np.pi * u1
    x, y, z = r * np.cos(ph), r * np.sin(ph), np.sqrt(np.maximum(0.0, 1.0 - u0))
    t, b = onb(n)
    return x[:, None] * t + y[:, None] * b + z[:, None] * n


SURFACE_ATTEMPTS = 8
N_UNIFORMS = 40   # per training ray: 4 outside, 8 x 4 attempts, 2 final direction, 2 spare


def training_rays(mesh, bmin, bmax, u: np.ndarray, n_outside: int):
    """Balanced sampling of Sec. 5.2 from per-ray uniforms u (n, 40).

    Rays [0, n_outside): origin uniform on the sphere about the AABB centre of
    radius 1.05 x half-diagonal (u0,u1), cosine-weighted direction about the
    inward direction (u2,u3). Rays [n_outside, n): up to 8 outside rays
    (u[4+4a : 8+4a], a = 0..7) are cast until one hits the mesh; the new ray
    starts at the hit, offset by 1e-4 x diagonal along the geometric normal
    facing the incoming ray, with a cosine-weighted direction about that
    normal (u36,u37). If no attempt hits, the ray stays the outside ray of
    u0..u3.
    Returns rays (8, n) float32 and a bool array 'surface'."""
    u = np.asarray(u, np.float64)
    n = u.shape[0]
    lo = np.asarray(bmin, np.float64)
    hi = np.asarray(bmax, np.float64)
    c = 0.5 * (lo + hi)
    diag = np.linalg.norm(hi - lo)
    R = 1.05 * 0.5 * diag

    def outside(uu):
        o = c + R * sphere_point(uu[:, 0], uu[:, 1])
        inward = (c - o) / np.linalg.norm(c - o, axis=1, keepdims=True)
        return o, cosine_dir(inward, uu[:, 2], uu[:, 3])

    o, d = outside(u[:, 0:4])
    surf = np.zeros(n, bool)
    idx = np.arange(n_outside, n)
    if idx.size:
        pending = idx.copy()
        for a in range(SURFACE_ATTEMPTS):
            if pending.size == 0:
                break
            oa, da = outside(u[pending, 4 + 4 * a:8 + 4 * a])
            rr = np.zeros((8, pending.size), np.float32)
            rr[0:3] = oa.T
            rr[3:6] = da.T
            rr[6] = 0.0
            rr[7] = np.inf
            j = judge(mesh, rr)
            got = j.tri >= 0
            if got.any():
                g = pending[got]
                ph = oa[got] + j.t[got, None] * da[got]
                geo = _face_normal(mesh, j.tri[got])
                side = np.sign(np.sum(geo * da[got], axis=1))
                side[side == 0] = 1.0
                nf = -side[:, None] * geo          # geometric normal facing the incoming ray
                o[g] = ph + 1e-4 * diag * nf
                d[g] = cosine_dir(nf, u[g, 36], u[g, 37])
                surf[g] = True
            pending = pending[~got]
    rays = np.zeros((8, n), np.float32)
    rays[0:3] = o.T
    rays[3:6] = d.T
    rays[6] = 0.0
    rays[7] = np.inf
    return rays, surf


def _face_normal(mesh, tri_idx: np.ndarray) -> np.ndarray:
    v = mesh.verts.astype(np.float64)
    t = mesh.tris[tri_idx]
    n = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


@dataclass
class Labels:
    occ: np.ndarray      # float64 0/1
    t_local: np.ndarray  # (t_hit - t0)/(t1 - t0), 0 where not occluded
    normal: np.ndarray   # (n, 3) unit shading normal
    albedo: np.ndarray   # (n, 3)
    mat: np.ndarray      # int32


def labels(mesh, rays: np.ndarray, t01: np.ndarray) -> Labels:
    """Ground truth of Sec. 5.2/5.3 from the judge: occlusion, local hit
    distance in the ray's AABB interval, shading normal, albedo, material."""
    j = judge(mesh, rays)
    occ = (j.tri >= 0).astype(np.float64)
    tl = np.zeros(j.t.size)
    m = j.tri >= 0
    tl[m] = (j.t[m] - t01[m, 0]) / (t01[m, 1] - t01[m, 0])
    mat = np.where(m, mesh.tri_mat[np.maximum(j.tri, 0)], 0).astype(np.int32)
    alb = np.where(m[:, None], mesh.albedo[mat].astype(np.float64), 0.0)
    return Labels(occ, tl, shading_normal(mesh, j), alb, mat)


# --------------------------------------------------------------------------
# losses (Sec. 5.3) and their gradient with respect to the logits
# --------------------------------------------------------------------------

REL_L2_EPS = 0.01
NORMAL_EPS = 1e-12


def loss_terms(Z: np.ndarray, lab: Labels, live: np.ndarray | None = None):
    """Per-ray loss terms and dLoss/dZ for the batch mean of the total over
    the rays that reach the network (`live`; all rays when None): a ray that
    meets no occupied voxel is answered without the network, so it takes no
    part in training.

    BCE on the occlusion logit (stable form); for rays whose reference is
    occluded also: MAE of sigmoid(z1) against the local hit distance, 1 -
    cosine similarity for the normal, relative L2 (x-y)^2/(sg(x)^2+0.01)
    averaged over RGB for albedo, cross-entropy for the material. Terms other
    than occlusion are zero when the reference is not occluded."""
    n = Z.shape[0]
    y = lab.occ
    z0 = Z[:, 0]
    l_occ = np.maximum(z0, 0) - z0 * y + np.log1p(np.exp(-np.abs(z0)))
    g = np.zeros_like(Z)
    g[:, 0] = sigmoid(z0) - y
    s1 = sigmoid(Z[:, 1])
    l_t = np.abs(s1 - lab.t_local)
    g[:, 1] = np.sign(s1 - lab.t_local) * s1 * (1 - s1)
    zn = Z[:, 2:5]
    nz = np.maximum(np.linalg.norm(zn, axis=1), NORMAL_EPS)
    dot = np.sum(zn * lab.normal, axis=1)
    l_n = 1.0 - dot / nz
    g[:, 2:5] = -(lab.normal / nz[:, None] - dot[:, None] * zn / nz[:, None] ** 3)
    sa = sigmoid(Z[:, 5:8])
    den = sa ** 2 + REL_L2_EPS
    l_a = np.mean((sa - lab.albedo) ** 2 / den, axis=1)
    g[:, 5:8] = (2.0 / 3.0) * (sa - lab.albedo) / den * sa * (1 - sa)
    zm = Z[:, 8:]
    mx = zm.max(axis=1, keepdims=True)
    ez = np.exp(zm - mx)
    lse = mx[:, 0] + np.log(ez.sum(axis=1))
    l_m = lse - zm[np.arange(n), lab.mat]
    sm = ez / ez.sum(axis=1, keepdims=True)
    sm[np.arange(n), lab.mat] -= 1.0
    g[:, 8:] = sm
    g[:, 1:] *= y[:, None]
    w = np.ones(n) if live is None else live.astype(np.float64)
    m = max(w.sum(), 1.0)
    per_ray = l_occ + y * (l_t + l_n + l_a + l_m)
    terms = dict(occ=(w * l_occ).sum() / m, t=(w * y * l_t).sum() / m, normal=(w * y * l_n).sum() / m,
                 albedo=(w * y * l_a).sum() / m, mat=(w * y * l_m).sum() / m, total=(w * per_ray).sum() / m)
    return terms, g * (w / m)[:, None]


# --------------------------------------------------------------------------
# training step (Sec. 5.2): forward, loss, backward, Adam
# --------------------------------------------------------------------------

def forward_backward(obj: OracleObject, rays: np.ndarray, lab: Labels, seg: Segments | None = None):
    """Loss terms and gradients of the batch-mean loss (over rays that reach
    the network) with respect to every network weight/bias and every
    hash-table entry."""
    cfg = obj.cfg
    seg = ray_segments(obj, rays) if seg is None else seg
    X = features(obj, seg)
    Z, cache = mlp_forward(X, obj.weights, cfg.activation, keep=True)
    terms, dZ = loss_terms(Z, lab, live=seg.k > 0)
    grads = []
    d = dZ
    for i in range(len(obj.weights) - 1, -1, -1):
        h_in, z = cache[i]
        W, _ = obj.weights[i]
        if i < len(obj.weights) - 1:
            d = d * activation_grad(z, cfg.activation)
        grads.append((d.T @ h_in, d.sum(axis=0)))
        d = d @ W
    grads.reverse()
    n, H = seg.k.size, cfg.H
    dX = d.reshape(n, H, cfg.L, cfg.F)
    live = np.arange(H)[None, :] < 2 * seg.k[:, None]
    gt = np.zeros_like(obj.tables)
    if live.any():
        encode_backward(seg.pts[live], obj.res, cfg.F, cfg.log2_T, dX[live], gt)
    return terms, grads, gt


@dataclass
class AdamState:
    m: list
    v: list
    step: int = 0


def adam_init(arrays) -> AdamState:
    return AdamState([np.zeros_like(a, dtype=np.float64) for a in arrays],
                     [np.zeros_like(a, dtype=np.float64) for a in arrays], 0)


def adam_step(params, grads, st: AdamState, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba) with bias correction; returns the updated params."""
    st.step += 1
    out = []
    for i, (p, g) in enumerate(zip(params, grads)):
        st.m[i] = b1 * st.m[i] + (1 - b1) * g
        st.v[i] = b2 * st.v[i] + (1 - b2) * g * g
        mh = st.m[i] / (1 - b1 ** st.step)
        vh = st.v[i] / (1 - b2 ** st.step)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return out


# --------------------------------------------------------------------------
# storage model (Sec. 5.1)
# --------------------------------------------------------------------------

def footprint_bytes(V: int, L: int, T: int, F: int, layer_dims, feat_bytes: int = 2,
                    weight_bytes: int = 2) -> dict:
    """Bytes of one object: V^3 occupancy bits, L x T x F features, network
    weights and biases."""
    vox = V ** 3 // 8
    enc = L * T * F * feat_bytes
    nn = sum(fi * fo + fo for fi, fo in layer_dims) * weight_bytes
    return dict(voxels=vox, encoder=enc, network=nn, total=vox + enc + nn)
