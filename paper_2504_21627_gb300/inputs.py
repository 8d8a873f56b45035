"""Seeded synthetic inputs for the LSNIF query: meshes, rays and parameters.

This module only draws random numbers and builds procedural geometry. It holds
none of the query's arithmetic (no bounding box, voxelization, traversal,
encoding, network or loss), so that both the CUDA path and the FP64 oracle can
consume exactly the same inputs without sharing any of the method.

Every generator takes an explicit integer seed and uses numpy's PCG64, whose
stream is stable across platforms, so x86 and Arm hosts build identical inputs.

The paper evaluates on production scenes that are not available here; the
procedural meshes below (an icosphere and a noise-displaced torus) stand in
for them with the sizes the workloads call for.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

@dataclass
class Mesh:
    verts: np.ndarray      # (nv, 3) float32, object space
    tris: np.ndarray       # (nt, 3) int32, counter-clockwise seen from outside
    vnormals: np.ndarray   # (nv, 3) float32, unit, area-weighted
    tri_mat: np.ndarray    # (nt,) int32 material index per triangle
    albedo: np.ndarray     # (n_mat, 3) float32 base colour per material
    n_mat: int = 1

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])


def _vertex_normals(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Area-weighted vertex normals (sum of unnormalised face normals)."""
    v = verts.astype(np.float64)
    fn = np.cross(v[tris[:, 1]] - v[tris[:, 0]], v[tris[:, 2]] - v[tris[:, 0]])
    acc = np.zeros_like(v)
    for c in range(3):
        np.add.at(acc, tris[:, c], fn)
    nrm = np.linalg.norm(acc, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return (acc / nrm).astype(np.float32)


def _albedo_table(n_mat: int, seed: int) -> np.ndarray:
    return rng(seed ^ 0xA1BED0).uniform(0.05, 0.95, size=(n_mat, 3)).astype(np.float32)


def icosphere(subdiv: int = 3, radius: float = 1.0, seed: int = 1) -> Mesh:
    """Unit icosphere; material = octant of the face centroid, mod 2.

    The octant is (cx>0) | (cy>0)<<1 | (cz>0)<<2 with strict comparisons, so
    faces whose centroid lies exactly on a coordinate plane get a fixed bit.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    v = (np.array(verts) * radius).astype(np.float32)
    f = np.array(faces, dtype=np.int32)
    cen = v[f].astype(np.float64).mean(axis=1)
    octant = (cen[:, 0] > 0).astype(np.int32) | ((cen[:, 1] > 0).astype(np.int32) << 1) \
        | ((cen[:, 2] > 0).astype(np.int32) << 2)
    mat = (octant % 2).astype(np.int32)
    return Mesh(v, f, _vertex_normals(v, f), mat, _albedo_table(2, seed), n_mat=2)


def _lattice_value(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray, salt: int) -> np.ndarray:
    """Hashed lattice value in [-1, 1] (SplitMix64 finaliser on the packed key)."""
    with np.errstate(over="ignore"):
        k = (ix.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
             ^ iy.astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)
             ^ iz.astype(np.uint64) * np.uint64(0x165667B19E3779F9)
             ^ np.uint64(salt & 0xFFFFFFFFFFFFFFFF))
        k = (k ^ (k >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        k = (k ^ (k >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        k = k ^ (k >> np.uint64(31))
    return (k >> np.uint64(11)).astype(np.float64) / float(1 << 53) * 2.0 - 1.0


def value_noise(p: np.ndarray, seed: int, octaves: int = 3, base_freq: float = 4.0) -> np.ndarray:
    """Sum of `octaves` value-noise octaves (smoothstep interpolation), in [-1, 1].

    Octave o has frequency base_freq * 2**o and amplitude 2**-o; the sum is
    divided by the total amplitude so the result stays in [-1, 1].
    """
    out = np.zeros(p.shape[0])
    total = 0.0
    for o in range(octaves):
        f = base_freq * (2 ** o)
        a = 0.5 ** o
        q = p * f
        i0 = np.floor(q).astype(np.int64)
        fr = q - i0
        s = fr * fr * (3.0 - 2.0 * fr)
        acc = np.zeros(p.shape[0])
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((s[:, 0] if dx else 1 - s[:, 0]) * (s[:, 1] if dy else 1 - s[:, 1])
                         * (s[:, 2] if dz else 1 - s[:, 2]))
                    acc += w * _lattice_value(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz,
                                              seed * 7919 + o)
        out += a * acc
        total += a
    return out / total


def noise_torus(seed: int, R: float = 1.0, r: float = 0.35, nu: int = 500, nv: int = 200,
                amplitude: float = 0.05, n_mat: int = 4) -> Mesh:
    """Torus (major radius R, minor r) on an nu x nv quad grid, 2*nu*nv triangles,
    displaced along the vertex normal by 3-octave value noise of peak `amplitude`.
    Material = sector of the major angle: floor(n_mat * i / nu) for quad column i.
    """
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    th = 2.0 * np.pi * i / nu
    ph = 2.0 * np.pi * j / nv
    ring = R + r * np.cos(ph)
    pos = np.stack([ring * np.cos(th), ring * np.sin(th), r * np.sin(ph) + 0 * th], -1).reshape(-1, 3)
    nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph) + 0 * th],
                   -1).reshape(-1, 3)
    pos = pos + nrm * (amplitude * value_noise(pos, seed))[:, None]
    idx = lambda a, b: (a % nu) * nv + (b % nv)  # noqa: E731
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a, b, c, d = idx(ii, jj), idx(ii + 1, jj), idx(ii + 1, jj + 1), idx(ii, jj + 1)
    t0 = np.stack([a, b, c], -1).reshape(-1, 3)
    t1 = np.stack([a, c, d], -1).reshape(-1, 3)
    tris = np.stack([t0, t1], 1).reshape(-1, 3).astype(np.int32)
    quad_mat = np.repeat((n_mat * ii // nu).reshape(-1), 2).astype(np.int32)
    v = pos.astype(np.float32)
    return Mesh(v, tris, _vertex_normals(v, tris), quad_mat, _albedo_table(n_mat, seed), n_mat=n_mat)


def icosphere_vec(subdiv: int, seed: int = 1) -> Mesh:
    """The icosphere of icosphere() (vertex positions equal to within one
    FP32 ulp, another vertex order), built with vectorised edge splitting
    (shared midpoints found with np.unique) for large subdivision levels."""
    base = icosphere(0, seed=seed)
    v = base.verts.astype(np.float64)
    f = base.tris.astype(np.int64)
    for _ in range(subdiv):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        es = np.sort(e, axis=1)
        uniq, inv = np.unique(es, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        m = v[uniq[:, 0]] + v[uniq[:, 1]]
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        mid = len(v) + inv
        nf = len(f)
        ab, bc, ca = mid[:nf], mid[nf:2 * nf], mid[2 * nf:]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1), np.stack([c, ca, bc], 1),
                            np.stack([ab, bc, ca], 1)])
        v = np.concatenate([v, m])
    v32 = v.astype(np.float32)
    f32 = f.astype(np.int32)
    cen = v32[f32].astype(np.float64).mean(axis=1)
    octant = (cen[:, 0] > 0).astype(np.int32) | ((cen[:, 1] > 0).astype(np.int32) << 1) \
        | ((cen[:, 2] > 0).astype(np.int32) << 2)
    return Mesh(v32, f32, _vertex_normals(v32, f32), (octant % 2).astype(np.int32), _albedo_table(2, seed), n_mat=2)


def noise_icosphere(seed: int, target_tris: int, amplitude: float = 0.05, n_mat: int = 4) -> Mesh:
    """Icosphere with about `target_tris` triangles (20 * 4**s, rounded to the
    nearest level), displaced by value noise; materials by octant mod n_mat."""
    s = int(round(math.log(max(target_tris, 20) / 20.0, 4)))
    m = icosphere(max(s, 0), seed=seed) if s <= 4 else icosphere_vec(s, seed=seed)
    v = m.verts.astype(np.float64)
    n = m.vnormals.astype(np.float64)
    v = v + n * (amplitude * value_noise(v, seed))[:, None]
    v = v.astype(np.float32)
    cen = v[m.tris].astype(np.float64).mean(axis=1)
    octant = (cen[:, 0] > 0).astype(np.int32) | ((cen[:, 1] > 0).astype(np.int32) << 1) \
        | ((cen[:, 2] > 0).astype(np.int32) << 2)
    return Mesh(v, m.tris, _vertex_normals(v, m.tris), (octant % n_mat).astype(np.int32),
                _albedo_table(n_mat, seed), n_mat=n_mat)


def noise_torus_tris(seed: int, target_tris: int, amplitude: float = 0.05, n_mat: int = 4) -> Mesh:
    """Noise torus with about `target_tris` triangles (quad grid 5:2)."""
    nv = max(8, int(round(math.sqrt(target_tris / 2 / 2.5))))
    nu = max(8, int(round(2.5 * nv)))
    return noise_torus(seed, nu=nu, nv=nv, amplitude=amplitude, n_mat=n_mat)


def cube(n_mat: int = 1) -> Mesh:
    """Surface of the unit cube [0, 1]^3: 12 triangles, outward winding."""
    v = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], dtype=np.float32)
    f = np.array([[0, 2, 1], [1, 2, 3], [4, 5, 6], [5, 7, 6],      # z = 0, z = 1
                  [0, 1, 4], [1, 5, 4], [2, 6, 3], [3, 6, 7],      # y = 0, y = 1
                  [0, 4, 2], [2, 4, 6], [1, 3, 5], [3, 7, 5]],     # x = 0, x = 1
                 dtype=np.int32)
    return Mesh(v, f, _vertex_normals(v, f), np.zeros(12, np.int32), _albedo_table(n_mat, 0), n_mat)


def tetrahedron(n_mat: int = 2) -> Mesh:
    """Regular tetrahedron inscribed in the unit sphere (alternate corners of
    a cube), outward winding; triangle i has material i mod n_mat."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float32) / np.float32(math.sqrt(3.0))
    f = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    mat = (np.arange(4) % n_mat).astype(np.int32)
    return Mesh(v, f, _vertex_normals(v, f), mat, _albedo_table(n_mat, 0), n_mat)


def single_triangle(a, b, c, n_mat: int = 1) -> Mesh:
    v = np.array([a, b, c], dtype=np.float32)
    f = np.array([[0, 1, 2]], dtype=np.int32)
    return Mesh(v, f, _vertex_normals(v, f), np.zeros(1, np.int32), _albedo_table(n_mat, 0), n_mat)


# --------------------------------------------------------------------------
# rays (SoA rows: ox oy oz dx dy dz tmin tmax), float32
# --------------------------------------------------------------------------

def _unit_sphere(g: np.random.Generator, n: int) -> np.ndarray:
    v = g.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def pack_rays(o: np.ndarray, d: np.ndarray, tmin=0.0, tmax=np.inf) -> np.ndarray:
    n = o.shape[0]
    r = np.empty((8, n), dtype=np.float32)
    r[0:3] = o.T
    r[3:6] = d.T
    r[6] = tmin
    r[7] = tmax
    return r


def rays_sphere_to_box(n: int, radius: float, bmin, bmax, seed: int) -> np.ndarray:
    """Origins uniform on a sphere of `radius` about the origin, each aimed at a
    uniform point of the box [bmin, bmax]; unit directions, tmin 0, tmax inf."""
    g = rng(seed)
    o = _unit_sphere(g, n) * radius
    tgt = g.uniform(np.asarray(bmin, np.float64), np.asarray(bmax, np.float64), size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return pack_rays(o, d)


@dataclass
class Camera:
    eye: np.ndarray
    forward: np.ndarray
    right: np.ndarray
    up: np.ndarray
    width: int
    height: int
    fov_deg: float


def seeded_camera(seed: int, radius: float = 4.0, width: int = 2048, height: int = 2048,
                  fov_deg: float = 45.0) -> Camera:
    """Pinhole camera at a seeded point of the sphere of `radius`, looking at
    the origin; up is +z unless the view is nearly vertical (then +y)."""
    eye = _unit_sphere(rng(seed), 1)[0] * radius
    fwd = -eye / np.linalg.norm(eye)
    up0 = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up0)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(eye, fwd, right, up, width, height, fov_deg)


def rays_pinhole(cam: Camera, px0: int = 0, py0: int = 0, w: int | None = None,
                 h: int | None = None) -> np.ndarray:
    """Primary rays through pixel centres (+0.5) of the window [px0, px0+w) x
    [py0, py0+h), row-major (y outer)."""
    w = cam.width if w is None else w
    h = cam.height if h is None else h
    ys, xs = np.meshgrid(np.arange(py0, py0 + h), np.arange(px0, px0 + w), indexing="ij")
    tan = math.tan(math.radians(cam.fov_deg) / 2.0)
    aspect = cam.width / cam.height
    u = ((xs.reshape(-1) + 0.5) / cam.width * 2.0 - 1.0) * tan * aspect
    v = (1.0 - (ys.reshape(-1) + 0.5) / cam.height * 2.0) * tan
    d = cam.forward[None, :] + u[:, None] * cam.right[None, :] + v[:, None] * cam.up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(cam.eye, d.shape)
    return pack_rays(o, d)


def uniforms(n: int, k: int, seed: int) -> np.ndarray:
    """(n, k) float32 uniforms in [0, 1): the random numbers a sampler consumes."""
    return rng(seed).random((n, k), dtype=np.float32)


# --------------------------------------------------------------------------
# configurations and parameters
# --------------------------------------------------------------------------

@dataclass
class Config:
    V: int = 32
    H: int = 18
    L: int = 8
    F: int = 2
    log2_T: int = 14
    N_min: int = 8
    N_max: int = 128
    n_hidden: int = 3
    width: int = 64
    n_mat: int = 2
    activation: int = 0          # 0 ReLU, 1 leaky ReLU (slope 0.01)
    table_init: float = 1e-4     # features drawn from U(-table_init, table_init)
    seed: int = 1

    @property
    def T(self) -> int:
        return 1 << self.log2_T

    @property
    def n_in(self) -> int:
        return self.H * self.L * self.F

    @property
    def n_out(self) -> int:
        return 8 + self.n_mat

    def layer_dims(self) -> list[tuple[int, int]]:
        """(fan_in, fan_out) of every dense layer, input to output."""
        dims = [self.n_in] + [self.width] * self.n_hidden + [self.n_out]
        return [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)]


def cfg_icosphere_small() -> Config:
    """1280-triangle icosphere, 32^3 voxels, 8 levels x 2 FP32 features,
    2^14 entries per level, resolutions 8..128, MLP 3 x 64 ReLU."""
    return Config(V=32, H=18, L=8, F=2, log2_T=14, N_min=8, N_max=128, n_hidden=3, width=64,
                  n_mat=2)


def cfg_torus_4m() -> Config:
    """200k-triangle noise torus, 128^3 voxels, 16 levels x 2 features,
    2^19 entries per level, resolutions 16..2048, MLP 4 x 64."""
    return Config(V=128, H=18, L=16, F=2, log2_T=19, N_min=16, N_max=2048, n_hidden=4,
                  width=64, n_mat=4)


@dataclass
class Params:
    tables: np.ndarray                      # (L, T, F) float32
    weights: list = field(default_factory=list)   # [(W (out,in) f32, b (out,) f32), ...]

    def packed_mlp(self) -> np.ndarray:
        return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)])
                               for W, b in self.weights]).astype(np.float32)


def batched_objects(n_obj: int = 64, seed: int = 3, total_rays: int = 16 << 20):
    """The many-object workload: n_obj seeded noise-displaced icospheres or
    tori of 5k..500k triangles (log-uniform), V in {64, 128, 256} and table
    size 2^16..2^20 (log-uniform), L = 16, F = 2, 4 x 64 network, and a
    power-law ray count per object (Pareto, clipped to [1k, 1M]) rescaled to
    about total_rays in all. Returns [(mesh, cfg, n_rays)]."""
    g = rng(seed)
    raw = 1000.0 * (1.0 + g.pareto(1.1, size=n_obj))
    counts = raw
    for _ in range(20):
        counts = np.clip(raw * total_rays / raw.sum(), 1000, 1 << 20)
        raw = counts
    counts = counts.astype(np.int64)
    out = []
    for i in range(n_obj):
        tris = int(math.exp(g.uniform(math.log(5000), math.log(500000))))
        V = int(64 * 2 ** g.integers(0, 3))
        log2_T = int(g.integers(16, 21))
        kind = g.integers(0, 2)
        mesh = noise_icosphere(seed + 100 + i, tris, n_mat=4) if kind == 0 else \
            noise_torus_tris(seed + 100 + i, tris, n_mat=4)
        cfg = Config(V=V, H=18, L=16, F=2, log2_T=log2_T, N_min=16, N_max=max(512, 8 * V), n_hidden=4, width=64,
                     n_mat=4, seed=seed + i)
        out.append((mesh, cfg, int(counts[i])))
    return out


def cfg_stress_object(log2_T: int = 21) -> Config:
    """Per-object configuration of the path-tracing stress scene: 128^3
    voxels, 16 levels x 4 features, 2^21 entries per level, resolutions
    16..2048, MLP 4 x 128, 4 materials."""
    return Config(V=128, H=18, L=16, F=4, log2_T=log2_T, N_min=16, N_max=2048, n_hidden=4,
                  width=128, n_mat=4)


def scene_objects(n_unique: int = 8, seed: int = 5, features: int = 2, width: int = 64):
    """The instanced scene's unique objects: seeded noise icospheres or tori
    of 50k..1M triangles (log-uniform), V = 128, L = 16, T = 2^21, F
    features per level and a 4 x width network (F = 4 and width 128 is the
    stress configuration). Returns [(mesh, cfg)]."""
    g = rng(seed)
    out = []
    for i in range(n_unique):
        tris = int(math.exp(g.uniform(math.log(50000), math.log(1000000))))
        mesh = noise_icosphere(seed + 200 + i, tris, n_mat=4) if i % 2 == 0 else \
            noise_torus_tris(seed + 200 + i, tris, n_mat=4)
        cfg = Config(V=128, H=18, L=16, F=features, log2_T=21, N_min=16, N_max=2048, n_hidden=4, width=width,
                     n_mat=4, seed=seed + i)
        out.append((mesh, cfg))
    return out


def camera_rays_spp(cam: Camera, spp: int, seed: int) -> np.ndarray:
    """spp jittered samples per pixel (seeded), pixel-major, as (8, w*h*spp)
    rays with tmin 0 and tmax inf."""
    g = rng(seed)
    w, h = cam.width, cam.height
    px = np.repeat(np.arange(w * h), spp)
    jx = g.random(px.size)
    jy = g.random(px.size)
    x = (px % w + jx) / w * 2.0 - 1.0
    y = 1.0 - (px // w + jy) / h * 2.0
    th = math.tan(math.radians(cam.fov_deg) / 2.0)
    aspect = w / h
    d = cam.forward[None, :] + (x * th * aspect)[:, None] * cam.right[None, :] + (y * th)[:, None] * cam.up[None, :]
    rays = np.zeros((8, px.size), np.float32)
    rays[0:3] = cam.eye[:, None]
    rays[3:6] = d.T
    rays[7] = np.inf
    return rays


def random_params(cfg: Config, seed: int, table_range: float | None = None,
                  bias_range: float = 0.0) -> Params:
    """Tables ~ U(-r, r); weights Xavier-uniform U(+-sqrt(6/(fan_in+fan_out)));
    biases U(-bias_range, bias_range) (zero by default)."""
    g = rng(seed)
    r = cfg.table_init if table_range is None else table_range
    tables = g.uniform(-r, r, size=(cfg.L, cfg.T, cfg.F)).astype(np.float32)
    ws = []
    for fi, fo in cfg.layer_dims():
        a = math.sqrt(6.0 / (fi + fo))
        W = g.uniform(-a, a, size=(fo, fi)).astype(np.float32)
        b = (g.uniform(-bias_range, bias_range, size=fo) if bias_range > 0
             else np.zeros(fo)).astype(np.float32)
        ws.append((W, b))
    return Params(tables, ws)


def constant_params(cfg: Config, out_bias, seed: int = 0) -> Params:
    """A network whose outputs are the constants out_bias for every input:
    all weights and hidden biases zero (tables seeded, unused)."""
    g = rng(seed)
    tables = g.uniform(-0.1, 0.1, size=(cfg.L, cfg.T, cfg.F)).astype(np.float32)
    ws = []
    dims = cfg.layer_dims()
    for i, (fi, fo) in enumerate(dims):
        b = np.zeros(fo, np.float32)
        if i == len(dims) - 1:
            b[:] = np.asarray(out_bias, np.float32)
        ws.append((np.zeros((fo, fi), np.float32), b))
    return Params(tables, ws)


def rotation(axis, angle: float) -> np.ndarray:
    """3 x 3 rotation about a unit axis (Rodrigues)."""
    k = np.asarray(axis, np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def seeded_instances(n: int, n_objects: int, seed: int, spread: float = 6.0, scale=(0.5, 2.0)):
    """n instances of n_objects objects: object index, world -> object map
    (A, b) of a seeded rotation, uniform scale and translation in a cube of
    side `spread` (object-to-world p = s R q + c, so A = R^T / s,
    b = -A c)."""
    g = rng(seed)
    out = []
    for i in range(n):
        R = rotation(g.normal(size=3), g.uniform(0, 2 * math.pi))
        sc = math.exp(g.uniform(math.log(scale[0]), math.log(scale[1])))
        c = g.uniform(-spread / 2, spread / 2, size=3)
        A = R.T / sc
        out.append((i % n_objects, A, -A @ c))
    return out


def unpack_mlp(cfg: Config, flat: np.ndarray) -> list:
    out, o = [], 0
    for fi, fo in cfg.layer_dims():
        W = flat[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = flat[o:o + fo]
        o += fo
        out.append((W, b))
    return out
