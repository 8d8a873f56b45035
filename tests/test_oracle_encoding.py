"""Pins for the oracle's sparse hash-grid encoding (Sec. 3.2)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _primes():
    out = {}
    for line in open(os.path.join(GOLDEN, "hash_primes.txt")):
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = int(line[1])
    return out


def test_hash_structure_against_published_multipliers():
    pr = _primes()
    for log2T in (4, 14, 19, 21):
        mask = (1 << log2T) - 1
        # pi_1 = 1: the x coordinate passes through
        for x in (0, 1, 7, 1000, 2**31 - 1):
            assert O.hash_index(x, 0, 0, log2T) == x & mask
        assert O.hash_index(0, 1, 0, log2T) == pr["pi2"] & mask
        assert O.hash_index(0, 0, 1, log2T) == pr["pi3"] & mask
        # uint32 wrap-around of the products
        assert O.hash_index(0, 3, 0, log2T) == (3 * pr["pi2"]) % 2**32 & mask
        g = np.random.default_rng(log2T)
        for x, y, z in g.integers(0, 4096, size=(50, 3)):
            # XOR decomposition over the axes
            h = O.hash_index(x, y, z, log2T)
            assert h == O.hash_index(x, 0, 0, log2T) ^ O.hash_index(0, y, 0, log2T) ^ O.hash_index(0, 0, z, log2T)


def test_hash_low_bits_the_gather_relies_on():
    """Index facts the GPU gathers use to skip per-corner work, checked on
    the oracle's hash: a step in y or in z flips bit 0 of the index (the y
    and z multipliers are odd), so one row's parity gives every row's; and
    the x neighbours' indices differ by (cx ^ (cx + 1)) & mask whatever y
    and z are, so whether they share an aligned pair is one test per cell."""
    pr = _primes()
    assert pr["pi2"] % 2 == 1 and pr["pi3"] % 2 == 1
    g = np.random.default_rng(11)
    for log2T in (2, 14, 19):
        mask = (1 << log2T) - 1
        for x, y, z in g.integers(0, 4096, size=(200, 3)):
            x, y, z = int(x), int(y), int(z)
            h = O.hash_index(x, y, z, log2T)
            assert (O.hash_index(x, y + 1, z, log2T) ^ h) & 1 == 1
            assert (O.hash_index(x, y, z + 1, log2T) ^ h) & 1 == 1
            assert (O.hash_index(x, y + 1, z + 1, log2T) ^ h) & 1 == 0
            assert O.hash_index(x + 1, y, z, log2T) ^ h == (x ^ (x + 1)) & mask


def test_weights_sum_to_one():
    g = np.random.default_rng(0)
    pts = g.random((500, 3))
    res = np.array([8, 13, 31, 128], np.int32)
    tables = np.ones((4, 1 << 10, 2))
    out, idx, w = O.encode(pts, res, 2, 10, tables, debug=True)
    assert np.allclose(w.sum(-1), 1.0, atol=1e-14)
    assert np.allclose(out, 1.0, atol=1e-14)
    assert np.all(w >= 0)


def test_multilinear_field_is_reproduced():
    """Trilinear interpolation reproduces any function that is linear in each
    coordinate separately. Pick a level whose lattice hashes without
    collisions (checked) and store f(x,y,z) at every vertex."""
    N, log2T = 4, 19
    verts = [(x, y, z) for x in range(N + 1) for y in range(N + 1) for z in range(N + 1)]
    hs = [O.hash_index(x, y, z, log2T) for x, y, z in verts]
    assert len(set(hs)) == len(hs)

    def f(x, y, z):
        return 1.0 + 2.0 * x - 3.0 * y + 0.5 * z + 0.25 * x * y * z - 0.75 * x * z

    tab = np.zeros((1, 1 << log2T, 1))
    for (x, y, z), h in zip(verts, hs):
        tab[0, h, 0] = f(x, y, z)
    g = np.random.default_rng(1)
    pts = g.random((300, 3))
    out = O.encode(pts, np.array([N], np.int32), 1, log2T, tab)
    x = pts * N
    assert np.allclose(out[:, 0, 0], f(x[:, 0], x[:, 1], x[:, 2]), rtol=0, atol=1e-12)


def test_face_points_need_four_corners():
    """A point with one coordinate on a lattice plane has exactly four
    non-zero trilinear weights (the sparse grid's 4-of-8 lookups, Sec. 3.2)."""
    g = np.random.default_rng(2)
    V, N = 32, 128
    pts = g.random((200, 3))
    axis = g.integers(0, 3, 200)
    pts[np.arange(200), axis] = g.integers(0, V + 1, 200) / V
    _, idx, w = O.encode(pts, np.array([N], np.int32), 2, 14, np.zeros((1, 1 << 14, 2)), debug=True)
    nz = (w[:, 0, :] != 0).sum(-1)
    assert np.all(nz <= 4) and (nz == 4).mean() > 0.95


def test_fp32_points_have_exact_fp64_lattice_products():
    """The cell decision is the floor of p * N for an FP32 point p: in FP64
    that product of a 24-bit and an (at most) 21-bit integer is exact, so the
    oracle's decision is the mathematical one."""
    g = np.random.default_rng(3)
    p = g.random(10000).astype(np.float32)
    for N in (16, 213, 2048, 1 << 20):
        x = p.astype(np.float64) * N
        # exact: splitting p into integer mantissa m and exponent gives m * N exactly
        m, e = np.frexp(p.astype(np.float64))
        mi = (m * 2 ** 24).astype(np.int64)
        assert np.array_equal(x, np.ldexp((mi * N).astype(np.float64), e - 24))


def test_backward_is_the_adjoint_of_the_encoding():
    """<encode(T), D> == <T, encode_backward(D)>: the scatter is the exact
    transpose of the gather."""
    g = np.random.default_rng(4)
    pts = g.random((300, 3))
    res = np.array([4, 9, 33], np.int32)
    log2T, F = 8, 2
    T = g.normal(size=(3, 1 << log2T, F))
    D = g.normal(size=(300, 3, F))
    lhs = np.sum(O.encode(pts, res, F, log2T, T) * D)
    G = np.zeros_like(T)
    O.encode_backward(pts, res, F, log2T, D, G)
    assert abs(lhs - np.sum(T * G)) < 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("x,expect", [(1.0, 1.0), (1.0 + 2**-8, 1.0), (1.0 + 3 * 2**-8, 1.0 + 2**-6),
                                       (-2.5, -2.5), (1.0 + 2**-7, 1.0 + 2**-7)])
def test_bf16_rounding_ties_to_even(x, expect):
    assert O.round_bf16(np.array([x]))[0] == expect


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(5)
    x = (g.normal(size=10000) * 10.0 ** g.integers(-6, 6, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), ref)
