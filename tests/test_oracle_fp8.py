"""Pins of the oracle's FP8 E4M3 arithmetic (the FP8 network of the stress
configuration): rounding against the format's own code table, the scale
rule, and an FP8 network whose every quantised value is representable,
which must then equal the FP64 network exactly."""
import math

import numpy as np

from oracle import oracle as O


def _e4m3_values():
    """Every finite E4M3 value, decoded from the bit layout (sign, 4 exponent
    bits with bias 7, 3 mantissa bits; exponent 0 is subnormal; the code
    S.1111.111 is NaN)."""
    vals = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        vals.append((-v if s else v, m))
    return vals


def test_round_e4m3_fixes_every_code_and_ties_to_even():
    vals = _e4m3_values()
    v = np.array([x for x, _ in vals])
    assert np.array_equal(O.round_e4m3(v), v)
    assert v.max() == 448.0 and np.min(v[v > 0]) == 2.0 ** -9
    pos = sorted({(x, m) for x, m in vals if x > 0})
    xs = np.array([x for x, _ in pos])
    for (a, ma), (b, mb) in zip(pos[:-1], pos[1:]):
        mid = 0.5 * (a + b)
        want = a if ma % 2 == 0 else b
        assert O.round_e4m3(np.array([mid]))[0] == want, (a, b)
        assert O.round_e4m3(np.array([np.nextafter(mid, 0)]))[0] == a
        assert O.round_e4m3(np.array([np.nextafter(mid, 1e9)]))[0] == b
    # saturation, zero, symmetry
    big = np.array([448.0, 449.0, 464.0, 479.0, 480.0, 1e6])
    assert np.all(O.round_e4m3(big) == 448.0) and np.all(O.round_e4m3(-big) == -448.0)
    assert O.round_e4m3(np.array([2.0 ** -10]))[0] == 0.0           # tie with 0 (even)
    g = np.random.default_rng(1).uniform(-500, 500, 20000)
    r = O.round_e4m3(g)
    assert np.array_equal(O.round_e4m3(-g), -r)
    assert np.all(np.isin(np.abs(r), np.concatenate([[0.0], xs])))
    # nearest: no representable value is closer than the result
    inside = np.abs(g) <= 448
    d = np.abs(g[inside, None] - np.concatenate([-xs[::-1], [0.0], xs])[None, :])
    assert np.all(np.abs(g[inside] - r[inside]) <= d.min(axis=1) + 1e-15)


def test_pow2_scale():
    g = np.random.default_rng(2)
    for m in np.concatenate([g.uniform(1e-6, 1e6, 500), [448.0, 224.0, 1.0, 2.0 ** -20]]):
        s = O.pow2_scale(float(m))
        assert math.frexp(s)[0] == 0.5                      # a power of two
        assert 224.0 < s * m <= 448.0
    assert O.pow2_scale(0.0) == 1.0


def test_fp8_network_is_exact_when_every_value_is_representable():
    """Inputs are basis vectors; first-layer weights have at most 4
    significant bits; the second layer has one power-of-two weight per row;
    biases are 0. Every scaled input, weight and hidden activation is then an
    E4M3 value, so the FP8 forward pass equals the FP64 one bit for bit."""
    g = np.random.default_rng(3)
    n_in, width, n_out = 24, 16, 5
    W0 = g.integers(-15, 16, size=(width, n_in)) * 2.0 ** g.integers(-3, 2, size=(width, n_in))
    W1 = np.zeros((width, width))
    W1[np.arange(width), g.permutation(width)] = g.choice([-2.0, -0.5, 0.25, 1.0, 4.0], size=width)
    W2 = g.integers(-15, 16, size=(n_out, width)) * 0.5
    weights = [(W0, np.zeros(width)), (W1, np.zeros(width)), (W2, np.zeros(n_out))]
    X = np.eye(n_in)
    fp8 = O.fp8_scales(1.0, weights)
    assert len(fp8[0]) == 3 and all(math.frexp(x)[0] == 0.5 for x in fp8[0] + fp8[1])
    got = O.mlp_forward(X, weights, 0, "fp8", fp8=fp8)
    want = O.mlp_forward(X, weights, 0, "f64")
    assert np.array_equal(got, want)
    assert np.abs(want).max() > 0
