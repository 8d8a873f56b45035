"""Pins of the oracle's BF16 network modes.

'bf16_plain' rounds every operand once to bfloat16. 'bf16' (the BF16
tensor-core path) does that in the first layer only; every later layer
takes activations and weights as two-term bfloat16 pairs (hi = BF16(x),
lo = BF16(x - hi)) and sums hi.hi + hi.lo + lo.hi, leaving out lo.lo."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("x,hi,lo", [
    (1.0, 1.0, 0.0),
    (1.0 + 2**-9 + 2**-13, 1.0, 2**-9 + 2**-13),       # below half a BF16 step: hi = 1, lo exact
    (1.0 + 2**-8, 1.0, 2**-8),                          # a tie: hi to even
    (1.0 + 3 * 2**-8, 1.0 + 2**-6, -2**-8),             # tie between 1 + 2^-7 and 1 + 2^-6: even is 2^-6
    (1.0 + 2**-7 + 2**-20, 1.0 + 2**-7, 2**-20),
    # 17 significant bits: lo itself is rounded (by hand: x - hi = -2^-8 + 2^-17 + 2^-18
    # = -2^-9 (2 - 2^-8 - 2^-9), whose 8-bit rounding is -2^-9 (2 - 2^-7))
    (1.0 + 2**-8 + 2**-17 + 2**-18, 1.0 + 2**-7, -2**-8 + 2**-16),
    (-3.0 - 2**-10, -3.0, -2**-10),
])
def test_split_bf16_by_hand(x, hi, lo):
    h, l = O.split_bf16(np.array([x]))
    assert h[0] == hi and l[0] == lo


def test_split_bf16_keeps_sixteen_bits():
    g = np.random.default_rng(3)
    x = g.normal(size=100000) * 10.0 ** g.integers(-6, 6, 100000)
    hi, lo = O.split_bf16(x)
    # two roundings to 8 significant bits: |x - hi - lo| <= 2^-8 |x - hi| <= 2^-16 |x|
    # (plus the float32 step of the conversion, 2^-24 |x|)
    assert np.all(np.abs(x - hi - lo) <= (2.0**-16 + 2.0**-23) * np.abs(x))
    # hi is the single-term rounding
    assert np.array_equal(hi, O.round_bf16(x))


def _net():
    # 1 -> 1 -> 1 network (values chosen by hand):
    #   input x = 1 + 2^-9            BF16: 1 (below half a step)
    #   W0 = 1, b0 = 2^-9 (FP32 bias, not rounded)
    #   z0 = 1 + 2^-9 in both BF16 modes (1 + 2^-8 + 0 in FP64: x W0 + b0 = 1 + 2^-8)
    #   activation h: plain rounds to 1; two-term keeps hi 1, lo 2^-9
    #   W1 = 1 + 2^-9: plain rounds to 1; two-term hi 1, lo 2^-9
    #   out: plain 1; two-term 1 + 2^-9 + 2^-9 = 1 + 2^-8 (lo.lo = 2^-18 left out)
    return [(np.array([[1.0]]), np.array([2**-9])), (np.array([[1.0 + 2**-9]]), np.array([0.0]))]


def test_bf16_modes_by_hand():
    X = np.array([[1.0 + 2**-9]])
    w = _net()
    assert O.mlp_forward(X, w, 0, "bf16_plain")[0, 0] == 1.0
    assert O.mlp_forward(X, w, 0, "bf16")[0, 0] == 1.0 + 2**-8
    assert O.mlp_forward(X, w, 0, "f64")[0, 0] == (1.0 + 2**-8) * (1.0 + 2**-9)


def test_bf16_two_term_layers_are_near_exact():
    """With first-layer operands exact in BF16, only the later layers round:
    the two-term form keeps them within a few 2^-16 of the FP64 network,
    while single rounding is off by about 2^-9."""
    g = np.random.default_rng(11)
    X = O.round_bf16(g.normal(size=(400, 32)))
    W0 = O.round_bf16(g.normal(size=(64, 32)) / 6)
    ws = [(W0, g.normal(size=64) * 0.1)]
    for fo in (64, 64, 12):
        ws.append((g.normal(size=(fo, 64)) / 8, g.normal(size=fo) * 0.1))
    z64 = O.mlp_forward(X, ws, 0, "f64")
    scale = np.abs(z64).max()
    e2 = np.abs(O.mlp_forward(X, ws, 0, "bf16") - z64).max() / scale
    e1 = np.abs(O.mlp_forward(X, ws, 0, "bf16_plain") - z64).max() / scale
    assert e2 < 2.0**-13, e2
    assert e1 > 2.0**-11, e1
    # the first layer alone is the same in both modes
    one = ws[:1]
    assert np.array_equal(O.mlp_forward(X, one, 0, "bf16"), O.mlp_forward(X, one, 0, "bf16_plain"))
