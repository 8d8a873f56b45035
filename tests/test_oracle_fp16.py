"""Pins of the oracle's FP16 network mode (the operand rounding of the
FP16 tensor-core path): IEEE binary16 rounding to nearest even with
saturation at the largest finite value, applied to the inputs, the weights
and the hidden activations, with float64 sums."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("x,expect", [
    (1.0, 1.0),
    (1.0 + 2**-11, 1.0),                    # half an ulp above 1: tie, to even
    (1.0 + 3 * 2**-11, 1.0 + 2**-9),        # tie between odd and even: up to the even one
    (1.0 + 2**-12, 1.0),                    # a quarter ulp: down
    (-2.5, -2.5),
    (65504.0, 65504.0),
    (65519.0, 65504.0),                     # below the overflow threshold: rounds down
    (70000.0, 65504.0),                     # saturates instead of overflowing
    (-1e9, -65504.0),
    (2**-25, 0.0),                          # half the smallest subnormal: tie, to even (zero)
    (3 * 2**-25, 2**-23),                   # 1.5 subnormal steps: tie, to the even step
    (2**-24, 2**-24),
])
def test_fp16_rounding_ties_to_even_and_saturates(x, expect):
    assert O.round_fp16_sat(np.array([x]))[0] == expect


def test_fp16_rounding_matches_torch_inside_the_range():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(6)
    x = (g.normal(size=20000) * 10.0 ** g.integers(-9, 5, 20000)).astype(np.float32)
    x = x[np.abs(x) < 65504.0]
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(O.round_fp16_sat(x), ref)


def _net():
    # 1 -> 1 -> 1 network; every value chosen so that FP16 and BF16 round it
    # differently (by hand):
    #   input 1 + 2^-12        FP16: 1 (quarter ulp)         BF16: 1
    #   W0 = 1 + 2^-9          FP16: exact (10-bit fraction) BF16: 1
    #   b0 = 2^-12 (bias, FP32, not rounded)
    #   z0 = x W0 + b0         FP16: 1 + 2^-9 + 2^-12 -> activation rounds to 1 + 2^-9
    #                          BF16: 1 + 2^-12        -> 1
    #   out = 2 h              FP16: 2 + 2^-8            BF16 (single rounding): 2
    return [(np.array([[1.0 + 2**-9]]), np.array([2**-12])), (np.array([[2.0]]), np.array([0.0]))]


def test_fp16_network_rounds_inputs_weights_and_activations():
    X = np.array([[1.0 + 2**-12]])
    w = _net()
    assert O.mlp_forward(X, w, 0, "fp16")[0, 0] == 2.0 + 2**-8
    assert O.mlp_forward(X, w, 0, "bf16_plain")[0, 0] == 2.0
    # two-term BF16 after the first layer: the activation 1 + 2^-12 survives as hi 1, lo 2^-12
    assert O.mlp_forward(X, w, 0, "bf16")[0, 0] == 2.0 + 2**-11
    exact = 2.0 * ((1.0 + 2**-12) * (1.0 + 2**-9) + 2**-12)
    assert O.mlp_forward(X, w, 0, "f64")[0, 0] == exact


def test_fp16_network_saturates_inputs_and_activations():
    w = [(np.array([[4.0]]), np.array([0.0])), (np.array([[0.5]]), np.array([1.0]))]
    # input 1e5 -> 65504; z0 = 262016 -> activation 65504; out = 32752 + 1
    assert O.mlp_forward(np.array([[1e5]]), w, 0, "fp16")[0, 0] == 32753.0


def test_fp16_network_is_exact_when_every_value_is_representable():
    g = np.random.default_rng(8)
    X = g.integers(-8, 9, size=(50, 16)) / 8.0
    w = [(g.integers(-4, 5, size=(8, 16)) / 4.0, g.integers(-4, 5, size=8) / 4.0),
         (g.integers(-4, 5, size=(3, 8)) / 4.0, np.zeros(3))]
    # every hidden activation is a multiple of 1/32 below 2^10: representable
    assert np.array_equal(O.mlp_forward(X, w, 0, "fp16"), O.mlp_forward(X, w, 0, "f64"))
