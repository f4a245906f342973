"""Pins of the FP64 proposal-network reference (no GPU): BF16 rounding
against its definition, GELU closed forms, the forward against a per-sample
loop, the backward against central finite differences of the loss, and the
first Adam step against its closed form."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding():
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1.0 + 2 ** -9) == 1.0                  # below the midpoint
    assert mlp.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7     # above the midpoint
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0                  # midpoint: ties to the even 1.0
    assert mlp.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6     # midpoint: ties to the even neighbour
    assert mlp.bf16_round(-3.0) == -3.0 and mlp.bf16_round(0.0) == 0.0
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16_round(x)
    # representable: at most 8 significant bits; nearest: within half an ulp
    m, e = np.frexp(r)
    assert np.all(m * 256 == np.round(m * 256))
    assert np.all(np.abs(r - x) <= np.ldexp(1.0, np.frexp(x)[1] - 9) + 1e-300)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    # z = 1: tanh(sqrt(2/pi) * 1.044715) = 0.6823..., GELU(1) = 0.8411920...
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.84119199) < 1e-8
    # GELU(-z) = GELU(z) - z (Phi(-z) = 1 - Phi(z); the tanh form keeps it)
    z = np.linspace(-5, 5, 101)
    assert np.allclose(mlp.gelu(-z), mlp.gelu(z) - z, atol=1e-15)
    # the tanh form stays within 4.8e-4 of the definition z Phi(z) (erf)
    zz = np.linspace(-8, 8, 16001)
    exact = 0.5 * zz * (1 + np.array([math.erf(v / math.sqrt(2)) for v in zz]))
    gap = np.abs(mlp.gelu(zz) - exact)
    assert gap.max() < 4.8e-4 and gap.max() > 4.0e-4
    z = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, mlp.gelu_grad(z), atol=1e-8)


def test_forward_matches_per_sample_loop():
    p = mlp.init_params(3)
    rng = np.random.default_rng(1)
    x = mlp.features(rng.uniform(0, 1, (5, 3)), rng.uniform(0, 1, (5, 3)), [0, 0, 0], [1, 1, 1])
    logits, _ = mlp.forward(p, x)
    W1, W2, W3 = (mlp.bf16_round(p[k]) for k in ("W1", "W2", "W3"))
    for i in range(len(x)):
        a0 = [float(mlp.bf16_round(v)) for v in x[i]]
        a1 = []
        for j in range(mlp.D_H):
            z = sum(a0[k] * W1[k, j] for k in range(mlp.D_PAD)) + p["b1"][j]
            a1.append(float(mlp.bf16_round(0.5 * z * (1 + math.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3))))))
        a2 = []
        for j in range(mlp.D_H):
            z = sum(a1[k] * W2[k, j] for k in range(mlp.D_H)) + p["b2"][j]
            a2.append(float(mlp.bf16_round(0.5 * z * (1 + math.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3))))))
        for j in range(0, mlp.D_OUT, 37):
            z = sum(a2[k] * W3[k, j] for k in range(mlp.D_H)) + p["b3"][j]
            assert abs(z - logits[i, j]) < 1e-9


def test_backward_matches_finite_differences():
    """Without the BF16 roundings (identity), the analytic gradient is the
    derivative of the loss; check it by central differences."""
    p = mlp.init_params(5)
    rng = np.random.default_rng(2)
    x = mlp.features(rng.uniform(0, 1, (7, 3)), rng.uniform(0, 1, (7, 3)), [0, 0, 0], [1, 1, 1])
    y = (rng.uniform(size=(7, mlp.D_OUT)) < 0.05).astype(float)
    orig = mlp.bf16_round
    mlp.bf16_round = lambda v: np.asarray(v, np.float64)
    try:
        logits, cache = mlp.forward(p, x)
        g = mlp.backward(p, cache, logits, y)
        for k, idx in (("W1", (2, 5)), ("W1", (0, 100)), ("b1", (7,)), ("W2", (3, 17)), ("b2", (90,)),
                       ("W3", (11, 200)), ("W3", (127, 3)), ("b3", (255,))):
            h = 1e-6
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pp[k][idx] += h
            lp = mlp.bce_loss(mlp.forward(pp, x)[0], y)
            pp[k][idx] -= 2 * h
            lm = mlp.bce_loss(mlp.forward(pp, x)[0], y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-7 + 1e-5 * abs(fd), (k, idx, fd, g[k][idx])
    finally:
        mlp.bf16_round = orig


def test_first_adam_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the update is
    -lr g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -1e-3, 0.0])}
    out = mlp.adam_step(p, g, {}, lr=0.01, eps=1e-8)
    expect = p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(out["w"], expect, rtol=1e-12, atol=0)


def test_later_adam_steps_closed_form():
    """With a constant gradient the bias-corrected moments stay g and g^2,
    so every step is -lr g / (|g| + eps); with the gradient g then -g, the
    second step's first moment is -(1 - b1)^2 g / (1 - b1^2) = -g (1 - b1) /
    (1 + b1) and its second moment still g^2."""
    g = np.array([0.3, -2.0, 1e-3])
    p, state = {"w": np.zeros(3)}, {}
    for t in range(1, 4):
        p = mlp.adam_step(p, {"w": g}, state, lr=0.01, b1=0.9, b2=0.999, eps=1e-8)
        assert np.allclose(p["w"], -0.01 * t * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    p, state = {"w": np.zeros(3)}, {}
    p1 = mlp.adam_step(p, {"w": g}, state, lr=0.01, b1=0.9, b2=0.999, eps=1e-8)
    p2 = mlp.adam_step(p1, {"w": -g}, state, lr=0.01, b1=0.9, b2=0.999, eps=1e-8)
    step2 = -0.01 * (-g * (1 - 0.9) / (1 + 0.9)) / (np.abs(g) + 1e-8)
    assert np.allclose(p2["w"] - p1["w"], step2, rtol=1e-10, atol=0)
    assert state["t"] == 2


def test_top4_order():
    z = np.array([[0.1, 5.0, 3.0, 5.0, -1.0, 4.0] + [0.0] * 250])
    assert mlp.top4(z).tolist() == [[1, 3, 5, 2]]


def test_features_map_the_extent_to_the_unit_cube():
    """End points at the low / high corner of the extent map to -1 / +1,
    the centre to 0, points far outside clamp to -4 / +4, a flat axis maps
    through a unit span, and the ten padding inputs are zero."""
    lo, hi = np.array([1.0, -2.0, 3.0]), np.array([3.0, 2.0, 3.0])
    F = np.array([lo, (lo + hi) / 2, [100.0, -100.0, 3.0]])
    E = np.array([hi, lo, [1.0, 2.0, 3.5]])
    x = mlp.features(F, E, lo, hi)
    assert x.shape == (3, mlp.D_PAD)
    np.testing.assert_array_equal(x[0, :6], [-1, -1, -1, 1, 1, -1])
    np.testing.assert_array_equal(x[1, :6], [0, 0, -1, -1, -1, -1])
    np.testing.assert_array_equal(x[2, :6], [4, -4, -1, -1, 1, 0])
    assert not x[:, 6:].any()
