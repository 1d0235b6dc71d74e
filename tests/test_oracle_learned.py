"""Pins of the oracle's learned-filter network (oracle/mlp.py) and of its moving-source
renderer (oracle.render_moving): finite differences, closed forms, and reduction to the
static renderer."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1502_03162_gb300 import synth

REFL = 200


def _params(rng, refl_len=REFL, scale=1.0):
    p = np.zeros(mlp.param_count(refl_len))
    o = 0
    for (fan_in, fan_out) in zip(mlp.layer_sizes(refl_len)[:-1], mlp.layer_sizes(refl_len)[1:]):
        n = fan_in * fan_out
        p[o:o + n] = rng.uniform(-1, 1, n) * scale * np.sqrt(6.0 / fan_in)
        o += n
        p[o:o + fan_out] = rng.uniform(-0.1, 0.1, fan_out)
        o += fan_out
    return p


def test_param_count_matches_layer_shapes():
    # 5 -> 256 -> 256 -> 256 -> 200
    assert mlp.param_count(200) == 256 * 5 + 256 + 2 * (256 * 256 + 256) + 200 * 256 + 200 == 184520


def test_features_closed_form():
    x = mlp.features([0.0, np.pi / 2], [np.pi, 0.0], [-1, 1])
    np.testing.assert_allclose(x, [[0, 1, 0, -1, -1], [1, 0, 0, 1, 1]], atol=1e-15)


def test_softplus_and_sigmoid_closed_forms():
    z = np.array([-800.0, -3.0, 0.0, 2.5, 800.0])
    np.testing.assert_allclose(mlp.softplus(z), [0.0, np.log1p(np.exp(-3.0)), np.log(2.0),
                                                 np.log1p(np.exp(2.5)), 800.0], rtol=1e-15)
    np.testing.assert_allclose(mlp.sigmoid(z), [0.0, 1 / (1 + np.exp(3.0)), 0.5,
                                                1 / (1 + np.exp(-2.5)), 1.0], rtol=1e-15)


def test_zero_network_output_and_gradient_closed_form():
    """All parameters zero: every tap is softplus(0) = log 2, and the only non-zero
    gradient is that of b4: dL/db4_j = mean_b (log 2 - T_bj) * sigmoid(0)."""
    rng = np.random.default_rng(0)
    B = 7
    X = mlp.features(rng.uniform(-3, 3, B), rng.uniform(-1, 1, B), rng.choice([-1, 1], B))
    T = rng.random((B, REFL))
    p = np.zeros(mlp.param_count(REFL))
    g, _ = mlp.forward(p, X, REFL)
    np.testing.assert_allclose(g, np.log(2.0), rtol=1e-15)
    L, grad = mlp.loss_and_grad(p, X, T, REFL)
    assert L == pytest.approx(0.5 * np.sum((np.log(2.0) - T) ** 2) / B, rel=1e-14)
    nb4 = REFL
    np.testing.assert_allclose(grad[-nb4:], 0.5 * np.mean(np.log(2.0) - T, axis=0), rtol=1e-13)
    assert not grad[:-nb4].any()


@pytest.mark.parametrize("refl_len", [200, 7])
def test_gradient_matches_central_differences(refl_len):
    rng = np.random.default_rng(1)
    B = 5
    X = mlp.features(rng.uniform(-3, 3, B), rng.uniform(-1, 1, B), rng.choice([-1, 1], B))
    T = rng.random((B, refl_len))
    p = _params(rng, refl_len)
    _, grad = mlp.loss_and_grad(p, X, T, refl_len)
    # indices in every weight matrix and every bias vector
    s = mlp.layer_sizes(refl_len)
    idx, o = [], 0
    for i in range(len(s) - 1):
        n = s[i + 1] * s[i]
        idx += list(rng.integers(o, o + n, 12))
        o += n
        idx += list(rng.integers(o, o + s[i + 1], 4))
        o += s[i + 1]
    num = mlp.numeric_grad(p, X, T, refl_len, idx)
    ana = grad[idx]
    scale = np.max(np.abs(ana))
    np.testing.assert_allclose(ana, num, atol=1e-7 * scale, rtol=1e-5)


def test_adam_constant_gradient_steps_closed_form():
    """With a constant gradient g, the bias-corrected moments equal g and g^2 at every step,
    so each step moves a parameter by exactly lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-3, 1e-8
    q = p.copy()
    for t in range(1, 6):
        q, m, v = mlp.adam_step(q, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(q, p - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(3)
    az = rng.uniform(-1.4, 1.4, 64)
    el = rng.uniform(-0.8, 4.0, 64)
    ear = rng.choice([-1.0, 1.0], 64)
    X = mlp.features(az, el, ear)
    T = np.abs(np.sin(np.outer(np.cos(az) + ear, np.arange(12) / 4.0)))
    p = _params(rng, 12, scale=0.5)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0, _ = mlp.loss_and_grad(p, X, T, 12)
    for t in range(1, 151):
        _, g = mlp.loss_and_grad(p, X, T, 12)
        p, m, v = mlp.adam_step(p, g, m, v, t, 3e-3)
    L1, _ = mlp.loss_and_grad(p, X, T, 12)
    assert L1 < 0.05 * L0


# ------------------------------------------------------------------- moving sources
def _static_tables(rng, S, n_seg, k):
    G = synth.reflection_bank(rng, S, n_refl=24)
    idx, w, nnz = oracle.topk(G, k)                   # [S][2][k]
    rep = lambda a: np.repeat(a[:, None], n_seg, axis=1)  # noqa: E731
    return idx, w, nnz, rep(idx), rep(w), rep(nnz)


def test_moving_with_constant_filters_equals_static_render():
    """A crossfade between identical filters is that filter: equals render_sparse."""
    rng = np.random.default_rng(4)
    S, L, seg = 3, 1500, 256
    y = synth.sources_ar1(rng, S, L)
    res = synth.resonance(rng)
    idx, w, nnz, mi, mw, mn = _static_tables(rng, S, (L + seg - 1) // seg, 8)
    got = oracle.render_moving(y, mi, mw, mn, seg, REFL, res)
    ref = oracle.render_sparse(y, np.arange(S, dtype=np.int32), idx, w, nnz, REFL, res)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_moving_single_segment_equals_static_render():
    rng = np.random.default_rng(5)
    S, L = 2, 700
    y = synth.sources_ar1(rng, S, L)
    res = synth.resonance(rng)
    idx, w, nnz, mi, mw, mn = _static_tables(rng, S, 1, 16)
    got = oracle.render_moving(y, mi, mw, mn, 4096, REFL, res)
    ref = oracle.render_sparse(y, np.arange(S, dtype=np.int32), idx, w, nnz, REFL, res)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_moving_crossfade_ramp_closed_form():
    """DC source, single-tap filters g_j = c_j delta, identity resonance: the output in
    segment j >= 1 is the ramp (1 - a) c_{j-1} + a c_j, a = (n - j seg + 1) / seg."""
    seg, n_seg = 16, 5
    L = seg * n_seg
    y = np.ones((1, L), np.float32)
    c = np.array([1.0, 3.0, -0.0, 2.0, 0.5], np.float32)
    idx = np.zeros((1, n_seg, 2, 1), np.uint16)
    w = np.zeros((1, n_seg, 2, 1), np.float32)
    w[0, :, 0, 0] = c
    w[0, :, 1, 0] = 2 * c
    nnz = np.ones((1, n_seg, 2), np.uint8)
    res = np.zeros((2, 4), np.float32)
    res[:, 0] = 1.0
    out = oracle.render_moving(y, idx, w, nnz, seg, 1, res)
    assert out.shape == (2, L + 3)
    n = np.arange(L)
    j = n // seg
    a = (n - j * seg + 1) / seg
    ramp = np.where(j == 0, c[0], (1 - a) * c[np.maximum(j - 1, 0)] + a * c[j])
    np.testing.assert_allclose(out[0, :L], ramp, rtol=1e-15)
    np.testing.assert_allclose(out[1, :L], 2 * ramp, rtol=1e-15)
    assert not out[:, L:].any()
