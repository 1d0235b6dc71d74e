"""Pins for the oracle's convolution, FFT, rendering and top-K functions.

Each check ties the oracle to something other than itself: closed forms, library routines
for special cases, brute force on tiny inputs, or identities the paper states (Eq. 2).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


# ----------------------------------------------------------------------------- direct conv
def test_conv_direct_impulse_returns_filter():
    rng = np.random.default_rng(0)
    h = rng.standard_normal(37)
    d = np.zeros(5)
    d[0] = 1.0
    out = oracle.conv_direct(d, h)
    assert out.shape == (41,)
    np.testing.assert_array_equal(out[:37], h)
    np.testing.assert_array_equal(out[37:], 0.0)
    # delayed impulse delays the filter
    d2 = np.zeros(5)
    d2[3] = 2.0
    out2 = oracle.conv_direct(h, d2)
    np.testing.assert_array_equal(out2[3:40], 2.0 * h)
    np.testing.assert_array_equal(out2[:3], 0.0)


def test_conv_direct_closed_forms():
    # boxcar * boxcar = trapezoid min(n+1, nx, ny, nx+ny-1-n)
    nx, ny = 7, 12
    out = oracle.conv_direct(np.ones(nx), np.ones(ny))
    n = np.arange(nx + ny - 1)
    expect = np.minimum.reduce([n + 1, np.full_like(n, nx), np.full_like(n, ny), nx + ny - 1 - n])
    np.testing.assert_array_equal(out, expect)
    # geometric sequences: sum_{j<=n} a^j b^(n-j) = (b^(n+1) - a^(n+1)) / (b - a) for n < min
    a, b = 0.9, -0.55
    x = a ** np.arange(40)
    y = b ** np.arange(30)
    out = oracle.conv_direct(x, y)
    n = np.arange(30)
    expect = (b ** (n + 1) - a ** (n + 1)) / (b - a)
    assert rel_err(out[:30], expect) < 1e-13


def test_conv_direct_matches_numpy_and_is_commutative_and_linear():
    rng = np.random.default_rng(1)
    x, y, z = rng.standard_normal(13), rng.standard_normal(29), rng.standard_normal(29)
    out = oracle.conv_direct(x, y)
    assert rel_err(out, np.convolve(x, y)) < 1e-14
    assert rel_err(oracle.conv_direct(y, x), out) < 1e-15
    lin = oracle.conv_direct(x, 2.0 * y - 3.0 * z)
    assert rel_err(lin, 2.0 * out - 3.0 * oracle.conv_direct(x, z)) < 1e-13


def test_conv_sparse_equals_zero_filled_dense():
    rng = np.random.default_rng(2)
    refl_len = 200
    idx = np.sort(rng.choice(refl_len, 16, replace=False)).astype(np.int32)
    w = rng.exponential(size=16)
    y = rng.standard_normal(333)
    g = np.zeros(refl_len)
    g[idx] = w
    sp = oracle.conv_sparse(idx, w, y, refl_len)
    assert sp.shape == (333 + refl_len - 1,)
    assert rel_err(sp, oracle.conv_direct(g, y)) < 1e-14
    # repeated indices add up
    sp2 = oracle.conv_sparse(np.array([5, 5], np.int32), np.array([1.0, 2.0]), y, 10)
    sp3 = oracle.conv_sparse(np.array([5], np.int32), np.array([3.0]), y, 10)
    assert rel_err(sp2, sp3) < 1e-15


def test_cascade_associativity_eq2():
    """y * x = (y * f) * g = (y * g) * f  with x = f * g (Eq. 2)."""
    rng = np.random.default_rng(3)
    f = rng.standard_normal(32)
    idx = np.sort(rng.choice(200, 16, replace=False)).astype(np.int32)
    w = rng.exponential(size=16)
    g = np.zeros(200)
    g[idx] = w
    y = rng.standard_normal(500)
    x = oracle.conv_direct(f, g)
    a = oracle.conv_direct(x, y)
    b = oracle.conv_sparse(idx, w, oracle.conv_direct(f, y), 200)
    c = oracle.conv_direct(f, oracle.conv_sparse(idx, w, y, 200))
    assert a.shape == b.shape == c.shape == (500 + 231 - 1,)
    assert rel_err(b, a) < 1e-13
    assert rel_err(c, a) < 1e-13


# ------------------------------------------------------------------------------------ FFT
def test_dft_definition_special_cases():
    n = 16
    d = np.zeros(n)
    d[0] = 1
    np.testing.assert_allclose(oracle.dft(d), np.ones(n), atol=1e-15)
    np.testing.assert_allclose(oracle.dft(np.ones(n)), np.eye(1, n, 0)[0] * n, atol=1e-12)
    # shifted impulse -> pure phase exp(-2 pi i k s / n)
    s = 3
    d = np.zeros(n)
    d[s] = 1
    k = np.arange(n)
    np.testing.assert_allclose(oracle.dft(d), np.exp(-2j * np.pi * k * s / n), atol=1e-14)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    np.testing.assert_allclose(oracle.dft(x), np.fft.fft(x), atol=1e-12)
    np.testing.assert_allclose(oracle.dft(oracle.dft(x), inverse=True), x, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_fft_equals_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = oracle.fft(x)
    assert np.max(np.abs(X - oracle.dft(x))) < 1e-12 * max(1, n)
    assert np.max(np.abs(oracle.fft(X, inverse=True) - x)) < 1e-13 * max(1, n)
    # Parseval: sum |x|^2 = (1/n) sum |X|^2
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / n) < 1e-11 * n


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12))


def test_conv_fft_equals_direct():
    rng = np.random.default_rng(5)
    for nx, ny in [(1, 1), (3, 5), (231, 700), (64, 64), (17, 1)]:
        x, y = rng.standard_normal(nx), rng.standard_normal(ny)
        d = oracle.conv_direct(x, y)
        f = oracle.conv_fft(x, y)
        assert f.shape == d.shape
        assert np.max(np.abs(f - d)) < 1e-12 * max(1.0, np.max(np.abs(d)))


# ------------------------------------------------------------------------------ rendering
def _tables(rng, n_dirs, k, refl_len=200, res_len=32):
    G = synth.reflection_bank(rng, n_dirs, n_refl=max(k + 4, 8), refl_len=refl_len)
    idx, w, nnz = oracle.topk(G, k)
    res = synth.resonance(rng, res_len)
    return idx, w, nnz, res


def test_render_impulse_returns_dense_hrir():
    rng = np.random.default_rng(6)
    idx, w, nnz, res = _tables(rng, 3, 16)
    y = np.zeros((1, 10), np.float32)
    y[0, 0] = 1.0
    out = oracle.render_sparse(y, np.array([2], np.int32), idx, w, nnz, 200, res)
    H = oracle.dense_hrirs(idx, w, nnz, 200, res)[2]
    assert out.shape == (2, 10 + 231 - 1)
    np.testing.assert_allclose(out[:, :231], H, atol=1e-15)
    np.testing.assert_array_equal(out[:, 231:], 0.0)
    # dense HRIR is f * g with g written densely
    g0 = np.zeros(200)
    g0[idx[2, 0, :nnz[2, 0]]] = w[2, 0, :nnz[2, 0]]
    np.testing.assert_allclose(H[0], np.convolve(res[0].astype(np.float64), g0), atol=1e-15)


def test_render_three_ways_agree_and_are_linear_in_sources():
    rng = np.random.default_rng(7)
    idx, w, nnz, res = _tables(rng, 5, 8)
    S, L, ld = 4, 301, 304
    y = np.full((S, ld), np.float32(1e30))            # padding beyond L must never be read
    y[:, :L] = rng.standard_normal((S, L)).astype(np.float32)
    dirs = np.array([4, 0, 4, 2], np.int32)
    a = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
    b = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L, order=1)
    c = oracle.render_dense(y, dirs, idx, w, nnz, 200, res, length=L)
    d = oracle.render_fft(y, dirs, idx, w, nnz, 200, res, length=L)
    assert a.shape == (2, L + 230)
    scale = np.max(np.abs(a))
    for other in (b, c, d):
        assert np.max(np.abs(other - a)) < 1e-12 * scale
    singles = sum(oracle.render_sparse(y[s:s + 1], dirs[s:s + 1], idx, w, nnz, 200, res, length=L)
                  for s in range(S))
    assert np.max(np.abs(singles - a)) < 1e-12 * scale


def test_render_at_equals_full_render():
    rng = np.random.default_rng(11)
    idx, w, nnz, res = _tables(rng, 6, 12)
    S, L = 5, 400
    y = rng.standard_normal((S, L)).astype(np.float32)
    dirs = rng.integers(0, 6, S).astype(np.int32)
    full = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res)
    pos = np.array([0, 1, 17, 199, 230, 399, 400, 628, 629, 630, -1, 10_000])
    at = oracle.render_at(y, dirs, idx, w, nnz, 200, res, pos)
    inside = (pos >= 0) & (pos < full.shape[1])
    assert np.max(np.abs(at[:, inside] - full[:, pos[inside]])) < 1e-12 * np.max(np.abs(full))
    assert not at[:, ~inside].any()


def test_render_edge_cases():
    rng = np.random.default_rng(8)
    idx, w, nnz, res = _tables(rng, 2, 4)
    # L = 0 -> empty output; S = 0 -> zeros of full length
    out = oracle.render_sparse(np.zeros((1, 4), np.float32), np.zeros(1, np.int32), idx, w, nnz,
                               200, res, length=0)
    assert out.shape == (2, 0)
    out = oracle.render_sparse(np.zeros((0, 7), np.float32), np.zeros(0, np.int32), idx, w, nnz,
                               200, res)
    assert out.shape == (2, 7 + 230) and not out.any()
    # L = 1 source: output is the HRIR scaled by the sample
    y = np.array([[3.0]], np.float32)
    out = oracle.render_sparse(y, np.array([1], np.int32), idx, w, nnz, 200, res)
    H = oracle.dense_hrirs(idx, w, nnz, 200, res)[1]
    np.testing.assert_allclose(out, 3.0 * H, rtol=1e-14, atol=1e-15)
    # a direction with no taps renders silence
    nnz0 = nnz.copy()
    nnz0[1] = 0
    out = oracle.render_sparse(y, np.array([1], np.int32), idx, w, nnz0, 200, res)
    assert not out.any()
    with pytest.raises(ValueError):
        oracle.render_sparse(y, np.array([2], np.int32), idx, w, nnz, 200, res)


# ----------------------------------------------------------------------------------- top-K
def _brute_topk(row, k):
    cand = [(float(v), j) for j, v in enumerate(row) if v > 0]
    kept = sorted(cand, key=lambda t: (-t[0], t[1]))[:k]
    kept = sorted(kept, key=lambda t: t[1])
    idx = [j for _, j in kept] + [0] * (k - len(kept))
    w = [v for v, _ in kept] + [0.0] * (k - len(kept))
    return idx, w, len(kept)


def test_topk_matches_bruteforce_sort():
    rng = np.random.default_rng(9)
    G = synth.reflection_bank(rng, 40, n_refl=30)
    G[0, 0, :] = 0                      # empty row
    G[1, 1, :] = -1                     # negatives are never taps
    G[2, 0, 5] = np.nan                 # NaN never a tap
    G[3, 0, :] = 0
    G[3, 0, [7, 3, 11, 2]] = 0.5        # ties -> smaller index first
    G[3, 0, 100] = 0.25
    for k in (0, 1, 3, 8, 16, 32, 40):
        idx, w, nnz = oracle.topk(G, k)
        for d, e in itertools.product(range(40), range(2)):
            bi, bw, bn = _brute_topk(G[d, e], k)
            assert nnz[d, e] == bn
            assert list(idx[d, e]) == bi
            assert list(w[d, e].astype(np.float64)) == [float(np.float32(v)) for v in bw]
    idx, w, nnz = oracle.topk(G, 3)
    assert list(idx[3, 0]) == [2, 3, 7] and nnz[3, 0] == 3


def test_topk_indices_ascending_and_bounded():
    rng = np.random.default_rng(10)
    G = synth.reflection_bank(rng, 50, n_refl=48)
    idx, w, nnz = oracle.topk(G, 16)
    assert np.all(nnz == 16)
    assert np.all(np.diff(idx.astype(np.int64), axis=-1) > 0)
    assert np.all(idx < 200) and np.all(w > 0)
    # the kept weights are the 16 largest of each row
    kth = -np.sort(-G, axis=-1)[..., 15]
    assert np.all(np.min(w, axis=-1) >= kth)
