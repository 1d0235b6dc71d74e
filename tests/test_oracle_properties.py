"""Property-based pins of the oracle (hypothesis): the definitions and invariants the paper
fixes, on generated inputs rather than fixed seeds.

  * direct convolution (Sec. I footnote 2) equals the brute-force double sum and is
    commutative and bilinear;
  * sparse convolution (Eq. 2) equals direct convolution with the zero-filled filter;
  * the radix-2 FFT equals the O(P^2) DFT, and FFT convolution (footnote 3) equals direct
    convolution;
  * top-K keeps the K largest strictly positive entries, larger value first and the smaller
    index on ties, stored in ascending index order (brute force by sorting);
  * the cascade (y * g) * f renders like y * (f * g) (Eqs. 1-2) and the mix is linear in the
    sources;
  * the multiplicative reflection update (Eq. 4) keeps G >= 0 (zeros stay zero) and never
    increases the residual; the L1-NNLS solution (Eq. 14) is feasible, meets the KKT
    conditions and no nearby feasible point has a lower objective; the resonance solve
    (Eqs. 9-11) zeroes the gradient of the least-squares objective;
  * the moving-source render is the per-segment linear crossfade between consecutive
    segments' filters (brute force with dense filters and numpy.convolve).
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402
from hypothesis.extra import numpy as hnp  # noqa: E402

import oracle  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None, derandomize=True)
finite = st.floats(-4.0, 4.0, allow_nan=False, allow_infinity=False, width=64)


def vec(min_size=1, max_size=40):
    return hnp.arrays(np.float64, st.integers(min_size, max_size), elements=finite)


@SETTINGS
@given(vec(), vec())
def test_conv_direct_is_the_double_sum(x, y):
    out = oracle.conv_direct(x, y)
    ref = np.zeros(x.size + y.size - 1)
    for j in range(x.size):
        for m in range(y.size):
            ref[j + m] += x[j] * y[m]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.conv_direct(y, x), out, rtol=1e-12, atol=1e-12)


@SETTINGS
@given(vec(), vec(), vec(), st.floats(-3, 3, allow_nan=False))
def test_conv_direct_is_bilinear(x, y, z, a):
    n = min(y.size, z.size)
    y, z = y[:n], z[:n]
    lhs = oracle.conv_direct(x, a * y + z)
    rhs = a * oracle.conv_direct(x, y) + oracle.conv_direct(x, z)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-9)


@SETTINGS
@given(st.integers(1, 60), st.data())
def test_conv_sparse_equals_zero_filled_dense(refl_len, data):
    k = data.draw(st.integers(0, refl_len))
    idx = np.array(sorted(data.draw(st.sets(st.integers(0, refl_len - 1), min_size=k, max_size=k))),
                   dtype=np.int32)
    w = data.draw(hnp.arrays(np.float64, idx.size, elements=st.floats(0, 3, allow_nan=False)))
    y = data.draw(vec(1, 50))
    g = np.zeros(refl_len)
    g[idx] = w
    np.testing.assert_allclose(oracle.conv_sparse(idx, w, y, refl_len), oracle.conv_direct(g, y),
                               rtol=1e-12, atol=1e-12)


@SETTINGS
@given(st.integers(0, 6), st.data())
def test_fft_equals_dft_and_inverts(log2p, data):
    p = 1 << log2p
    re = data.draw(hnp.arrays(np.float64, p, elements=finite))
    im = data.draw(hnp.arrays(np.float64, p, elements=finite))
    x = re + 1j * im
    X = oracle.fft(x)
    np.testing.assert_allclose(X, oracle.dft(x), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(oracle.fft(X, inverse=True), x, rtol=1e-10, atol=1e-10)


@SETTINGS
@given(vec(1, 70), vec(1, 70))
def test_conv_fft_equals_direct(x, y):
    d = oracle.conv_direct(x, y)
    scale = max(1.0, np.abs(x).sum() * np.abs(y).max())
    np.testing.assert_allclose(oracle.conv_fft(x, y), d, rtol=0, atol=1e-11 * scale)


def _topk_brute(row, k):
    cand = [(-float(v), i) for i, v in enumerate(row) if v > 0]      # NaN > 0 is False
    cand.sort()
    keep = sorted(i for _, i in cand[:k])
    return keep


@settings(max_examples=120, deadline=None, derandomize=True)
@given(st.integers(1, 48), st.integers(0, 20), st.data())
def test_topk_against_sorting(refl_len, k, data):
    # few distinct values so that ties are common; negatives, zeros and NaN never selected
    pool = st.sampled_from([0.0, -1.0, float("nan"), 0.25, 0.5, 1.0, 1.5, 2.0, 1e-30, 3.0e5])
    row = np.array(data.draw(st.lists(pool, min_size=refl_len, max_size=refl_len)), np.float32)
    idx, w, nnz = oracle.topk(row[None], k)
    keep = _topk_brute(row, k)
    assert int(nnz[0]) == len(keep)
    assert list(idx[0, :len(keep)]) == keep
    np.testing.assert_array_equal(w[0, :len(keep)], row[keep])
    assert not idx[0, len(keep):].any() and not w[0, len(keep):].any()


@settings(max_examples=25, deadline=None, derandomize=True)
@given(st.integers(1, 4), st.integers(1, 300), st.integers(1, 8), st.data())
def test_render_cascade_and_linearity(S, L, k, data):
    rng = np.random.default_rng(data.draw(st.integers(0, 2 ** 31 - 1)))
    refl_len, res_len, n_dirs = 40, 7, 3
    G = rng.random((n_dirs, 2, refl_len)) * (rng.random((n_dirs, 2, refl_len)) < 0.3)
    idx, w, nnz = oracle.topk(G.astype(np.float32), k)
    res = rng.standard_normal((2, res_len)).astype(np.float32)
    y = rng.standard_normal((S, L)).astype(np.float32)
    dirs = rng.integers(0, n_dirs, S).astype(np.int32)
    out = oracle.render_sparse(y, dirs, idx, w, nnz, refl_len, res)
    # Eq. 1-2: the cascade equals convolution with the dense HRIR f * g, summed over sources
    ref = np.zeros((2, L + refl_len + res_len - 2))
    for s in range(S):
        for e in range(2):
            g = np.zeros(refl_len)
            n = int(nnz[dirs[s], e])
            g[idx[dirs[s], e, :n].astype(int)] = w[dirs[s], e, :n]
            h = np.convolve(res[e].astype(np.float64), g)
            ref[e] += np.convolve(y[s].astype(np.float64), h)
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-10)
    # linear in the sources
    parts = sum(oracle.render_sparse(y[s:s + 1], dirs[s:s + 1], idx, w, nnz, refl_len, res)
                for s in range(S))
    np.testing.assert_allclose(out, parts, rtol=1e-10, atol=1e-10)


# ---- filter production (Sec. III) ----------------------------------------------------------
from oracle import factorize as fz  # noqa: E402


@settings(max_examples=40, deadline=None, derandomize=True)
@given(st.integers(0, 2 ** 31 - 1), st.integers(3, 12), st.integers(2, 8), st.integers(1, 6))
def test_reflection_update_keeps_sign_and_never_increases_the_residual(seed, N, Lg, Lf):
    rng = np.random.default_rng(seed)
    M = Lf + Lg - 1
    X = rng.standard_normal((M, N))
    f = rng.standard_normal(Lf)
    F = fz.toeplitz_filter_matrix(f, Lg)
    G = rng.random((N, Lg)) * (rng.random((N, Lg)) < 0.8)
    r0 = float(np.sum((X - F @ G.T) ** 2))
    for _ in range(5):
        G1 = fz.update_reflections(X, F, G)
        assert np.all(G1 >= 0) and np.all(G1[G == 0] == 0)       # zeros stay zero (Eq. 4)
        r1 = float(np.sum((X - F @ G1.T) ** 2))
        assert r1 <= r0 * (1 + 1e-12) + 1e-12
        G, r0 = G1, r1


@settings(max_examples=40, deadline=None, derandomize=True)
@given(st.integers(0, 2 ** 31 - 1), st.integers(2, 8), st.integers(1, 5),
       st.floats(0.0, 2.0, allow_nan=False))
def test_l1_nnls_is_the_constrained_minimiser(seed, Lg, Lf, lam):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(Lf)
    f[0] = 1.0 + abs(f[0])                                       # full column rank
    F = fz.toeplitz_filter_matrix(f, Lg)
    x = rng.standard_normal(F.shape[0])
    g = fz.l1_nnls(F, x, lam)
    assert np.all(g >= 0)
    assert fz.kkt_violation(F, x, g, lam) <= 1e-8 * max(1.0, np.abs(F.T @ x).max())
    obj = lambda v: float(np.sum((F @ v - x) ** 2) + lam * np.sum(v))  # noqa: E731
    for _ in range(20):                                          # no feasible point is better
        v = np.maximum(0.0, g + 0.1 * rng.standard_normal(Lg))
        assert obj(g) <= obj(v) + 1e-10


@settings(max_examples=40, deadline=None, derandomize=True)
@given(st.integers(0, 2 ** 31 - 1), st.integers(2, 10), st.integers(1, 6), st.integers(1, 5))
def test_resonance_solve_zeroes_the_gradient(seed, N, Lg, Lf):
    rng = np.random.default_rng(seed)
    M = Lf + Lg - 1
    X = rng.standard_normal((M, N))
    G = rng.random((N, Lg)) + 0.1
    f = fz.solve_resonance(X, G, Lf)
    # d/df sum_i ||X_i - C(g_i) f||^2 = -2 sum_i C(g_i)^T (X_i - C(g_i) f) = 0
    grad = np.zeros(Lf)
    for i in range(N):
        C = fz.conv_matrix(G[i], Lf)
        grad += C.T @ (X[:, i] - C @ f)
    assert np.abs(grad).max() <= 1e-9 * max(1.0, np.abs(X).max() * N)


@settings(max_examples=25, deadline=None, derandomize=True)
@given(st.integers(0, 2 ** 31 - 1), st.integers(1, 3), st.integers(1, 400), st.sampled_from([8, 32, 100]))
def test_moving_render_is_the_segment_crossfade(seed, S, L, seg_len):
    # brute force with dense filters and numpy.convolve: in segment j >= 1 the reflection output
    # moves linearly from the previous segment's filter to the current one, a = (n - j seg + 1) / seg
    rng = np.random.default_rng(seed)
    refl_len, res_len, k = 30, 5, 4
    n_seg = (L + seg_len - 1) // seg_len
    G = rng.random((S, n_seg, 2, refl_len)) * (rng.random((S, n_seg, 2, refl_len)) < 0.4)
    idx, w, nnz = oracle.topk(G.astype(np.float32), k)
    res = rng.standard_normal((2, res_len)).astype(np.float32)
    y = rng.standard_normal((S, L)).astype(np.float32)
    out = oracle.render_moving(y, idx, w, nnz, seg_len, refl_len, res)
    n_z = L + refl_len - 1
    z = np.zeros((2, n_z))
    for s in range(S):
        for e in range(2):
            full = []
            for j in range(n_seg):
                g = np.zeros(refl_len)
                g[idx[s, j, e, :nnz[s, j, e]].astype(int)] = w[s, j, e, :nnz[s, j, e]]
                full.append(np.convolve(y[s].astype(np.float64), g))
            for n in range(n_z):
                j = min(n // seg_len, n_seg - 1)
                if 1 <= n // seg_len < n_seg:
                    a = (n - j * seg_len + 1) / seg_len
                    z[e, n] += (1 - a) * full[j - 1][n] + a * full[j][n]
                else:
                    z[e, n] += full[j][n]
    ref = np.stack([np.convolve(res[e].astype(np.float64), z[e]) for e in range(2)])
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-10)
