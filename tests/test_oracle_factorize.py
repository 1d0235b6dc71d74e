"""Pins for the oracle's filter production (Sec. III) and metrics (Sec. IV-B, IV-G)."""
import itertools
import os

import numpy as np
import pytest
import scipy.optimize

import oracle
from oracle import factorize as fz

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def planted(rng, N=60, Lg=12, Lf=6, density=0.3):
    """X = F~(f*) G*^T exactly, with G* sparse and non-negative."""
    f = rng.standard_normal(Lf)
    f[0] = 1.5
    G = rng.exponential(size=(N, Lg)) * (rng.random((N, Lg)) < density)
    G[:, 0] += 0.5
    X = fz.toeplitz_filter_matrix(f, Lg) @ G.T
    return X, f, G


def test_toeplitz_matrix_is_convolution():
    rng = np.random.default_rng(0)
    f, g = rng.standard_normal(7), rng.standard_normal(11)
    F = fz.toeplitz_filter_matrix(f, 11)
    assert F.shape == (17, 11)
    np.testing.assert_allclose(F @ g, np.convolve(f, g), atol=1e-14)
    np.testing.assert_allclose(fz.conv_matrix(g, 7) @ f, np.convolve(f, g), atol=1e-14)
    # constant along diagonals: F[i, j] depends on i - j only
    for i, j in itertools.product(range(16), range(10)):
        assert F[i + 1, j + 1] == F[i, j]


def test_resonance_system_equals_bruteforce_normal_equations():
    rng = np.random.default_rng(1)
    N, Lg, Lf = 9, 8, 5
    G = rng.random((N, Lg))
    X = rng.standard_normal((Lf + Lg - 1, N))
    A, b = fz.resonance_system(X, G, Lf)
    A_bf = sum(fz.conv_matrix(G[i], Lf).T @ fz.conv_matrix(G[i], Lf) for i in range(N))
    b_bf = sum(fz.conv_matrix(G[i], Lf).T @ X[:, i] for i in range(N))
    np.testing.assert_allclose(A, A_bf, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(b, b_bf, rtol=1e-13, atol=1e-13)
    # symmetric Toeplitz (Sec. III-C)
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    for i, j in itertools.product(range(Lf - 1), range(Lf - 1)):
        assert abs(A[i + 1, j + 1] - A[i, j]) < 1e-12


def test_resonance_solve_is_least_squares_optimum():
    rng = np.random.default_rng(2)
    N, Lg, Lf = 20, 10, 6
    G = rng.random((N, Lg))
    X = rng.standard_normal((Lf + Lg - 1, N))
    f = fz.solve_resonance(X, G, Lf)
    # library least squares on the stacked convolution system
    C = np.vstack([fz.conv_matrix(G[i], Lf) for i in range(N)])
    f_ls = np.linalg.lstsq(C, X.T.reshape(-1), rcond=None)[0]
    np.testing.assert_allclose(f, f_ls, rtol=1e-10, atol=1e-12)
    r0 = fz.residual(X, f, G)
    for l in range(Lf):
        for eps in (1e-4, -1e-4):
            fp = f.copy()
            fp[l] += eps
            assert fz.residual(X, fp, G) >= r0


def test_resonance_solve_reduces_to_semi_nmf_f_update_when_lg_is_1():
    """With Lg = 1 the Toeplitz F~ is the single column f and the solve must equal the
    unconstrained semi-NMF update F = X G (G^T G)^-1 of Eq. 4."""
    rng = np.random.default_rng(3)
    N, M = 15, 9
    G = rng.random((N, 1))
    X = rng.standard_normal((M, N))
    f = fz.solve_resonance(X, G, M)
    F_semi = X @ G @ np.linalg.inv(G.T @ G)
    np.testing.assert_allclose(f, F_semi[:, 0], rtol=1e-12)


def test_resonance_solve_lf_is_1_closed_form():
    """Lf = 1: F~ = f0 I, the optimum is f0 = tr(X G) / tr(G^T G)."""
    rng = np.random.default_rng(4)
    N, M = 11, 7
    G = rng.random((N, M))
    X = rng.standard_normal((M, N))
    f = fz.solve_resonance(X, G, 1)
    assert f.shape == (1,)
    assert abs(f[0] - np.trace(X @ G) / np.trace(G.T @ G)) < 1e-13


def test_reflection_update_nonnegative_monotone_and_fixed_point():
    rng = np.random.default_rng(5)
    X, f_true, G_true = planted(rng)
    Lg = G_true.shape[1]
    F = fz.toeplitz_filter_matrix(f_true, Lg)
    # exact non-negative solution is a fixed point (numerator = denominator)
    G_fix = fz.update_reflections(X, F, G_true)
    np.testing.assert_allclose(G_fix, G_true, rtol=1e-10, atol=1e-12)
    # from a random start with F fixed: G stays >= 0, zeros stay zero, residual never rises
    G = rng.random(G_true.shape)
    G[0, 3] = 0.0
    prev = fz.residual(X, f_true, G)
    for _ in range(30):
        G = fz.update_reflections(X, F, G)
        assert np.all(G >= 0) and G[0, 3] == 0.0
        cur = fz.residual(X, f_true, G)
        assert cur <= prev * (1 + 1e-12) + 1e-300
        prev = cur


def test_factorize_residual_nonincreasing_and_fits_planted_model():
    rng = np.random.default_rng(6)
    X, f_true, G_true = planted(rng, N=80, Lg=12, Lf=6)
    G0 = rng.random(G_true.shape)
    f, G, trace = fz.factorize(X, 12, G0, iters=300)
    assert np.all(np.diff(trace) <= 1e-12 * trace[:-1] + 1e-300)
    assert trace[-1] < 1e-3 * trace[0]
    assert np.all(G >= 0)
    assert abs(np.linalg.norm(f) - 1.0) < 1e-12
    # rescaling leaves the product unchanged
    assert abs(fz.residual(X, f, G) - trace[-1]) <= 1e-9 * max(trace[-1], 1e-300) + 1e-12


def test_factorize_paper_lengths_run():
    """The paper's own split (M = 200, Lg = 25, f of length 176; Sec. IV-C) on a small
    synthetic set: runs, stays non-negative, residual non-increasing."""
    rng = np.random.default_rng(7)
    M, Lg, N = 200, 25, 40
    f = np.exp(-np.arange(M - Lg + 1) / 20.0) * rng.standard_normal(M - Lg + 1)
    Gs = rng.exponential(size=(N, Lg)) * (rng.random((N, Lg)) < 0.3)
    X = fz.toeplitz_filter_matrix(f, Lg) @ Gs.T + 1e-3 * rng.standard_normal((M, N))
    f_hat, G_hat, trace = fz.factorize(X, Lg, rng.random((N, Lg)), iters=10)
    assert f_hat.shape == (176,) and G_hat.shape == (N, Lg)
    assert np.all(G_hat >= 0)
    assert np.all(np.diff(trace) <= 1e-12 * trace[:-1])


# --------------------------------------------------------------------------- L1-NNLS
def _qp_problem(rng, M=12, n=5):
    F = rng.standard_normal((M, n))
    x = rng.standard_normal(M)
    return F, x


def test_l1_nnls_lambda0_equals_lawson_hanson_library():
    rng = np.random.default_rng(8)
    for _ in range(20):
        F, x = _qp_problem(rng, 15, 7)
        g = fz.l1_nnls(F, x, 0.0)
        g_ref, _ = scipy.optimize.nnls(F, x)
        np.testing.assert_allclose(g, g_ref, atol=1e-10)


def test_l1_nnls_equals_support_enumeration_on_tiny_problems():
    rng = np.random.default_rng(9)
    for lam in (0.0, 0.05, 0.5):
        for _ in range(10):
            F, x = _qp_problem(rng, 8, 4)
            best, best_obj = None, np.inf
            for r in range(5):
                for supp in itertools.combinations(range(4), r):
                    g = np.zeros(4)
                    if supp:
                        s = list(supp)
                        Q = F[:, s].T @ F[:, s]
                        c = F[:, s].T @ x - lam / 2
                        gs = np.linalg.solve(Q, c)
                        if np.any(gs < 0):
                            continue
                        g[s] = gs
                    obj = np.sum((F @ g - x) ** 2) + lam * np.sum(g)
                    if obj < best_obj:
                        best, best_obj = g, obj
            g = fz.l1_nnls(F, x, lam)
            np.testing.assert_allclose(g, best, atol=1e-10)


def test_l1_nnls_kkt_and_special_cases():
    rng = np.random.default_rng(10)
    f = rng.standard_normal(8)
    f[0] = 1.0
    F = fz.toeplitz_filter_matrix(f, 20)
    x = rng.standard_normal(27)
    for lam in (0.0, 1e-3, 0.1, 1.0):
        g = fz.l1_nnls(F, x, lam)
        assert np.all(g >= 0)
        assert fz.kkt_violation(F, x, g, lam) < 1e-9
    # large lambda switches every tap off: lam >= 2 max(F^T x)
    lam_big = 2.0 * np.max(F.T @ x) + 1e-9
    assert not np.any(fz.l1_nnls(F, x, lam_big))
    # when the unconstrained LS solution is positive it is the answer at lambda = 0
    g_true = rng.random(20) + 0.1
    x2 = F @ g_true
    np.testing.assert_allclose(fz.l1_nnls(F, x2, 0.0), g_true, atol=1e-9)
    # sparsity grows with lambda (NNZE non-increasing on this problem family)
    nz = [np.count_nonzero(fz.l1_nnls(F, x, lam)) for lam in (0.0, 0.3, 3.0, 30.0)]
    assert nz[0] >= nz[-1] and nz[-1] == 0


def test_window_transform_limits():
    D = fz.window_transform(5, 2.0)
    np.testing.assert_allclose(np.diag(D), np.exp(-np.arange(5) ** 2 / 4.0))
    # sigma -> infinity gives the identity transform D_I (Sec. IV-E)
    rng = np.random.default_rng(11)
    F, x = _qp_problem(rng, 10, 4)
    F = np.abs(F)
    g_id = fz.l1_nnls(F, x, 0.01)
    g_w = fz.l1_nnls(F, x, 0.01, D=fz.window_transform(10, 1e9))
    np.testing.assert_allclose(g_w, g_id, atol=1e-9)
    g_w30 = fz.l1_nnls(F, x, 0.01, D=fz.window_transform(10, 3.0))
    assert fz.kkt_violation(F, x, g_w30, 0.01, D=fz.window_transform(10, 3.0)) < 1e-9


def test_sparsify_discards_small_taps():
    rng = np.random.default_rng(12)
    X, f_true, G_true = planted(rng, N=10, Lg=12, Lf=6)
    G = fz.sparsify(X, f_true, 12, lam=0.0)
    np.testing.assert_allclose(G, fz.discard_small(G_true), atol=1e-8)
    Gs = fz.sparsify(X, f_true, 12, lam=1.0)
    assert fz.nnze(Gs) <= fz.nnze(G)
    assert np.all((Gs == 0) | (Gs > 1e-4))


# ---------------------------------------------------------------------------- metrics
def test_metrics_closed_forms():
    rng = np.random.default_rng(13)
    x = rng.standard_normal(64)
    assert fz.spectral_distortion(x, x) == 0.0
    # a uniform gain of 2 is a flat 20 log10(1/2) dB error at every bin
    assert abs(fz.spectral_distortion(x, 2 * x) - 20 * np.log10(2.0)) < 1e-12
    X, f, G = planted(rng, N=5, Lg=4, Lf=3)
    assert fz.rmse(X, f, G) < 1e-14
    Xp = X + 0.5
    assert abs(fz.rmse(Xp, f, G) - 0.5) < 1e-14
    assert fz.nnze(np.array([[0, 1, 2], [0, 0, 3.0]])) == 1.5


def test_cost_model_against_paper_printed_crossovers():
    """Sec. IV-G prints crossovers of 127 taps (|y| = 44100) and 90 taps (|y| = 2205).
    Evaluating the printed formula gives about 124.5 and 95.6; the paper's figures are
    approximate, so the pin is a 7% band around the printed values."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "cost_model_sec4g.txt"))
            if l.strip() and not l.startswith("#")]
    for len_y, printed in rows:
        x = fz.crossover(float(len_y))
        assert abs(x - float(printed)) / float(printed) < 0.07
        assert abs(fz.fft_cost(float(len_y), x) - x) < 1e-6
    # hand evaluation: |y| = 1024, |x| = 1 -> 68/9 * (1024*10 + 1024) / 1024 = 68/9 * 11
    assert abs(fz.fft_cost(1024.0, 1.0) - 68.0 / 9.0 * 11.0) < 1e-12
