"""Filter production: Toeplitz-constrained semi-NMF, L1-NNLS sparsification, metrics.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Plain FP64 numpy restatement of Sec. III
and Sec. IV-B of Luo, Zotkin & Duraiswami, "Sparse Head-Related Impulse Response for
Efficient Direct Convolution".  Library primitives used as steps: matrix products,
Cholesky (scipy.linalg.cho_factor/cho_solve), dense solves and numpy's FFT (only for the
spectral-distortion metric).  Nothing here is shared with, or called by, the CUDA path.

Notation (the paper's, Sec. II-III; sizes of the filter split follow the paper's Eq. 1):
  X       M x N HRIR matrix, column i is the HRIR of direction i      (Sec. II, a)
  f       resonance filter, length Lf = M - Lg + 1                    (Eq. 13)
  G       N x Lg non-negative reflection matrix, row i = g_i          (Sec. II, d)
  F~      M x Lg banded Toeplitz of f, F~[m, j] = f[m - j]            (Eq. 12)
so that column i of F~ G^T is the convolution f * g_i.

Readings taken where the paper is silent or inconsistent (each also listed in the design
notes of the repository):
  * Eq. 9-11 index ranges carry inconsistent signs; the f-solve is written as the normal
    equations of min_f sum_i ||X_i - F~ g_i||^2, which is sign-convention free.
  * b has Lf entries (the garbled "M x 1" of Eq. 10 cannot match |Theta| unknowns).
  * Algorithm 1's rand(N, K) initialisation is passed in as an input (G0 >= 0).
  * In the multiplicative update (Eq. 4) entries with G_ij = 0 stay 0; for G_ij > 0 the
    denominator is >= G_ij ||f||^2 > 0, so no epsilon is needed.
  * After the last iteration, f is rescaled to unit L2 norm and G by the inverse factor
    (F~ G^T is unchanged).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------------------
# Toeplitz structure (Eqs. 5, 6, 12)
# ---------------------------------------------------------------------------------------


def toeplitz_filter_matrix(f, refl_len: int) -> np.ndarray:
    """Banded Toeplitz matrix of Eq. 12: M x Lg, column j is f shifted down by j."""
    f = np.asarray(f, dtype=np.float64)
    Lf = f.size
    M = Lf + refl_len - 1
    F = np.zeros((M, refl_len))
    for j in range(refl_len):
        F[j:j + Lf, j] = f
    return F


def conv_matrix(g, res_len: int) -> np.ndarray:
    """C(g): M x Lf matrix with C(g) f = f * g (used only to cross-check A and b)."""
    g = np.asarray(g, dtype=np.float64)
    M = g.size + res_len - 1
    C = np.zeros((M, res_len))
    for l in range(res_len):
        C[l:l + g.size, l] = g
    return C


# ---------------------------------------------------------------------------------------
# resonance solve (Eqs. 9-11 restricted to the non-zero parameters of Eqs. 12-13)
# ---------------------------------------------------------------------------------------


def resonance_system(X, G, res_len: int):
    """A f = b, the zero-gradient condition of ||X - F~ G^T||_F^2 w.r.t. f (Eq. 9, 10).

    A[l, l'] = tr(G^T G  Sbar^{l-l'}): the sum along the (l-l')-th diagonal of G^T G;
    b[l]     = tr(S^{l T} X G):        the sum along the l-th sub-diagonal of X G.
    A is symmetric Toeplitz (Sec. III-C)."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    GtG = G.T @ G
    XG = X @ G
    A = np.empty((res_len, res_len))
    for l in range(res_len):
        for lp in range(res_len):
            A[l, lp] = np.trace(GtG, offset=l - lp)
    b = np.array([np.trace(XG, offset=-l) for l in range(res_len)])
    return A, b


def solve_resonance(X, G, res_len: int) -> np.ndarray:
    """Theta = A^{-1} b (Eq. 11) by Cholesky; returns f = {Theta_0 .. Theta_{K-M}} (Eq. 13)."""
    A, b = resonance_system(X, G, res_len)
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, b)


# ---------------------------------------------------------------------------------------
# reflection update (Eq. 4, the semi-NMF multiplicative rule with F = F~)
# ---------------------------------------------------------------------------------------


def _pos(Q):
    return (np.abs(Q) + Q) / 2.0


def _neg(Q):
    return (np.abs(Q) - Q) / 2.0


def update_reflections(X, F, G) -> np.ndarray:
    """G_ij <- G_ij sqrt( ((X^T F)^+ + [G (F^T F)^-])_ij / ((X^T F)^- + [G (F^T F)^+])_ij )."""
    X = np.asarray(X, dtype=np.float64)
    XtF = X.T @ F
    FtF = F.T @ F
    num = _pos(XtF) + G @ _neg(FtF)
    den = _neg(XtF) + G @ _pos(FtF)
    out = np.zeros_like(G)
    live = G > 0
    out[live] = G[live] * np.sqrt(num[live] / den[live])
    return out


def residual(X, f, G) -> float:
    """||X - F~ G^T||_F^2 (Eq. 3 with F = F~)."""
    F = toeplitz_filter_matrix(f, G.shape[1])
    R = np.asarray(X, dtype=np.float64) - F @ G.T
    return float(np.sum(R * R))


def factorize(X, refl_len: int, G0, iters: int = 50, normalise: bool = True):
    """The alternating minimisation of Algorithm 1 (without its final sparsifying fine-tune):
    T rounds of a resonance solve with G fixed followed by a reflection update with f fixed.

    X: M x N HRIRs (columns).  G0: N x Lg non-negative initialisation.
    Returns (f, G, trace) where trace[t] = residual after iteration t (trace[0] is the
    residual of the first f-solve paired with G0)."""
    X = np.asarray(X, dtype=np.float64)
    M, N = X.shape
    res_len = M - refl_len + 1
    if res_len < 1:
        raise ValueError("refl_len must be <= M")
    G = np.array(G0, dtype=np.float64)
    if G.shape != (N, refl_len) or np.any(G < 0):
        raise ValueError("G0 must be a non-negative N x Lg matrix")
    trace = []
    f = None
    for t in range(iters):
        # the least-squares resonance for the current G: normal equations of Eq. 9-10,
        # solved as in Eq. 11 over the Lf free parameters of the banded form (Eq. 13)
        f = solve_resonance(X, G, res_len)
        # its banded Toeplitz matrix (Eq. 12), the F of the semi-NMF objective (Eq. 3)
        F = toeplitz_filter_matrix(f, refl_len)
        if t == 0:
            trace.append(residual(X, f, G))
        # non-negative reflections for that F: the sign-split ratio rule of Eq. 4
        G = update_reflections(X, F, G)
        trace.append(residual(X, f, G))
    if normalise and f is not None:
        s = float(np.linalg.norm(f))
        if s > 0:
            f = f / s
            G = G * s
    return f, G, np.array(trace)


# ---------------------------------------------------------------------------------------
# sparsification: L1-NNLS (Eq. 14) with D_I (identity) or D_W (window, Eq. 16)
# ---------------------------------------------------------------------------------------


def window_transform(M: int, sigma: float) -> np.ndarray:
    """D_W = diag(v_sigma(0..M-1)), v_sigma(x) = exp(-x^2 / sigma^2)  (Eq. 16)."""
    x = np.arange(M, dtype=np.float64)
    return np.diag(np.exp(-(x * x) / (sigma * sigma)))


def l1_nnls(F, x, lam: float, D=None, tol: float = 1e-12, max_iter: int = 10000) -> np.ndarray:
    """min_g ||D (F g - x)||^2 + lam * sum(g)  s.t. g >= 0   (Eq. 14; |g|_1 = sum g on g >= 0).

    Written as the quadratic program  g^T Q g - 2 c^T g  with Q = F^T D^T D F and
    c = F^T D^T D x - lam/2, solved by an active-set method (Lawson & Hanson's NNLS scheme
    applied to the normal-equation form).  Q is positive definite when F~ has full column
    rank (f_0 != 0), so the minimiser is unique and is characterised by the KKT
    conditions checked in the tests."""
    F = np.asarray(F, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if D is not None:
        F = D @ F
        x = D @ x
    Q = F.T @ F
    c = F.T @ x - lam / 2.0
    n = Q.shape[0]
    g = np.zeros(n)
    P = np.zeros(n, dtype=bool)
    scale = max(1.0, float(np.max(np.abs(c))) if c.size else 1.0)
    for _ in range(max_iter):
        w = c - Q @ g                      # minus half the gradient
        cand = np.where(~P, w, -np.inf)
        j = int(np.argmax(cand)) if n else 0
        if n == 0 or cand[j] <= tol * scale:
            break
        P[j] = True
        while True:
            idx = np.flatnonzero(P)
            s = np.zeros(n)
            s[idx] = np.linalg.solve(Q[np.ix_(idx, idx)], c[idx])
            if np.all(s[idx] > 0):
                g = s
                break
            bad = idx[s[idx] <= 0]
            alpha = np.min(g[bad] / (g[bad] - s[bad]))
            g = g + alpha * (s - g)
            drop = P & (g <= 1e-300)
            g[drop] = 0.0
            P &= ~drop
            if not P.any():
                break
    return g


def kkt_violation(F, x, g, lam: float, D=None) -> float:
    """Largest violation of the KKT conditions of Eq. 14 at g (0 at the exact minimiser):
    gradient zero on the support, gradient >= 0 off it, g >= 0."""
    F = np.asarray(F, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if D is not None:
        F = D @ F
        x = D @ x
    grad = 2.0 * (F.T @ (F @ g - x)) + lam
    on = g > 0
    v = 0.0
    if on.any():
        v = max(v, float(np.max(np.abs(grad[on]))))
    if (~on).any():
        v = max(v, float(np.max(np.maximum(0.0, -grad[~on]))))
    v = max(v, float(np.max(np.maximum(0.0, -g))) if g.size else 0.0)
    return v


def discard_small(G, thresh: float = 1e-4) -> np.ndarray:
    """Drop entries whose magnitude is <= 1e-4 (Sec. III-D, after Eq. 16)."""
    G = np.array(G, dtype=np.float64)
    G[np.abs(G) <= thresh] = 0.0
    return G


def sparsify(X, f, refl_len: int, lam: float, sigma: float | None = None,
             thresh: float = 1e-4) -> np.ndarray:
    """Fine-tune step of Algorithm 1: per direction, L1-NNLS with F~ fixed (Eq. 14) using
    D_I (sigma None) or D_W (Eq. 16), then the small-tap discard.  Returns N x Lg."""
    X = np.asarray(X, dtype=np.float64)
    F = toeplitz_filter_matrix(f, refl_len)
    D = None if sigma is None else window_transform(F.shape[0], sigma)
    G = np.stack([l1_nnls(F, X[:, i], lam, D) for i in range(X.shape[1])])
    return discard_small(G, thresh)


# ---------------------------------------------------------------------------------------
# metrics (Eq. 17) and the cost model of Sec. IV-G
# ---------------------------------------------------------------------------------------


def rmse(X, f, G) -> float:
    """sqrt(||X - F~ G^T||_F^2 / (M N))."""
    M, N = np.asarray(X).shape
    return float(np.sqrt(residual(X, f, G) / (M * N)))


def spectral_distortion(x, x_hat, floor: float = 1e-300) -> float:
    """SD = sqrt( (1/M) sum_{i=1..M} (20 log10 |H_i| / |H~_i|)^2 ), H = M-point DFT."""
    x = np.asarray(x, dtype=np.float64)
    x_hat = np.asarray(x_hat, dtype=np.float64)
    H = np.maximum(np.abs(np.fft.fft(x)), floor)
    Ht = np.maximum(np.abs(np.fft.fft(x_hat)), floor)
    d = 20.0 * np.log10(H / Ht)
    return float(np.sqrt(np.mean(d * d)))


def nnze(G) -> float:
    """Mean number of non-zero entries per reflection filter (row of G)."""
    return float(np.mean(np.count_nonzero(np.asarray(G), axis=-1)))


def direct_cost(nnz_x: float) -> float:
    """Sec. IV-G: real flops per output sample of direct convolution = NNZE of the filter."""
    return float(nnz_x)


def fft_cost(len_y: float, len_x: float) -> float:
    """Sec. IV-G: complex flops per output sample of split-radix FFT convolution,
    (68/9)(|y| log2 |y| + |y|) / (|y| - |x| + 1)."""
    return (68.0 / 9.0) * (len_y * np.log2(len_y) + len_y) / (len_y - len_x + 1.0)


def crossover(len_y: float) -> float:
    """Filter length at which the two per-sample costs of Sec. IV-G are equal."""
    lo, hi = 1.0, float(len_y)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if direct_cost(mid) < fft_cost(len_y, mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
