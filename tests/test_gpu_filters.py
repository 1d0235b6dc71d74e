"""GPU parity of the filter production (Sec. III) against the FP64 oracle: the alternating
minimisation of Algorithm 1 (hrir_factorize), its L1-NNLS fine-tune (Eq. 14 with D_I or D_W,
hrir_sparsify), and the renderer on the variable-NNZE tap tables they produce."""
import numpy as np
import pytest

import oracle
from oracle import factorize as fz
from paper_1502_03162_gb300 import synth
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LG = 200


@pytest.fixture(scope="module")
def rend():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    yield r
    r.close()


@pytest.fixture(scope="module")
def hset():
    """Synthetic HRIR set 4 (1250 directions x 2 ears x 231 taps), as FP32 (what the device
    reads; the oracle gets the same values in FP64)."""
    X, az, el, p = synth.hrir_set(4)
    return np.ascontiguousarray(X, np.float32), az, el, p


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_one_round_matches_oracle(rend, hset):
    """From the same starting G: the resonance solve (Eqs. 9-11), the update of G (Eq. 4) and
    both residuals of the first round (Algorithm 1).  The products are FP32-accurate (sums of
    up to 1250 terms accumulated in FP32), the Toeplitz sums, the solve and the residuals
    FP64: f, G and the trace agree with the FP64 oracle to a few 1e-7 relative."""
    from paper_1502_03162_gb300 import hrir
    X, _, _, _ = hset
    N = X.shape[0]
    rng = np.random.default_rng(5)
    G0 = rng.random((N, 2, LG), dtype=np.float32)
    G0[rng.random(G0.shape) < 0.3] = 0.0          # zeros stay zero
    Gd = _cuda(G0)
    f, tr = hrir.hrir_factorize(rend.ctx, _cuda(X), Gd, LG, iters=1, normalise=False)
    assert rend.sync() == 0
    f, tr, G1 = f.cpu().numpy(), tr.cpu().numpy(), Gd.cpu().numpy()
    for e in range(2):
        Xe = X[:, e, :].T.astype(np.float64)
        Ge = G0[:, e, :].astype(np.float64)
        f0 = fz.solve_resonance(Xe, Ge, 32)
        ref = fz.update_reflections(Xe, fz.toeplitz_filter_matrix(f0, LG), Ge)
        df_ = np.abs(f[e] - f0).max() / np.abs(f0).max()
        dG = np.abs(G1[:, e] - ref).max() / ref.max()
        r0, r1 = fz.residual(Xe, f0, Ge), fz.residual(Xe, f0, ref)
        dtr = np.abs(tr[e] / [r0, r1] - 1).max()
        print(f"FACTORIZE one round ear {e}: f {df_:.2e}, G {dG:.2e}, trace {dtr:.2e}")
        assert np.all(G1[:, e][Ge == 0] == 0)
        assert df_ <= 1e-5 and dG <= 1e-5 and dtr <= 1e-5


def test_fifty_rounds_track_the_oracle(rend, hset):
    """Algorithm 1 with the paper's 50 rounds from the same random start: the residual trace
    does not increase (the exact resonance solve and Eq. 4 never increase it), follows the
    FP64 trace, and the normalised resonance and the reconstruction f * g agree."""
    from paper_1502_03162_gb300 import hrir
    X, _, _, _ = hset
    N = X.shape[0]
    rng = np.random.default_rng(6)
    G0 = rng.random((N, 2, LG), dtype=np.float32)
    Gd = _cuda(G0)
    f, tr = hrir.hrir_factorize(rend.ctx, _cuda(X), Gd, LG, iters=50, normalise=True)
    assert rend.sync() == 0
    f, tr, G = f.cpu().numpy(), tr.cpu().numpy(), Gd.cpu().numpy()
    for e in range(2):
        Xe = X[:, e, :].T.astype(np.float64)
        fo, Go, tro = fz.factorize(Xe, LG, G0[:, e, :].astype(np.float64), iters=50)
        dtr = np.abs(tr[e] / tro - 1).max()
        df_ = np.abs(f[e] - fo).max() / np.abs(fo).max()
        rec = np.stack([np.convolve(f[e].astype(np.float64), g) for g in G[:, e].astype(np.float64)])
        reco = (fz.toeplitz_filter_matrix(fo, LG) @ Go.T).T
        drec = np.abs(rec - reco).max() / np.abs(reco).max()
        print(f"FACTORIZE 50 rounds ear {e}: trace {dtr:.2e}, f {df_:.2e}, f*g {drec:.2e}, "
              f"residual {tro[0]:.4e} -> {tro[-1]:.4e}")
        assert np.all(np.diff(tr[e]) <= 1e-5 * tr[e][0]), "GPU residual trace increased"
        assert dtr <= 1e-4 and df_ <= 1e-4 and drec <= 1e-4
        assert abs(np.linalg.norm(f[e].astype(np.float64)) - 1.0) < 1e-5


@pytest.mark.parametrize("lam,sigma", [(0.0, 0.0), (1e-3, 0.0), (1e-3, 60.0), (1e-2, 0.0)])
def test_sparsify_matches_oracle(rend, hset, lam, sigma):
    """Eq. 14 with D_I (sigma 0) or D_W (Eq. 16), f fixed, on 100 directions x 2 ears: the
    GPU's undiscarded solution satisfies the KKT conditions (checked in FP64), and after the
    1e-4 discard it equals the oracle's active-set solution to FP32 accuracy."""
    from paper_1502_03162_gb300 import hrir
    X, _, _, p = hset
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(X.shape[0], 100, replace=False))
    Xs = np.ascontiguousarray(X[sel])
    f = (p["res"] / np.linalg.norm(p["res"], axis=1, keepdims=True)).astype(np.float32)
    Xd, fd = _cuda(Xs), _cuda(f)
    g_raw, _ = hrir.hrir_sparsify(rend.ctx, Xd, fd, LG, lam, sigma, thresh=0.0)
    g_cut, nnz = hrir.hrir_sparsify(rend.ctx, Xd, fd, LG, lam, sigma, thresh=1e-4)
    assert rend.sync() == 0
    g_raw, g_cut, nnz = g_raw.cpu().numpy(), g_cut.cpu().numpy(), nnz.cpu().numpy()
    assert np.all(g_raw >= 0) and np.array_equal(nnz, np.count_nonzero(g_cut, axis=2))
    worst_kkt, worst = 0.0, 0.0
    for e in range(2):
        F = fz.toeplitz_filter_matrix(f[e].astype(np.float64), LG)
        D = None if sigma <= 0 else fz.window_transform(F.shape[0], sigma)
        Xe = Xs[:, e, :].T.astype(np.float64)
        ref = fz.sparsify(Xe, f[e].astype(np.float64), LG, lam, sigma if sigma > 0 else None)
        for i in range(Xs.shape[0]):
            x = Xe[:, i]
            scale = np.abs(F.T @ x).max()
            kkt = fz.kkt_violation(F, x, g_raw[i, e].astype(np.float64), lam, D)
            worst_kkt = max(worst_kkt, kkt / scale)
            a, b = g_cut[i, e].astype(np.float64), ref[i]
            # entries within FP32 noise of the 1e-4 threshold may land on either side
            near = np.abs(np.maximum(a, b) - 1e-4) <= 1e-5 * max(b.max(), 1e-30)
            d = np.abs(a - b)
            d[near & ((a == 0) | (b == 0))] = 0.0
            worst = max(worst, d.max() / max(b.max(), 1e-30))
    print(f"SPARSIFY lam={lam} sigma={sigma}: kkt/scale {worst_kkt:.2e}, max diff/max {worst:.2e}, "
          f"mean NNZE {nnz.mean():.2f}")
    assert worst_kkt <= 1e-5
    assert worst <= 1e-4


def _tables_from(G, k=None):
    """Variable-NNZE tap tables keeping every non-zero of G [n_dirs][2][Lg] (oracle top-K with
    k = the largest row count)."""
    counts = np.count_nonzero(G, axis=2)
    k = int(counts.max()) if k is None else k
    idx, w, nnz = oracle.topk(np.ascontiguousarray(G, np.float32), k)
    assert np.array_equal(nnz, counts)
    return idx, w, nnz


@pytest.mark.parametrize("lam", [1e-3, 0.0])
def test_render_variable_nnze_tables_from_oracle_sparsify(rend, hset, lam):
    """Tables of variable NNZE per (direction, ear) from the oracle's L1-NNLS (Eq. 14, the
    paper's lambda = 1e-3, and lambda = 0) through hrir_load_filters: the three render paths
    against the oracle's mix."""
    X, _, _, p = hset
    rng = np.random.default_rng(8)
    sel = np.sort(rng.choice(X.shape[0], 60, replace=False))
    f = (p["res"] / np.linalg.norm(p["res"], axis=1, keepdims=True)).astype(np.float32)
    G = np.stack([fz.sparsify(X[sel, e, :].T.astype(np.float64), f[e].astype(np.float64), LG, lam)
                  for e in range(2)], axis=1)
    idx, w, nnz = _tables_from(G)
    assert nnz.min() < nnz.max()                     # the NNZE does vary
    S, L = 90, 30011
    y = np.zeros((S, 30016), np.float32)               # rows padded to 16 bytes
    y[:, :L] = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, sel.size)
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, LG, f, length=L)
    rend.load_filters(idx, w, nnz, LG, f)
    for m in ("sparse", "dense", "fft"):
        o = rend.render(_cuda(y), _cuda(dirs), mode=m, length=L).cpu().numpy()
        assert rend.sync() == 0
        assert_close(o, ref, what=f"variable NNZE (lam {lam}) {m}")


def test_fine_tune_on_the_device_feeds_the_renderer(rend, hset):
    """HRIRs factorized by Algorithm 1 (the oracle's 50 rounds, per ear) -> the L1-NNLS
    fine-tune at the paper's lambda = 1e-3 on the device for all 1250 directions -> tap tables
    on the device (top-K keeping every non-zero) -> render.  The device's fine-tune matches the
    oracle's on sampled directions, and the render matches the oracle's mix on those tables."""
    from paper_1502_03162_gb300 import hrir
    X, _, _, _ = hset
    N = X.shape[0]
    rng = np.random.default_rng(9)
    f = np.stack([fz.factorize(X[:, e, :].T.astype(np.float64), LG, rng.random((N, LG)), iters=50)[0]
                  for e in range(2)]).astype(np.float32)
    Gs, nnz = hrir.hrir_sparsify(rend.ctx, _cuda(X), _cuda(f), LG, 1e-3, 0.0, 1e-4)
    k = int(nnz.max().item())
    idx_d, w_d, nnz_d = rend.topk_pack(Gs, k)
    assert rend.sync() == 0
    idx = (idx_d.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
    w, nn = w_d.cpu().numpy(), nnz_d.cpu().numpy()
    assert np.array_equal(nn, nnz.cpu().numpy())
    sel = rng.choice(N, 40, replace=False)
    G_dev = Gs.cpu().numpy()
    for e in range(2):
        ref = fz.sparsify(X[sel, e, :].T.astype(np.float64), f[e].astype(np.float64), LG, 1e-3)
        assert np.abs(G_dev[sel, e].astype(np.float64) - ref).max() <= 1e-4 * ref.max()
    print(f"FILTERS fine-tune of all 1250 x 2 rows: mean NNZE {nn.mean():.2f} (max {k})")
    S, L = 64, 20000
    y = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, N)
    rend.load_filters(idx, w, nn, LG, f)
    o = rend.render(_cuda(y), _cuda(dirs)).cpu().numpy()
    assert rend.sync() == 0
    assert_close(o, oracle.render_sparse(y, dirs, idx, w, nn, LG, f), what="device fine-tuned tables")


def test_device_factorization_feeds_the_fine_tune_and_the_renderer(rend, hset):
    """Filters made entirely on the device: Algorithm 1 (hrir_factorize, 50 rounds) -> the
    L1-NNLS fine-tune at lambda = 1e-3 (hrir_sparsify) -> tap tables (hrir_topk_pack keeping
    every non-zero) -> render, against the oracle's mix on the same tables."""
    from paper_1502_03162_gb300 import hrir
    X, _, _, _ = hset
    N = X.shape[0]
    rng = np.random.default_rng(10)
    Gd = _cuda(rng.random((N, 2, LG), dtype=np.float32))
    Xd = _cuda(X)
    f, _ = hrir.hrir_factorize(rend.ctx, Xd, Gd, LG, iters=50)
    Gs, nnz = hrir.hrir_sparsify(rend.ctx, Xd, f, LG, 1e-3, 0.0, 1e-4)
    k = int(nnz.max().item())
    idx_d, w_d, nnz_d = rend.topk_pack(Gs, k)
    assert rend.sync() == 0
    idx = (idx_d.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
    w, nn, fh = w_d.cpu().numpy(), nnz_d.cpu().numpy(), f.cpu().numpy()
    print(f"FILTERS from the device factorization: mean NNZE {nn.mean():.2f} (max {k})")
    S, L = 64, 20000
    y = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, N)
    rend.load_filters(idx, w, nn, LG, fh)
    o = rend.render(_cuda(y), _cuda(dirs)).cpu().numpy()
    assert rend.sync() == 0
    assert_close(o, oracle.render_sparse(y, dirs, idx, w, nn, LG, fh), what="device-made filters")
