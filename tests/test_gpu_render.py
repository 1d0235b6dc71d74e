"""GPU parity: the CUDA rendering path (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth
from tests.gpu_util import TOL, assert_close, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rend():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    yield r
    r.close()


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ------------------------------------------------------------------------------- top-K pack
def _topk_rows(rng, refl_len):
    """64 x 2 reflection rows with the cases the selection rule has to get right."""
    G = synth.reflection_bank(rng, 64, n_refl=min(60, refl_len), refl_len=refl_len)
    G[0, 0] = 0
    G[1, 1] = -1
    G[2, 0, 5 % refl_len] = np.nan
    G[3, 0] = 0
    G[3, 0, [7 % refl_len, 3 % refl_len, 11 % refl_len, 2 % refl_len]] = 0.5
    G[4, 1, :] = 0.25                                  # all equal: the k smallest indices win
    G[5, 0, :] = np.float32(1e-42)                     # denormals are positive
    G[6, 0, :] = np.float32(np.inf)                    # infinities are the largest values
    G[6, 1, ::3] = np.float32(0.125)                   # ties at the k-th value
    G[7, 0, :] = rng.integers(1, 4, refl_len).astype(np.float32)   # few distinct values
    G[7, 1, : refl_len // 2] = -0.0
    return G


def _check_topk(rend, g, G, k):
    idx, w, nnz = rend.topk_pack(g, k)
    torch.cuda.synchronize()
    ri, rw, rn = oracle.topk(G, k)
    np.testing.assert_array_equal(nnz.cpu().numpy(), rn)
    np.testing.assert_array_equal(idx.cpu().numpy().astype(np.int64) & 0xFFFF, ri.astype(np.int64))
    np.testing.assert_array_equal(w.cpu().numpy().view(np.uint32), rw.view(np.uint32))


@pytest.mark.parametrize("refl_len", [200, 4, 36, 128, 256, 33, 500, 1000, 2048])
def test_topk_pack_bit_exact(rend, refl_len):
    rng = np.random.default_rng(100 + refl_len)
    G = _topk_rows(rng, refl_len)
    g = _dev(G)
    for k in (0, 1, 2, 8, 9, 16, 17, 24, 25, 32, 33, 48, 64, 100, 255):
        _check_topk(rend, g, G, k)


@pytest.mark.parametrize("refl_len", [200, 128])
def test_topk_pack_unaligned_rows_bit_exact(rend, refl_len):
    """The same rows at an address that is not 16-byte aligned."""
    rng = np.random.default_rng(7 + refl_len)
    G = _topk_rows(rng, refl_len)
    buf = torch.zeros(G.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(G.reshape(-1)).cuda()
    g = buf[1:].view(G.shape)
    assert g.data_ptr() % 16 != 0
    for k in (0, 5, 16, 40):
        _check_topk(rend, g, G, k)


@pytest.mark.parametrize("refl_len", [200, 203])         # 16-byte row loads / scalar loads
def test_topk_pack_neighbour_rows_bit_exact(rend, refl_len):
    """Rows like the network's: row r close to row r - 2 (the same ear of the previous
    segment), whose threshold the kernel counts first.  Exact copies, tiny drifts that keep or
    swap the K-th and (K + 1)-th entries, ties planted at the K-th value, all-zero rows and
    fresh rows, over runs long enough that every warp walks many rows."""
    rng = np.random.default_rng(refl_len)
    n_rows = 40000
    G = np.empty((n_rows, refl_len), np.float32)
    G[:2] = rng.random((2, refl_len), dtype=np.float32)
    for r in range(2, n_rows):
        kind = r % 97
        if kind == 0 or not G[r - 2].any():
            G[r] = rng.random(refl_len, dtype=np.float32)                     # fresh row
        elif kind == 13:
            G[r] = 0.0                                                        # nothing selectable
        elif kind % 5 == 0:
            G[r] = G[r - 2]                                                   # exact copy
        else:
            G[r] = G[r - 2] * (1 + 1e-5 * rng.standard_normal(refl_len)).astype(np.float32)
        if kind % 7 == 3:                                                     # a tie at the 16th value
            order = np.argsort(-G[r], kind="stable")
            G[r, order[17]] = G[r, order[15]]
    for k in (1, 8, 16, 32):
        _check_topk(rend, _dev(G), G, k)


@pytest.mark.parametrize("n_rows,refl_len,k", [(40000, 200, 16), (40001, 128, 32), (20000, 1000, 16)])
def test_topk_pack_many_rows_bit_exact(rend, n_rows, refl_len, k):
    """More rows than one resident wave of warps: every warp walks several rows."""
    rng = np.random.default_rng(n_rows + refl_len)
    G = rng.random((n_rows, refl_len), dtype=np.float32)
    G[rng.random((n_rows, refl_len)) < 0.5] = 0.0
    G[::7, :] = np.float32(0.5)                          # ties everywhere in some rows
    _check_topk(rend, _dev(G), G, k)


# ------------------------------------------------------------------------------ rendering
MODES = ("sparse", "dense", "fft")


def _render_both(rend, y, dirs, idx, w, nnz, res, modes=MODES, length=None,
                 dtype=None, refl_len=200):
    rend.load_filters(idx, w, nnz, refl_len, res)
    yd = _dev(y, dtype)
    dd = _dev(dirs.astype(np.int32))
    outs = {}
    for m in modes:
        for full in (True, False):
            o = rend.render(yd, dd, mode=m, full=full, length=length)
            assert rend.sync() == 0
            outs[(m, full)] = o.cpu().numpy()
    return outs


def test_tiny_config_matches_oracle(rend):
    cfg = synth.tiny_config(seed=1)
    idx, w, nnz = oracle.topk(cfg["G"], cfg["k"])
    assert np.all(nnz == 16)
    ref = oracle.render_sparse(cfg["y"], cfg["dirs"], idx, w, nnz, 200, cfg["res"])
    outs = _render_both(rend, cfg["y"], cfg["dirs"], idx, w, nnz, cfg["res"])
    L = cfg["y"].shape[1]
    for m in MODES:
        assert outs[(m, True)].shape == (2, L + 230)
        assert_close(outs[(m, True)], ref, what=f"tiny {m} full")
        assert outs[(m, False)].shape == (2, L)
        assert_close(outs[(m, False)], ref[:, :L], what=f"tiny {m} same")


@pytest.mark.parametrize("S,L,k,n_dirs", [(37, 30001, 16, 50), (5, 9216 * 2 - 199, 8, 7),
                                          (130, 4099, 32, 1250), (3, 200, 16, 3)])
def test_batched_matches_oracle(rend, S, L, k, n_dirs):
    rng = np.random.default_rng(S * 7 + L)
    _, idx, w, nnz, res = tables(rng, n_dirs, k)
    ld = (L + 7) // 8 * 8 + 8
    y = np.full((S, ld), np.nan, dtype=np.float32)       # padding must never be read
    y[:, :L] = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, n_dirs)
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
    outs = _render_both(rend, y, dirs, idx, w, nnz, res, length=L)
    for m in MODES:
        assert np.isfinite(outs[(m, True)]).all()
        assert_close(outs[(m, True)], ref, what=f"{m} S={S} L={L}")
        assert_close(outs[(m, False)], ref[:, :L], what=f"{m} same S={S} L={L}")


@pytest.mark.parametrize("refl_len,k", [(300, 16), (700, 24)])
def test_long_reflection_filters_match_oracle(rend, refl_len, k):
    """Lg longer than one window segment of 204 filter offsets: the sparse kernel walks
    ceil(Lg / 204) segments per unit (a window per segment, taps split by segment)."""
    rng = np.random.default_rng(refl_len + k)
    n_dirs, S, L = 9, 11, 7001
    _, idx, w, nnz, res = tables(rng, n_dirs, k, refl_len=refl_len)
    ld = (L + 7) // 8 * 8 + 8
    y = np.full((S, ld), np.nan, dtype=np.float32)       # padding must never be read
    y[:, :L] = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, n_dirs)
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, refl_len, res, length=L)
    outs = _render_both(rend, y, dirs, idx, w, nnz, res, length=L, refl_len=refl_len)
    H = 32 + refl_len - 1
    for m in MODES:
        assert outs[(m, True)].shape == (2, L + H - 1)
        assert_close(outs[(m, True)], ref, what=f"{m} Lg={refl_len}")
        assert_close(outs[(m, False)], ref[:, :L], what=f"{m} same Lg={refl_len}")


def test_expired_wait_reports_timeout_and_context_stays_usable(rend):
    """The failure path of the bounded device waits: a wait that nothing completes gives up
    after its limit, the next sync reports HRIR_ETIMEDOUT, and the context still renders."""
    from paper_1502_03162_gb300 import hrir
    assert hrir.hrir_selftest_wait_timeout(rend.ctx) == hrir.HRIR_OK
    assert rend.sync() == hrir.HRIR_ETIMEDOUT
    assert rend.sync() == 0                               # the flag was cleared
    cfg = synth.tiny_config(seed=3)
    idx, w, nnz = oracle.topk(cfg["G"], cfg["k"])
    ref = oracle.render_sparse(cfg["y"], cfg["dirs"], idx, w, nnz, 200, cfg["res"])
    outs = _render_both(rend, cfg["y"], cfg["dirs"], idx, w, nnz, cfg["res"], modes=("sparse",))
    assert_close(outs[("sparse", True)], ref, what="render after an expired wait")


def test_edge_cases(rend):
    rng = np.random.default_rng(5)
    _, idx, w, nnz, res = tables(rng, 4, 16)
    nnz = nnz.copy()
    nnz[3] = 0                                           # a direction with no taps
    rend.load_filters(idx, w, nnz, 200, res)
    for L in (1, 3, 7, 199, 200, 201, 9216, 9217):
        y = rng.standard_normal((6, (L + 7) // 8 * 8)).astype(np.float32)
        dirs = np.array([0, 1, 2, 3, 0, 3], np.int32)
        ref = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
        for m in MODES:
            o = rend.render(_dev(y), _dev(dirs), mode=m, length=L).cpu().numpy()
            assert rend.sync() == 0
            assert_close(o, ref, what=f"{m} L={L}")
    # silent direction only -> exact zeros
    y = rng.standard_normal((2, 64)).astype(np.float32)
    for m in MODES:
        o = rend.render(_dev(y), _dev(np.array([3, 3], np.int32)), mode=m).cpu().numpy()
        assert not o.any()
    # no sources -> zeros of full length; empty sources -> empty output
    o = rend.render(_dev(np.zeros((0, 64), np.float32)), _dev(np.zeros(0, np.int32)), length=64)
    assert o.shape == (2, 64 + 230) and not o.cpu().numpy().any()
    o = rend.render(_dev(y), _dev(np.array([0, 1], np.int32)), length=0)
    assert o.shape[1] == 0


def test_bad_direction_is_silent_and_flagged(rend):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(6)
    _, idx, w, nnz, res = tables(rng, 4, 16)
    rend.load_filters(idx, w, nnz, 200, res)
    y = rng.standard_normal((3, 1000)).astype(np.float32)
    ref = oracle.render_sparse(y[:1], np.array([1], np.int32), idx, w, nnz, 200, res)
    for m in MODES:
        o = rend.render(_dev(y), _dev(np.array([1, 9, -2], np.int32)), mode=m).cpu().numpy()
        assert rend.sync() == hrir.HRIR_EINVAL
        assert rend.sync() == 0                          # flag cleared
        assert_close(o, ref, what=f"bad dirs {m}")


def test_invalid_arguments_rejected(rend):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(7)
    _, idx, w, nnz, res = tables(rng, 4, 16)
    bad_idx = idx.copy()
    bad_idx[0, 0, :2] = [5, 5]
    with pytest.raises(hrir.HRIRError):
        rend.load_filters(bad_idx, w, nnz, 200, res)
    bad_w = w.copy()
    bad_w[1, 1, 0] = -1.0
    with pytest.raises(hrir.HRIRError):
        rend.load_filters(idx, bad_w, nnz, 200, res)
    rend.load_filters(idx, w, nnz, 200, res)
    y = torch.zeros((2, 1001), device="cuda")            # row stride not a multiple of 16 bytes
    with pytest.raises(hrir.HRIRError):
        rend.render(y, _dev(np.zeros(2, np.int32)))


@pytest.mark.parametrize("dt", ["bfloat16", "float16"])
def test_16bit_sources(rend, dt):
    rng = np.random.default_rng(8)
    _, idx, w, nnz, res = tables(rng, 40, 16)
    S, L = 70, 20011
    ld = (L + 7) // 8 * 8
    y = np.zeros((S, ld), np.float32)
    y[:, :L] = synth.sources_ar1(rng, S, L)
    tdt = getattr(torch, dt)
    yq = torch.from_numpy(y).to(tdt)
    ydq = yq.float().numpy()                             # the values the kernel sees
    dirs = synth.directions(rng, S, 40)
    ref = oracle.render_sparse(ydq, dirs, idx, w, nnz, 200, res, length=L)
    rend.load_filters(idx, w, nnz, 200, res)
    for m in MODES:
        o = rend.render(yq.cuda(), _dev(dirs), mode=m, length=L).cpu().numpy()
        assert rend.sync() == 0
        assert_close(o, ref, what=f"{dt} {m}")


def test_deterministic_and_host_path(rend):
    rng = np.random.default_rng(9)
    _, idx, w, nnz, res = tables(rng, 30, 16)
    S, L = 300, 12345
    y = np.zeros((S, 12352), np.float32)
    y[:, :L] = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, 30)
    rend.load_filters(idx, w, nnz, 200, res)
    yd, dd = _dev(y), _dev(dirs)
    a = rend.render(yd, dd, length=L).cpu().numpy()
    b = rend.render(yd, dd, length=L).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    yh = torch.from_numpy(y).pin_memory()
    h = rend.render_host(yh, torch.from_numpy(dirs), length=L).numpy()
    h2 = rend.render_host(yh, torch.from_numpy(dirs), length=L).numpy()
    np.testing.assert_array_equal(h, h2)                  # the host path is deterministic too
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
    assert_close(a, ref, what="S=300")
    # the host path renders the sources in chunks (copies overlapped with the renders) and sums
    # the chunk outputs: the same result up to the order of the FP32 sums
    assert_close(h, ref, what="S=300 host path")
    hs = rend.render_host(torch.from_numpy(y[:7]).pin_memory(), torch.from_numpy(dirs[:7]), length=L).numpy()
    np.testing.assert_array_equal(hs, rend.render(_dev(y[:7]), _dev(dirs[:7]), length=L).cpu().numpy())


@pytest.fixture(scope="module")
def full_batch():
    """The batched workload (1024 sources x 480000 samples, 1250 directions) with the oracle's
    worker pool holding its sources (spawned processes: safe after CUDA initialisation)."""
    from oracle.pool import SlicedRenderer
    cfg = synth.batched_config(S=1024, L=480000, seed=2)
    ri, rw, rn = oracle.topk(cfg["G"], 16)
    pool = SlicedRenderer(cfg["y"], cfg["dirs"], ri, rw, rn, 200, cfg["res"])
    yield cfg, pool
    pool.close()


@pytest.mark.parametrize("k", [8, 16, 32])
def test_full_size_batched_config_every_output(rend, full_batch, k):
    """1024 sources x 480000 samples (10 s at 48 kHz), 1250 directions: the launch the
    benchmark times, compared with the FP64 oracle's full mix at every output sample (the
    oracle renders contiguous source slices in worker processes and sums them in FP64)."""
    cfg, pool = full_batch
    G = torch.from_numpy(cfg["G"]).cuda()
    idx_d, w_d, nnz_d = rend.topk_pack(G, k)
    idx = (idx_d.cpu().numpy().astype(np.int64) & 0xFFFF).astype(np.uint16)
    w, nnz = w_d.cpu().numpy(), nnz_d.cpu().numpy()
    ri, rw, rn = oracle.topk(cfg["G"], k)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(w.view(np.uint32), rw.view(np.uint32))
    rend.load_filters(idx, w, nnz, 200, cfg["res"])
    y = cfg["y"]
    S, L = y.shape
    out = {}
    yd = torch.from_numpy(y).cuda()
    for m in MODES:
        o = rend.render(yd, _dev(cfg["dirs"]), mode=m)
        assert rend.sync() == 0
        out[m] = o.cpu().numpy()
        assert out[m].shape == (2, L + 230) and np.isfinite(out[m]).all()
    pool.set_tables(ri, rw, rn)
    _, ref = pool.run(S, L, "sparse")
    rms = np.sqrt(np.mean(ref ** 2, axis=1))
    assert np.all(rms > 0)
    for m in MODES:
        err = np.max(np.abs(out[m] - ref), axis=1)
        print(f"FULLSIZE mode={m} K={k} max_err/rms={np.max(err / rms):.3e} (all {2 * (L + 230)} outputs)")
        assert np.all(err <= TOL * rms), f"{m} K={k}: err {err} > {TOL} x oracle rms {rms}"
