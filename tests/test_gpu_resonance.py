"""GPU parity of the per-source resonance stage (y * f, the first half of Eq. 2 in the order
(y * f) * g) computed as a Toeplitz-block GEMM on the tensor cores, against the oracle's
direct convolution (Sec. I footnote 2) of the dequantised 16-bit sources."""
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


@pytest.mark.parametrize("dt", ["bfloat16", "float16"])
@pytest.mark.parametrize("S,L,res_len", [(5, 20011, 32), (3, 4096, 32), (2, 4097, 32), (4, 31, 32),
                                         (1, 1, 32), (6, 9000, 17)])
def test_resonance_gemm_matches_direct_convolution(rend, dt, S, L, res_len):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(S * 1000 + L + res_len)
    _, idx, w, nnz, res = tables(rng, 4, 16, res_len=res_len)
    rend.load_filters(idx, w, nnz, 200, res)
    ld = (L + 7) // 8 * 8 + 8
    y = np.zeros((S, ld), np.float32)
    y[:, :L] = synth.sources_ar1(rng, S, L)
    y[:, L:] = np.nan                                    # padding is never read
    yq = torch.from_numpy(y).to(getattr(torch, dt))
    ydq = yq.float().numpy()
    for full in (True, False):
        u = hrir.hrir_resonance_per_source(rend.ctx, yq.cuda(), full=full, length=L)
        assert rend.sync() == 0
        u = u.cpu().numpy().astype(np.float64)
        n_out = L + res_len - 1 if full else L
        assert u.shape == (S, 2, n_out)
        for s in range(S):
            for e in range(2):
                ref = oracle.conv_direct(res[e], ydq[s, :L])[:n_out]
                rms = np.sqrt(np.mean(ref ** 2))
                err = np.max(np.abs(u[s, e] - ref))
                assert err <= TOL * rms, f"{dt} s={s} e={e} full={full}: {err} > {TOL} x {rms}"


def test_resonance_gemm_rejects_fp32_sources(rend):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(3)
    _, idx, w, nnz, res = tables(rng, 4, 16)
    rend.load_filters(idx, w, nnz, 200, res)
    y = torch.zeros((2, 64), device="cuda")
    with pytest.raises(ValueError):
        hrir.hrir_resonance_per_source(rend.ctx, y)


@pytest.mark.parametrize("dt,S,L,n_views", [("bfloat16", 37, 20011, 3), ("float16", 130, 4099, 2),
                                            ("bfloat16", 3, 200, 1)])
def test_precomputed_resonance_rendered_to_several_views(rend, dt, S, L, n_views):
    """The order (y * f) * g of Eq. 2: u = y * f once per source on the tensor cores, then each
    view mixes u through its own directions' reflection taps alone.  Every view equals the
    oracle's mix in that order (and so the direct render of the same sources, Eq. 2)."""
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(S + L + n_views)
    n_dirs = 50
    _, idx, w, nnz, res = tables(rng, n_dirs, 16)
    rend.load_filters(idx, w, nnz, 200, res)
    ld = (L + 7) // 8 * 8
    y = np.zeros((S, ld), np.float32)
    y[:, :L] = synth.sources_ar1(rng, S, L)
    yq = torch.from_numpy(y).to(getattr(torch, dt))
    ydq = yq.float().numpy()
    u = hrir.hrir_resonance_per_source(rend.ctx, yq.cuda(), full=True, length=L)
    dirs = np.stack([synth.directions(rng, S, n_dirs) for _ in range(n_views)])
    dirs[0, 0] = n_dirs + 5                          # an id out of range: that source is silent
    out = hrir.hrir_render_precomputed(rend.ctx, u, torch.from_numpy(dirs).cuda())
    assert rend.sync() == hrir.HRIR_EINVAL            # the bad id is flagged ...
    assert rend.sync() == 0
    out = out.cpu().numpy()
    assert out.shape == (n_views, 2, L + 230)
    for v in range(n_views):
        keep = np.ones(S, bool)
        if v == 0:
            keep[0] = False                          # ... and rendered as silence
        ref = oracle.render_sparse(ydq[keep], dirs[v][keep], idx, w, nnz, 200, res, length=L, order=1)
        assert_close(out[v], ref, what=f"{dt} view {v}")
    if n_views > 1:
        same = hrir.hrir_render_precomputed(rend.ctx, u, torch.from_numpy(dirs[1:]).cuda(), full=False)
        assert rend.sync() == 0
        Lu = u.shape[2]                              # u holds the full y * f: L + Lf - 1 samples
        assert same.shape == (n_views - 1, 2, Lu)
        assert_close(same.cpu().numpy()[0], out[1, :, :Lu], what="first len(u) samples")
