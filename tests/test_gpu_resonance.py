"""GPU parity of the per-source resonance stage (y * f, the first half of Eq. 2 in the order
(y * f) * g) computed as a Toeplitz-block GEMM on the tensor cores, against the oracle's
direct convolution (Sec. I footnote 2) of the dequantised 16-bit sources."""
import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth
from tests.gpu_util import TOL, tables

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
