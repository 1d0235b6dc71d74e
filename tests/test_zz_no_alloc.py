"""hrir_render_batch_noalloc: the render for callers that must not allocate device memory
(real-time audio threads, fixed-budget hosts).  It keeps its partial sums in the library's
fixed device array; here it must give the same mix as hrir_render_batch, call after call.

Collected last (file name) so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_1502_03162_gb300 import synth
from tests.gpu_util import assert_close, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_render_batch_on_consecutive_calls():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    try:
        rng = np.random.default_rng(31)
        _, idx, w, nnz, res = tables(rng, 60, 16)
        r.load_filters(idx, w, nnz, 200, res)
        for call, (S, L) in enumerate([(200, 60001), (77, 33333)]):
            ld = (L + 7) // 8 * 8
            y = np.zeros((S, ld), np.float32)
            y[:, :L] = synth.sources_ar1(rng, S, L)
            dirs = synth.directions(rng, S, 60)
            yd = torch.from_numpy(y).cuda()
            dd = torch.from_numpy(dirs).cuda()
            for mode in ("sparse", "dense"):
                ref = r.render(yd, dd, mode=mode, length=L).cpu().numpy()
                out = torch.full((2, L + 230), float("nan"), device="cuda")
                got = hrir.hrir_render_batch_noalloc(r.ctx, yd, dd, out, mode=mode, length=L)
                assert r.sync() == 0
                got = got.cpu().numpy()
                assert got.shape == ref.shape and np.isfinite(got).all()
                assert_close(got, ref, what=f"noalloc call {call} {mode}")
    finally:
        r.close()


def test_noalloc_rejects_renders_beyond_its_fixed_scratch():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    try:
        rng = np.random.default_rng(32)
        _, idx, w, nnz, res = tables(rng, 8, 16)
        r.load_filters(idx, w, nnz, 200, res)
        S, L = 4096, 100000           # partial sums of ~55 MB > 32 MiB
        y = torch.empty((S, L), dtype=torch.bfloat16, device="cuda")
        d = torch.zeros(S, dtype=torch.int32, device="cuda")
        out = torch.empty((2, L + 230), device="cuda")
        with pytest.raises(hrir.HRIRError) as ei:
            hrir.hrir_render_batch_noalloc(r.ctx, y, d, out)
        assert ei.value.status == hrir.HRIR_EINVAL and "scratch" in str(ei.value)
    finally:
        r.close()
