"""hrir_render_batch_noalloc: the render for callers that must not allocate device memory
while rendering -- a real-time audio thread, where an allocator call can block for an
unbounded time, or a host that gives the library a fixed device-memory budget up front.  It
keeps its partial sums in the library's fixed device array instead of the context's
growable workspace.

Here it must give the same mix as hrir_render_batch, bit for bit (same kernels, same work
partition, same summation order), call after call, leave the device's free memory unchanged
once its first call has set it up, and agree with the FP64 oracle.

Collected last (file name) so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth
from tests.gpu_util import assert_close, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(200, 60001), (77, 33333)]      # (sources, samples): two calls of different shapes


def test_noalloc_matches_render_batch_on_consecutive_calls():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    try:
        rng = np.random.default_rng(31)
        _, idx, w, nnz, res = tables(rng, 60, 16)
        r.load_filters(idx, w, nnz, 200, res)
        inputs = []
        for S, L in CASES:
            ld = (L + 7) // 8 * 8
            y = np.zeros((S, ld), np.float32)
            y[:, :L] = synth.sources_ar1(rng, S, L)
            dirs = synth.directions(rng, S, 60)
            inputs.append((S, L, y, dirs, torch.from_numpy(y).cuda(), torch.from_numpy(dirs).cuda()))
        # every buffer is allocated before the free-memory reading; one set-up call per mode
        # (the first call on a device looks up, and under lazy loading reserves, the array)
        outs = {(c, m): torch.full((2, L + 230), float("nan"), device="cuda")
                for c, (S, L, *_) in enumerate(inputs) for m in ("sparse", "dense")}
        for m in ("sparse", "dense"):
            S, L, _, _, yd, dd = inputs[0]
            hrir.hrir_render_batch_noalloc(r.ctx, yd, dd, outs[(0, m)], mode=m, length=L)
        assert r.sync() == 0
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        got = {}
        for c, (S, L, _, _, yd, dd) in enumerate(inputs):
            for m in ("sparse", "dense"):
                got[(c, m)] = hrir.hrir_render_batch_noalloc(r.ctx, yd, dd, outs[(c, m)], mode=m,
                                                             length=L)
                assert r.sync() == 0
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        for c, (S, L, y, dirs, yd, dd) in enumerate(inputs):
            ref = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
            for m in ("sparse", "dense"):
                g = got[(c, m)].cpu().numpy()
                assert g.shape == (2, L + 230) and np.isfinite(g).all()
                want = r.render(yd, dd, mode=m, length=L).cpu().numpy()
                assert r.sync() == 0
                np.testing.assert_array_equal(g, want, err_msg=f"noalloc call {c} {m}")
                assert_close(g, ref, what=f"noalloc call {c} {m} vs oracle")
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
