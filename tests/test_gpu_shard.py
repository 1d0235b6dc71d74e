"""GPU parity of the source-sharding calls (hrir_render_reflections, hrir_apply_resonance)
against the FP64 oracle, with the shards of several ranks emulated on one GPU: each slice of
the batch is rendered to its reflection mix, the mixes are stacked in rank order (what the
gather of paper_1502_03162_gb300.shard delivers) and the resonance is applied once."""
import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth
from paper_1502_03162_gb300.shard import render_sharded, shard_range
from tests.gpu_util import assert_close, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rend():
    from paper_1502_03162_gb300 import hrir
    r = hrir.Renderer(0)
    yield r
    r.close()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("S,L,world,full", [(37, 20011, 2, True), (37, 20011, 3, False),
                                            (200, 50000, 4, True), (5, 7000, 8, True)])
def test_emulated_shards_match_the_oracle(rend, S, L, world, full):
    rng = np.random.default_rng(S + L + world)
    _, idx, w, nnz, res = tables(rng, 300, 16)
    rend.load_filters(idx, w, nnz, 200, res)
    ld = (L + 3) // 4 * 4
    y = np.zeros((S, ld), np.float32)
    y[:, :L] = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, 300)
    yd, dd = _cuda(y), _cuda(dirs)
    z_len = L + 199 if full else L
    parts = torch.empty((world, 2, z_len), dtype=torch.float32, device="cuda")
    for r in range(world):
        s0, s1 = shard_range(S, r, world)
        rend.render_reflections(yd[s0:s1], dd[s0:s1], full=full, length=L, z=parts[r])
    out = rend.apply_resonance(parts, full=full).cpu().numpy()
    assert rend.sync() == 0
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, 200, res, length=L)
    if not full:
        ref = ref[:, :L]
    assert out.shape == ref.shape
    assert_close(out, ref, what=f"{world} shards of {S} sources")
    # the reflection mix of one shard alone: the oracle with the identity resonance
    s0, s1 = shard_range(S, 0, world)
    z0 = oracle.render_sparse(y[s0:s1], dirs[s0:s1], idx, w, nnz, 200, np.ones((2, 1), np.float32),
                              length=L)[:, :z_len]
    assert_close(parts[0].cpu().numpy(), z0, what="one shard's reflection mix")


def test_one_part_equals_the_fused_render(rend):
    """Without a process group render_sharded is the reflection mix plus the resonance; it
    agrees with hrir_render_batch (the resonance fused into the reduction) to FP32 rounding,
    and BF16 sources take the same path."""
    rng = np.random.default_rng(3)
    _, idx, w, nnz, res = tables(rng, 300, 16)
    rend.load_filters(idx, w, nnz, 200, res)
    S, L = 64, 40000
    y = synth.sources_ar1(rng, S, L)
    dirs = synth.directions(rng, S, 300)
    yd, dd = _cuda(y), _cuda(dirs)
    a = render_sharded(rend, yd, dd).cpu().numpy()
    b = rend.render(yd, dd).cpu().numpy()
    assert rend.sync() == 0
    assert_close(a, b, tol=2e-6, what="sharded vs fused")
    yb = yd.to(torch.bfloat16)
    c = render_sharded(rend, yb, dd).cpu().numpy()
    ref = oracle.render_sparse(yb.float().cpu().numpy(), dirs, idx, w, nnz, 200, res)
    assert_close(c, ref, what="BF16 sources, sharded")


def test_empty_shard_and_lengths(rend):
    """A rank without sources contributes a zero mix; z_len 0 and out_len 0 are no-ops."""
    rng = np.random.default_rng(4)
    _, idx, w, nnz, res = tables(rng, 50, 8)
    rend.load_filters(idx, w, nnz, 200, res)
    L = 3000
    y = synth.sources_ar1(rng, 3, L)
    dirs = synth.directions(rng, 3, 50)
    parts = torch.full((2, 2, L + 199), 7.0, dtype=torch.float32, device="cuda")
    rend.render_reflections(_cuda(y), _cuda(dirs), z=parts[0])
    rend.render_reflections(_cuda(y[:0]), _cuda(dirs[:0]), length=L, z=parts[1])
    assert torch.count_nonzero(parts[1]).item() == 0
    out = rend.apply_resonance(parts).cpu().numpy()
    assert rend.sync() == 0
    assert_close(out, oracle.render_sparse(y, dirs, idx, w, nnz, 200, res), what="empty shard")
    assert rend.render_reflections(_cuda(y), _cuda(dirs), length=0).shape[1] == 0
