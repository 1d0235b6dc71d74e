"""Source sharding on the host: the source partition, and two ranks over gloo (world size 2)
running paper_1502_03162_gb300.shard.render_sharded with the oracle standing in for the
library's two calls.  The sharded output (every rank's reflection mix gathered in rank order,
the resonance applied once to their sum) must equal the oracle's render of the whole batch on
both ranks.  On GPUs the same module runs over NCCL with the library's kernels
(tests/test_gpu_shard.py checks those kernels on one GPU with emulated shards)."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_range_partitions_the_sources():
    from paper_1502_03162_gb300.shard import shard_range
    for n in (0, 1, 5, 7, 1024, 1031):
        for world in (1, 2, 3, 8):
            rs = [shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))     # contiguous, disjoint
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
    with pytest.raises(ValueError):
        shard_range(10, 0, 0)


def _batch():
    """A small seeded batch with the benchmark's structure (AR(1) sources, top-K taps)."""
    from paper_1502_03162_gb300 import synth
    import oracle
    rng = np.random.default_rng(11)
    S, L, Lg, K = 9, 700, 200, 16
    y = synth.sources_ar1(rng, S, L)
    G = synth.reflection_bank(rng, 40, n_refl=60, refl_len=Lg)
    idx, w, nnz = oracle.topk(G, K)
    dirs = synth.directions(rng, S, 40)
    res = (rng.standard_normal((2, 32)) * np.exp(-np.arange(32) / 6.0)).astype(np.float32)
    return y, dirs, idx, w, nnz, Lg, res


class OracleRenderer:
    """The library's two sharding calls restated with the oracle (FP64, host tensors)."""

    def __init__(self, idx, w, nnz, Lg, res):
        self.idx, self.w, self.nnz, self.Lg, self.res = idx, w, nnz, Lg, res

    def render_reflections(self, src, dirs, full=True, length=None, stream=None):
        import oracle
        import torch
        one = np.ones((2, 1))                                   # the identity resonance
        z = oracle.render_sparse(src.numpy(), dirs.numpy(), self.idx, self.w, self.nnz, self.Lg, one,
                                 length=length)
        return torch.from_numpy(np.ascontiguousarray(z))

    def apply_resonance(self, parts, full=True, stream=None):
        import torch
        z = parts.numpy().sum(axis=0)                           # rank order
        return torch.from_numpy(np.stack([np.convolve(z[e], self.res[e].astype(np.float64))
                                          for e in range(2)]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        from paper_1502_03162_gb300.shard import render_sharded, shard_range
        dist.init_process_group("gloo")
        y, dirs, idx, w, nnz, Lg, res = _batch()
        s0, s1 = shard_range(y.shape[0], rank, world)
        rend = OracleRenderer(idx, w, nnz, Lg, res)
        out = render_sharded(rend, torch.from_numpy(np.ascontiguousarray(y[s0:s1])),
                             torch.from_numpy(dirs[s0:s1]))
        q.put((rank, out.numpy(), (s0, s1)))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, never silently lost
        q.put((rank, "error", repr(e)))


def test_two_ranks_render_the_whole_batch():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            item = q.get(timeout=180)
            got[item[0]] = item
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs), got
    y, dirs, idx, w, nnz, Lg, res = _batch()
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, Lg, res)
    assert got[0][2] == (0, 5) and got[1][2] == (5, 9)          # disjoint slices of 9 sources
    for r in (0, 1):
        out = got[r][1]
        assert not isinstance(out, str), out
        assert out.shape == ref.shape
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(got[0][1], got[1][1])                  # the same output on every rank


def test_single_process_is_one_part(monkeypatch):
    """No process group: the rank's own mix is the only part."""
    import oracle
    import torch
    from paper_1502_03162_gb300.shard import render_sharded
    y, dirs, idx, w, nnz, Lg, res = _batch()
    out = render_sharded(OracleRenderer(idx, w, nnz, Lg, res), torch.from_numpy(y),
                         torch.from_numpy(dirs))
    ref = oracle.render_sparse(y, dirs, idx, w, nnz, Lg, res)
    assert np.max(np.abs(out.numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
