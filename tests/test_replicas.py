"""The multi-process path of bench.py on the host: two ranks over gloo (world size 2).

Each rank renders its own batch, so the only cross-rank steps are the barrier around the
timed region, the maximum of the step times over ranks and the whole-job rate.  These run
here as two CPU processes on the gloo backend; under torchrun on GPUs the same class runs
over NCCL.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    try:
        import bench
        r = bench.Replicas("gloo", device="cpu")
        r.barrier()
        ms = r.max_over_ranks(1.5 + rank)          # rank 1 is the slower one
        q.put((rank, r.world, ms, r.whole_job(1000, ms), r.seed(2)))
        r.barrier()
        r.close()
    except Exception as e:  # reported to the parent, never silently lost
        q.put((rank, "error", repr(e)))


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            item = q.get(timeout=120)
            got[item[0]] = item
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for rank in (0, 1):
        _, world, ms, value, seed = got[rank]
        assert world == 2
        assert ms == 2.5                              # the slowest rank's step time on both
        assert value == pytest.approx(1000 * 2 / 2.5e-3)
        assert seed == 2 + rank                       # independent batches


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Replicas("gloo", device="cpu")
    assert (r.rank, r.world, r.dist) == (0, 1, None)
    r.barrier()
    assert r.max_over_ranks(3.25) == 3.25
    assert r.whole_job(10, 2.0) == pytest.approx(5000.0)
    r.close()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args) is None          # no oracle work, nothing printed
    assert capsys.readouterr().out == ""
