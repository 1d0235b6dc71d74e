"""GPU tests of the block-streaming path (continuous batching, Sec. IV-G partitioned
convolution): parity with the oracle and with the batch render, a session identical alone
and in a mix, admission refusal."""
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
    rng = np.random.default_rng(40)
    r = hrir.Renderer(0)
    _, idx, w, nnz, res = tables(rng, 30, 16)
    r.load_filters(idx, w, nnz, 200, res)
    r.tables = (idx, w, nnz, res)
    yield r
    r.close()


def run_to_completion(st, schedule, max_steps=100000):
    """schedule: {step: [(req_id, session, samples, dir), ...]}.  Returns {session: [2][n]}
    with each session's blocks concatenated from its first step, and admission codes."""
    out, codes = {}, {}
    live = set()
    step = 0
    while step < max_steps:
        for (rid, sess, y, d) in schedule.get(step, []):
            codes[rid] = st.admit(rid, sess, y, d)
            if codes[rid] == 0:
                live.add(rid)
        blocks, sessions, done = st.step()
        for r, s in enumerate(sessions):
            out.setdefault(s, []).append(np.array(blocks[r]))
        live -= set(done)
        step += 1
        if not live and step > max(schedule):
            a, p, _ = st.stats()
            if a == 0 and p == 0:
                break
    return {s: np.concatenate(v, axis=1) for s, v in out.items()}, codes


@pytest.mark.parametrize("block", [128, 256])
def test_single_source_stream_equals_full_convolution(rend, block):
    from paper_1502_03162_gb300 import hrir
    idx, w, nnz, res = rend.tables
    rng = np.random.default_rng(41)
    L = 12345
    y = synth.sources_ar1(rng, 1, L)[0].copy()
    st = hrir.Stream(rend, block, 16, 1 << 24)
    try:
        got, codes = run_to_completion(st, {0: [(7, 1, y, 5)]})
    finally:
        st.close()
    assert codes[7] == 0
    n_full = L + 230
    z = got[1]
    assert z.shape[1] == -(-n_full // block) * block
    ref = oracle.render_sparse(y[None], np.array([5], np.int32), idx, w, nnz, 200, res)
    assert_close(z[:, :n_full], ref, what=f"stream B={block}")
    assert not z[:, n_full:].any()
    yp = np.zeros((1, (L + 7) // 8 * 8), np.float32)
    yp[0, :L] = y
    b = rend.render(torch.from_numpy(yp).cuda(), torch.tensor([5], dtype=torch.int32, device="cuda"),
                    length=L)
    assert_close(z[:, :n_full], b.cpu().numpy(), what="stream vs batch")


def test_session_identical_alone_and_in_mix(rend):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(42)
    srcs = [synth.sources_ar1(rng, 1, int(n))[0].copy() for n in rng.integers(500, 20000, 24)]
    dirs = rng.integers(0, 30, 24)
    # session 3 has two sources starting at steps 2 and 9; the rest one session each
    sched = {}
    for i in range(24):
        if i in (3, 11):
            continue
        sched.setdefault(int(rng.integers(0, 40)), []).append((i, 100 + i, srcs[i], int(dirs[i])))
    sched.setdefault(2, []).append((3, 3, srcs[3], int(dirs[3])))
    sched.setdefault(9, []).append((11, 3, srcs[11], int(dirs[11])))
    st = hrir.Stream(rend, 256, 64, 1 << 24)
    try:
        mixed, codes = run_to_completion(st, sched)
    finally:
        st.close()
    assert all(c == 0 for c in codes.values())
    # session 3 alone, same schedule for its own sources
    alone_sched = {k: [r for r in v if r[1] == 3] for k, v in sched.items()}
    alone_sched = {k: v for k, v in alone_sched.items() if v}
    st = hrir.Stream(rend, 256, 64, 1 << 24)
    try:
        alone, _ = run_to_completion(st, alone_sched)
    finally:
        st.close()
    np.testing.assert_array_equal(alone[3], mixed[3])
    # and session 3 equals the oracle mix of its two sources with their start offsets
    idx, w, nnz, res = rend.tables
    starts = {r[0]: 256 * (k - min(alone_sched)) for k, v in alone_sched.items() for r in v}
    n = max(starts[i] + srcs[i].size for i in starts)
    y = np.zeros((len(starts), n), np.float32)
    d = []
    for j, i in enumerate(sorted(starts)):
        y[j, starts[i]:starts[i] + srcs[i].size] = srcs[i]
        d.append(int(dirs[i]))
    ref = oracle.render_sparse(y, np.array(d, np.int32), idx, w, nnz, 200, res)
    assert_close(alone[3][:, :ref.shape[1]], ref, what="two-source session")


def test_admission_refused_then_admitted(rend):
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(43)
    a = synth.sources_ar1(rng, 1, 3000)[0].copy()
    b = synth.sources_ar1(rng, 1, 3000)[0].copy()
    c = synth.sources_ar1(rng, 1, 3000)[0].copy()
    st = hrir.Stream(rend, 128, 2, 3000 * 4 * 2 + 4096)    # room for two sources
    try:
        assert st.admit(1, 1, a, 0) == hrir.HRIR_OK
        assert st.admit(2, 2, b, 1) == hrir.HRIR_OK
        assert st.admit(3, 3, c, 2) == hrir.HRIR_EBUSY      # no slot
        done = []
        for _ in range(200):
            _, _, d = st.step()
            done += d
            if 1 in done:
                break
        assert 1 in done
        assert st.admit(3, 3, c, 2) == hrir.HRIR_OK
        big = synth.sources_ar1(rng, 1, 10000)[0].copy()
        while 2 not in done:
            _, _, d = st.step()
            done += d
        assert st.admit(4, 4, big, 0) == hrir.HRIR_ENOMEM   # pool has no room
        with pytest.raises(hrir.HRIRError):
            st.admit(5, 5, a, 999)                          # bad direction
    finally:
        st.close()
