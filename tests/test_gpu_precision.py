"""GPU parity of the precision workload: sources stored in BF16 / FP16, FP32 arithmetic,
1024..8192 sources of 480000 samples mixed with a compensated sum, K = 4..64 taps.

The mix is checked at sampled output positions against the FP64 oracle, which needs only the
231 source samples before each position: the oracle renders, per position, the window
y[s][p - 230 .. p] of every source (the full render's output at p depends on nothing else),
so its cost does not grow with the source length.  Two errors per case, both per ear as
max |gpu - oracle| / RMS(oracle) over the sampled positions:
  * against the oracle on the dequantised sources (the values the kernel reads): the
    arithmetic error, bounded by 1e-5 as for the FP32 path;
  * against the oracle on the FP32 sources before quantisation: the storage error of the
    16-bit type, reported (it is the input's own rounding, about 2^-9 / 2^-12 relative)."""
import numpy as np
import pytest

import oracle
from paper_1502_03162_gb300 import synth
from tests.gpu_util import TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

S_MAX, L = 8192, 480000
N_DIRS, REFL, NREFL = 1250, 200, 96       # 96 reflections per row, so top-64 keeps 64 taps
H = 32 + REFL - 1


@pytest.fixture(scope="module")
def batch():
    """S_MAX sources x L samples of AR(1) noise (seed 3), on the device as BF16 and FP16 (each
    converted on the host, so the oracle's dequantised values are exactly the device's), and
    the FP32 windows before the sampled output positions."""
    from paper_1502_03162_gb300 import hrir
    rng = np.random.default_rng(3)
    res = synth.resonance(rng)
    G = synth.reflection_bank(rng, N_DIRS, n_refl=NREFL)
    dirs = synth.directions(rng, S_MAX, N_DIRS)
    edges = np.array([0, 1, 230, 6655, 6656, L - 1, L, L + 229])
    pos = np.unique(np.concatenate([edges, rng.integers(0, L + 230, 100)]))
    lo = np.maximum(pos - 230, 0)
    hi = np.minimum(pos + 1, L)
    win = np.zeros((pos.size, S_MAX, 231), np.float32)
    dev = {dt: torch.empty((S_MAX, L), dtype=getattr(torch, dt), device="cuda")
           for dt in ("bfloat16", "float16")}
    chunk = 256
    for s0 in range(0, S_MAX, chunk):
        y = synth.sources_ar1(rng, chunk, L)
        for dt, d in dev.items():
            d[s0:s0 + chunk].copy_(torch.from_numpy(y).to(getattr(torch, dt)))
        for i in range(pos.size):
            win[i, s0:s0 + chunk, :hi[i] - lo[i]] = y[:, lo[i]:hi[i]]
    torch.cuda.synchronize()
    r = hrir.Renderer(0)
    yield dict(r=r, dev=dev, res=res, G=G, dirs=dirs, pos=pos, lo=lo, hi=hi, win=win)
    r.close()


def _oracle_at(b, win, S, idx, w, nnz):
    """The exact mix of the first S sources at every sampled position, [2][n_pos]."""
    ref = np.zeros((2, b["pos"].size))
    for i, p in enumerate(b["pos"]):
        n = int(b["hi"][i] - b["lo"][i])
        y = np.ascontiguousarray(win[i, :S, :max(n, 1)])
        ref[:, i] = oracle.render_at(y, b["dirs"][:S], idx, w, nnz, REFL, b["res"],
                                     [int(p - b["lo"][i])], length=n)[:, 0]
    return ref


CASES = [("bfloat16", 2048, 16), ("float16", 2048, 16), ("bfloat16", 8192, 16),
         ("float16", 8192, 16), ("bfloat16", 8192, 4), ("bfloat16", 8192, 8),
         ("bfloat16", 8192, 32), ("bfloat16", 8192, 64), ("float16", 8192, 4),
         ("float16", 8192, 64), ("bfloat16", 1024, 64)]


@pytest.mark.parametrize("dt,S,k", CASES)
def test_16bit_sources_many_sources_sampled(batch, dt, S, k):
    b = batch
    idx, w, nnz = oracle.topk(b["G"], k)
    assert np.all(nnz == k)
    r = b["r"]
    r.load_filters(idx, w, nnz, REFL, b["res"])
    out = r.render(b["dev"][dt][:S], torch.from_numpy(b["dirs"][:S]).cuda(), mode="sparse")
    assert r.sync() == 0
    out = out.cpu().numpy()
    assert out.shape == (2, L + H - 1) and np.isfinite(out).all()
    got = out[:, b["pos"]].astype(np.float64)
    if ("deq", dt) not in b:      # the windows as the device holds them (same host rounding)
        b[("deq", dt)] = torch.from_numpy(b["win"]).to(getattr(torch, dt)).float().numpy()
    deq = b[("deq", dt)]
    ref_q = _oracle_at(b, deq, S, idx, w, nnz)
    ref_f = _oracle_at(b, b["win"], S, idx, w, nnz)
    rms = np.sqrt(np.mean(ref_q ** 2, axis=1))
    err_q = np.max(np.abs(got - ref_q), axis=1) / rms
    err_f = np.max(np.abs(got - ref_f), axis=1) / np.sqrt(np.mean(ref_f ** 2, axis=1))
    print(f"PRECISION dtype={dt} S={S} K={k} err_vs_dequantised/rms={err_q.max():.3e} "
          f"err_vs_fp32_sources/rms={err_f.max():.3e}")
    assert np.all(err_q <= TOL), f"{dt} S={S} K={k}: {err_q} > {TOL}"
