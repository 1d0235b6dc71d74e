"""The Python binding's argument checks, on the CPU.

The C ABI receives raw pointers and sizes, so the binding checks every tensor against the
extents the kernels will touch before it calls the library.  Here the library is replaced by
a recorder and CUDA tensors by host tensors that report themselves as CUDA tensors, so that
the call patterns of the tests and the benchmark run through every wrapper without a GPU:
valid calls reach the library with the right sizes, invalid ones raise ValueError first.
"""
import numpy as np
import pytest
import torch

import oracle.mlp as omlp
from paper_1502_03162_gb300 import hrir

CTX = 12345
FAKE_DEVICE = "fake-cuda"


class FakeCuda:
    """A host tensor that reports itself as a CUDA tensor (metadata and pointers only)."""

    def __init__(self, t):
        self._t = t

    is_cuda = True
    device = FAKE_DEVICE

    def __getattr__(self, name):
        return getattr(self._t, name)

    def __getitem__(self, i):
        return FakeCuda(self._t[i])


def fc(shape, dtype=torch.float32):
    return FakeCuda(torch.zeros(shape, dtype=dtype))


class FakeLib:
    """Records the library calls; out_len follows the loaded filters (Lf 32, Lg 200)."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("hrir_"):
            raise AttributeError(name)

        def call(*args):
            self.calls.append((name, args))
            if name == "hrir_out_len":
                return args[1] + 230 if args[2] else args[1]
            if name == "hrir_mlp_param_count":
                return omlp.param_count(args[0])
            if name == "hrir_mlp_act_stride":
                return 3 * 256
            if name == "hrir_last_error":
                return b""
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    fake = FakeLib()
    monkeypatch.setattr(hrir, "_lib", fake)
    real_empty = torch.empty

    def empty(*shape, dtype=None, device=None, **kw):
        if device == FAKE_DEVICE:
            return FakeCuda(real_empty(*shape, dtype=dtype, **kw))
        return real_empty(*shape, dtype=dtype, device=device, **kw)
    monkeypatch.setattr(torch, "empty", empty)
    monkeypatch.setitem(hrir._RES_LEN, CTX, 32)
    return fake


def last(fake, name):
    calls = [a for n, a in fake.calls if n == name]
    assert calls, f"{name} was not called"
    return calls[-1]


# ---- valid call patterns reach the library -------------------------------------------------
def test_render_batch_valid(lib):
    S, L, ld = 37, 30001, 30008
    src, dirs = fc((S, ld)), fc((S,), torch.int32)
    out = hrir.hrir_render_batch(CTX, src, dirs, length=L, stream=0)
    a = last(lib, "hrir_render_batch")
    assert a[1:4] == (S, L, ld) and tuple(out.shape) == (2, L + 230)
    hrir.hrir_render_batch(CTX, fc((S, ld), torch.bfloat16), dirs, length=L, out=fc((2, L + 230)),
                           stream=0)
    hrir.hrir_render_batch(CTX, fc((0, 64)), fc((0,), torch.int32), length=64, stream=0)
    hrir.hrir_render_batch(CTX, fc((2, 64)), fc((2,), torch.int32), length=0, stream=0)
    hrir.hrir_render_batch(CTX, fc((2, 1001)), fc((2,), torch.int32), stream=0)  # C side judges ld


def test_render_host_and_noalloc_valid(lib):
    S, L, ld = 7, 12345, 12352
    out = hrir.hrir_render_batch_host(CTX, torch.zeros((S, ld)), torch.zeros(S, dtype=torch.int32),
                                      length=L, stream=0)
    assert tuple(out.shape) == (2, L + 230) and last(lib, "hrir_render_batch_host")[1:4] == (S, L, ld)
    hrir.hrir_render_batch_noalloc(CTX, fc((S, ld)), fc((S,), torch.int32), fc((2, L + 230)),
                                   length=L, stream=0)


def test_topk_moving_resonance_mlp_valid(lib):
    S, n_seg, k, L = 4, 12, 16, 3000
    g = fc((S, n_seg, 2, 200))
    idx, w, nnz = hrir.hrir_topk_pack(CTX, g, k, stream=0)
    assert last(lib, "hrir_topk_pack")[1:4] == (S * n_seg * 2, 200, k)
    hrir.hrir_topk_pack(CTX, g, k, fc((S, n_seg, 2, k), torch.int16), fc((S, n_seg, 2, k)),
                        fc((S, n_seg, 2), torch.uint8), stream=0)
    out = hrir.hrir_render_moving(CTX, fc((S, 3000)), idx, w, nnz, 256, length=L, stream=0)
    assert tuple(out.shape) == (2, L + 230)
    u = hrir.hrir_resonance_per_source(CTX, fc((S, 3008), torch.float16), length=L, stream=0)
    assert tuple(u.shape) == (S, 2, L + 31)
    n, P = 77, omlp.param_count(200)
    rows, params = fc((n, 3)), fc((P,))
    o = hrir.hrir_mlp_forward(CTX, rows, params, 200, acts=fc((n, 3 * 256)), stream=0)
    hrir.hrir_mlp_forward_bf16(CTX, rows, params, 200, stream=0)
    hrir.hrir_mlp_backward(CTX, rows, params, fc((n, 3 * 256)), o, fc((n, 200)), 200, stream=0)
    hrir.hrir_mlp_adam(CTX, params, fc((P,)), fc((P,)), fc((P,)), 1, 1e-3, stream=0)


def test_load_filters_and_admit_valid(lib):
    idx = np.zeros((5, 2, 16), np.uint16)
    hrir.hrir_load_filters(CTX, idx, np.zeros((5, 2, 16), np.float32), np.zeros((5, 2), np.uint8),
                           200, np.zeros((2, 32), np.float32))
    assert last(lib, "hrir_load_filters")[1:5] == (5, 2, 200, 16)
    hrir.hrir_load_filters(CTX, idx.astype(np.int64), np.zeros((5, 2, 16)), np.zeros((5, 2)), 200,
                           np.zeros((2, 32)))
    assert hrir.hrir_stream_admit(CTX, 1, 1, np.zeros(3000, np.float32), 0) == 0
    assert hrir.hrir_stream_admit(CTX, 2, 2, torch.zeros(100), 3) == 0


# ---- invalid calls never reach the library --------------------------------------------------
def _rejected(lib, fn, *args, **kw):
    n = len(lib.calls)
    with pytest.raises(ValueError):
        fn(*args, **kw)
    assert not [c for c in lib.calls[n:] if c[0] not in ("hrir_out_len", "hrir_mlp_param_count",
                                                         "hrir_mlp_act_stride")]


def test_render_batch_rejects(lib):
    S, ld = 8, 1000
    dirs = fc((S,), torch.int32)
    r = lambda *a, **k: _rejected(lib, hrir.hrir_render_batch, CTX, *a, stream=0, **k)  # noqa: E731
    r(torch.zeros((S, ld)), dirs)                          # host source
    r(fc((S, ld), torch.float64), dirs)                    # dtype
    r(fc((S, ld)), dirs, length=ld + 1)                    # longer than the rows
    r(fc((S, ld)), fc((S - 1,), torch.int32))              # too few directions
    r(fc((S, ld)), fc((S,), torch.int64))                  # direction dtype
    r(fc((S, ld)), dirs, out=fc((2, ld + 229)))            # output too short
    r(fc((S, ld)), dirs, out=fc((1, ld + 230)))            # one ear only
    r(fc((S, ld)), dirs, out=fc((2, ld + 230), torch.float16))
    r(FakeCuda(torch.zeros((ld, S)).t()), dirs)            # column-major rows


def test_host_and_noalloc_reject(lib):
    S, ld = 4, 500
    _rejected(lib, hrir.hrir_render_batch_host, CTX, fc((S, ld)), torch.zeros(S, dtype=torch.int32),
              stream=0)
    _rejected(lib, hrir.hrir_render_batch_host, CTX, torch.zeros((S, ld)),
              torch.zeros(S, dtype=torch.int64), stream=0)
    _rejected(lib, hrir.hrir_render_batch_host, CTX, torch.zeros((S, ld)),
              torch.zeros(S, dtype=torch.int32), out=torch.zeros((2, 10)), stream=0)
    _rejected(lib, hrir.hrir_render_batch_noalloc, CTX, fc((S, ld)), torch.zeros(S, dtype=torch.int32),
              fc((2, ld + 230)), stream=0)
    _rejected(lib, hrir.hrir_render_batch_noalloc, CTX, fc((S, ld)), fc((S,), torch.int32),
              fc((2, ld)), stream=0)


def test_topk_and_moving_reject(lib):
    S, n_seg, k = 3, 5, 16
    g = fc((S, n_seg, 2, 200))
    _rejected(lib, hrir.hrir_topk_pack, CTX, fc((S, n_seg, 2, 200), torch.float64), k, stream=0)
    _rejected(lib, hrir.hrir_topk_pack, CTX, g, k, fc((S, n_seg, 2, k), torch.uint8), stream=0)
    _rejected(lib, hrir.hrir_topk_pack, CTX, g, k, None, fc((S, n_seg, 2, k - 1)), stream=0)
    _rejected(lib, hrir.hrir_topk_pack, CTX, g, k, None, None, fc((S, n_seg, 2), torch.int32),
              stream=0)
    idx, w, nnz = fc((S, n_seg, 2, k), torch.int16), fc((S, n_seg, 2, k)), fc((S, n_seg, 2), torch.uint8)
    y = fc((S, 1200))
    mv = lambda *a, **kw: _rejected(lib, hrir.hrir_render_moving, CTX, *a, stream=0, **kw)  # noqa: E731
    mv(y, fc((S, n_seg, 2, k), torch.uint8), w, nnz, 256)  # index bytes too narrow
    mv(y, idx, fc((S, n_seg, 2, k), torch.float64), nnz, 256)
    mv(y, idx, w, fc((S, n_seg, 2), torch.int32), 256)
    mv(y, idx, w, fc((S, n_seg - 1, 2), torch.uint8), 256)
    mv(fc((S + 1, 1200)), idx, w, nnz, 256)                # tables for other sources
    mv(y, idx, w, nnz, 256, length=1201)
    mv(y, idx, w, nnz, 256, out=fc((2, 1200)))


def test_resonance_mlp_filters_admit_reject(lib):
    _rejected(lib, hrir.hrir_resonance_per_source, CTX, fc((2, 64)), stream=0)   # FP32 source
    _rejected(lib, hrir.hrir_resonance_per_source, CTX, fc((2, 64), torch.bfloat16),
              out=fc((2, 2, 64)), stream=0)
    _rejected(lib, hrir.hrir_resonance_per_source, CTX, fc((2, 64), torch.bfloat16),
              out=FakeCuda(torch.zeros((2, 2, 100)).transpose(0, 1)), stream=0)
    P = omlp.param_count(200)
    _rejected(lib, hrir.hrir_mlp_forward, CTX, fc((10, 3)), fc((P - 1,)), 200, stream=0)
    _rejected(lib, hrir.hrir_mlp_forward, CTX, fc((10, 2)), fc((P,)), 200, stream=0)
    _rejected(lib, hrir.hrir_mlp_forward_bf16, CTX, fc((10, 3)), fc((P,), torch.bfloat16), 200,
              stream=0)
    _rejected(lib, hrir.hrir_mlp_adam, CTX, fc((P,)), fc((P - 1,)), fc((P,)), fc((P,)), 1, 1e-3,
              stream=0)
    idx = np.zeros((5, 2, 16), np.int64)
    w, nnz, res = np.zeros((5, 2, 16), np.float32), np.zeros((5, 2), np.uint8), np.zeros((2, 32))
    bad = idx.copy()
    bad[0, 0, 0] = 70000                                   # does not fit 16 bits
    _rejected(lib, hrir.hrir_load_filters, CTX, bad, w, nnz, 200, res)
    _rejected(lib, hrir.hrir_load_filters, CTX, idx, w[:, :, :8], nnz, 200, res)
    _rejected(lib, hrir.hrir_load_filters, CTX, idx, w, nnz[:4], 200, res)
    _rejected(lib, hrir.hrir_load_filters, CTX, idx, w, nnz, 200, np.zeros((1, 32)))
    _rejected(lib, hrir.hrir_stream_admit, CTX, 1, 1, np.zeros(10, np.float64), 0)
    _rejected(lib, hrir.hrir_stream_admit, CTX, 1, 1, np.zeros(20, np.float32)[::2], 0)
    _rejected(lib, hrir.hrir_stream_admit, CTX, 1, 1, fc((10,)), 0)


# ---- filter production and the precomputed-resonance views ---------------------------------
def test_sparsify_and_views_valid(lib, monkeypatch):
    monkeypatch.setitem(hrir._REFL_LEN, CTX, 200)
    X, f = fc((1250, 2, 231)), fc((2, 32))
    G, nnz = hrir.hrir_sparsify(CTX, X, f, 200, 1e-3, 60.0, 1e-4, stream=0)
    a = last(lib, "hrir_sparsify")
    assert a[1:5] == (1250, 2, 231, 200) and tuple(G.shape) == (1250, 2, 200)
    assert tuple(nnz.shape) == (1250, 2)
    S, Lu = 37, 20042
    u = fc((S, 2, 20044))
    out = hrir.hrir_render_precomputed(CTX, u, fc((3, S), torch.int32), length=Lu, stream=0)
    a = last(lib, "hrir_render_precomputed")
    assert a[1:4] == (S, Lu, 20044) and a[5] == 3 and tuple(out.shape) == (3, 2, Lu + 199)
    assert a[9] == out.stride(1) and a[10] == out.stride(0)


def test_sparsify_and_views_reject(lib, monkeypatch):
    monkeypatch.setitem(hrir._REFL_LEN, CTX, 200)
    sp = lambda *a, **k: _rejected(lib, hrir.hrir_sparsify, CTX, *a, stream=0, **k)  # noqa: E731
    sp(torch.zeros((10, 2, 231)), fc((2, 32)), 200, 1e-3)            # host HRIRs
    sp(fc((10, 3, 231)), fc((3, 32)), 200, 1e-3)                     # three ears
    sp(fc((10, 2, 231)), fc((2, 31)), 200, 1e-3)                     # resonance length
    sp(fc((10, 2, 231)), fc((2, 32)), 240, 1e-3)                     # Lg > M
    sp(fc((10, 2, 231)), fc((2, 32)), 200, 1e-3, G=fc((10, 2, 199)))  # output rows
    sp(fc((10, 2, 231)), fc((2, 32)), 200, 1e-3, nnz=fc((10, 2), torch.int64))
    S = 5
    v = lambda *a, **k: _rejected(lib, hrir.hrir_render_precomputed, CTX, *a, stream=0, **k)  # noqa: E731
    v(fc((S, 1, 1000)), fc((2, S), torch.int32))                     # one ear
    v(fc((S, 2, 1000)), fc((2, S + 1), torch.int32))                 # directions per view
    v(fc((S, 2, 1000)), fc((2, S), torch.int64))                     # direction dtype
    v(fc((S, 2, 1000)), fc((2, S), torch.int32), length=1001)        # longer than u
    v(fc((S, 2, 1000)), fc((2, S), torch.int32), out=fc((2, 2, 1198)))  # output too short
    v(FakeCuda(torch.zeros((2, S, 1000)).transpose(0, 1)), fc((2, S), torch.int32))  # ears apart


def test_sharding_calls_valid(lib, monkeypatch):
    monkeypatch.setitem(hrir._REFL_LEN, CTX, 200)
    S, L, ld = 37, 30001, 30008
    z = hrir.hrir_render_reflections(CTX, fc((S, ld)), fc((S,), torch.int32), length=L, stream=0)
    a = last(lib, "hrir_render_reflections")
    assert a[1:4] == (S, L, ld) and a[7] == 1 and tuple(z.shape) == (2, L + 199)
    z0 = hrir.hrir_render_reflections(CTX, fc((S, ld)), fc((S,), torch.int32), full=False, length=L,
                                      stream=0)
    assert tuple(z0.shape) == (2, L)
    parts = fc((3, 2, L + 199))
    out = hrir.hrir_apply_resonance(CTX, parts, stream=0)
    a = last(lib, "hrir_apply_resonance")
    assert a[1:4] == (3, L + 199, L + 199) and tuple(out.shape) == (2, L + 199 + 31)
    out = hrir.hrir_apply_resonance(CTX, fc((2, L + 199)), full=False, stream=0)   # one part
    a = last(lib, "hrir_apply_resonance")
    assert a[1] == 1 and tuple(out.shape) == (2, L + 199)


def test_sharding_calls_reject(lib, monkeypatch):
    monkeypatch.setitem(hrir._REFL_LEN, CTX, 200)
    r = lambda *a, **k: _rejected(lib, hrir.hrir_render_reflections, CTX, *a, stream=0, **k)  # noqa: E731
    r(torch.zeros((4, 1000)), fc((4,), torch.int32))                  # host sources
    r(fc((4, 1000)), fc((3,), torch.int32))                           # too few directions
    r(fc((4, 1000)), fc((4,), torch.int32), z=fc((2, 1198)))          # z too short
    ap = lambda *a, **k: _rejected(lib, hrir.hrir_apply_resonance, CTX, *a, stream=0, **k)  # noqa: E731
    ap(torch.zeros((2, 2, 100)))                                      # host parts
    ap(fc((2, 3, 100)))                                               # three ears
    ap(fc((2, 2, 100)), length=101)                                   # longer than the parts
    ap(fc((2, 2, 100)), out=fc((2, 130)))                             # output too short
    ap(FakeCuda(torch.zeros((2, 2, 100)).transpose(0, 1)))            # ears not adjacent


def test_factorize_valid_and_reject(lib):
    X, G = fc((1250, 2, 231)), fc((1250, 2, 200))
    f, tr = hrir.hrir_factorize(CTX, X, G, 200, iters=50, stream=0)
    a = last(lib, "hrir_factorize")
    assert a[1:5] == (1250, 2, 231, 200) and a[9:11] == (50, 1)
    assert tuple(f.shape) == (2, 32) and tuple(tr.shape) == (2, 51)
    fa = lambda *a, **k: _rejected(lib, hrir.hrir_factorize, CTX, *a, stream=0, **k)  # noqa: E731
    fa(torch.zeros((10, 2, 231)), fc((10, 2, 200)), 200)             # host HRIRs
    fa(fc((10, 2, 231)), fc((10, 2, 199)), 200)                      # G rows
    fa(fc((10, 2, 231)), fc((10, 2, 200)), 240)                      # Lg > M
    fa(fc((10, 2, 231)), fc((10, 2, 200)), 200, iters=0)             # no rounds
    fa(fc((10, 2, 231)), fc((10, 2, 200)), 200, f=fc((2, 31)))       # resonance length
    fa(fc((10, 2, 231)), fc((10, 2, 200)), 200, iters=5, trace=fc((2, 5)))   # trace length
