"""Thin ctypes binding of the C ABI in include/hrir.h (argument marshalling only).

Every function named ``hrir_*`` here calls the C function of the same name in
``_lib/libhrir.so``; all rendering work runs in that library's CUDA kernels.  There is no
CPU fallback: importing this module on a machine without the built library, or calling it
without a CUDA device, raises.

Tensors are torch tensors (device memory and streams only); pointers are passed through
``data_ptr()`` and streams through ``torch.cuda.Stream.cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhrir.so")

HRIR_OK, HRIR_EINVAL, HRIR_ENOMEM, HRIR_ECUDA, HRIR_ETIMEDOUT, HRIR_EBUSY, HRIR_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
HRIR_F32, HRIR_BF16, HRIR_F16 = 0, 1, 2
HRIR_SPARSE, HRIR_DENSE, HRIR_FFT = 0, 1, 2
MODES = {"sparse": HRIR_SPARSE, "dense": HRIR_DENSE, "fft": HRIR_FFT}
STATUS_NAMES = {0: "HRIR_OK", -1: "HRIR_EINVAL", -2: "HRIR_ENOMEM", -3: "HRIR_ECUDA",
                -4: "HRIR_ETIMEDOUT", -5: "HRIR_EBUSY", -6: "HRIR_ESTATE"}

# every symbol the header declares, with its ctypes signature
_vp, _i, _i64, _cp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_char_p
SIGNATURES = {
    "hrir_version": ([], _i),
    "hrir_create": ([ctypes.POINTER(_vp), _i], _i),
    "hrir_destroy": ([_vp], None),
    "hrir_last_error": ([_vp], _cp),
    "hrir_sync": ([_vp, _vp], _i),
    "hrir_selftest_wait_timeout": ([_vp, _vp], _i),
    "hrir_topk_pack": ([_vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "hrir_load_filters": ([_vp, _i, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _i], _i),
    "hrir_out_len": ([_vp, _i64, _i], _i64),
    "hrir_render_batch": ([_vp, _i, _i64, _i64, _i, _vp, _vp, _i, _i, _vp, _i64, _vp], _i),
    "hrir_render_batch_host": ([_vp, _i, _i64, _i64, _i, _vp, _vp, _i, _i, _vp, _i64, _vp], _i),
    "hrir_render_batch_noalloc": ([_vp, _i, _i64, _i64, _i, _vp, _vp, _i, _i, _vp, _i64, _vp], _i),
    "hrir_stream_open": ([_vp, _i, _i, ctypes.c_size_t, _vp], _i),
    "hrir_stream_admit": ([_vp, _i64, _i64, _vp, _i64, _i], _i),
    "hrir_stream_step": ([_vp, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)),
                          ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                          ctypes.POINTER(ctypes.c_int), _vp, ctypes.POINTER(ctypes.c_int)], _i),
    "hrir_stream_stats": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int64)], _i),
    "hrir_stream_close": ([_vp], _i),
    "hrir_mlp_param_count": ([_i], _i64),
    "hrir_mlp_act_stride": ([_i], _i64),
    "hrir_mlp_forward": ([_vp, _i64, _vp, _i, _vp, _vp, _vp, _vp], _i),
    "hrir_mlp_forward_bf16": ([_vp, _i64, _vp, _i, _vp, _vp, _vp], _i),
    "hrir_mlp_backward": ([_vp, _i64, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "hrir_mlp_adam": ([_vp, _i64, _vp, _vp, _vp, _vp, _i, ctypes.c_float, ctypes.c_float,
                       ctypes.c_float, ctypes.c_float, _vp], _i),
    "hrir_render_moving": ([_vp, _i, _i64, _i64, _vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _i64,
                            _vp], _i),
    "hrir_resonance_per_source": ([_vp, _i, _i64, _i64, _i, _vp, _i, _vp, _i64, _vp], _i),
    "hrir_factorize": ([_vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "hrir_sparsify": ([_vp, _i, _i, _i, _i, _vp, _vp, ctypes.c_float, ctypes.c_float,
                       ctypes.c_float, _vp, _vp, _vp], _i),
    "hrir_render_precomputed": ([_vp, _i, _i64, _i64, _vp, _i, _vp, _i, _vp, _i64, _i64, _vp], _i),
    "hrir_render_reflections": ([_vp, _i, _i64, _i64, _i, _vp, _vp, _i, _vp, _i64, _vp], _i),
    "hrir_apply_resonance": ([_vp, _i, _i64, _i64, _vp, _i, _vp, _i64, _vp], _i),
    "hrir_set_timing": ([_vp, _i], _i),
    "hrir_kernel_times": ([_vp, _vp, _vp, _i], _i),
}
HRIR_K_COUNT = 9
KERNEL_NAMES = {0: "mix_sparse", 1: "mix_dense", 2: "reduce_fir", 3: "fft", 4: "tables",
                5: "mlp", 6: "mix_moving", 7: "resonance_gemm", 8: "filters"}

_lib = None
_lock = threading.Lock()


class HRIRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhrir.so (built by paper_1502_03162_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is not built; run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(ctx, rc: int):
    if rc != HRIR_OK:
        msg = load_library().hrir_last_error(ctx)
        raise HRIRError(rc, msg.decode() if msg else "")


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dtype_code(t) -> int:
    import torch
    codes = {torch.float32: HRIR_F32, torch.bfloat16: HRIR_BF16, torch.float16: HRIR_F16}
    _require(t.dtype in codes, f"source dtype {t.dtype}: expected float32, bfloat16 or float16")
    return codes[t.dtype]


# ---------------------------------------------------------------------------------------
# argument checks: the C ABI receives raw pointers and sizes, so every extent a kernel will
# read or write is checked here against the tensor that backs it (ValueError otherwise)
# ---------------------------------------------------------------------------------------
def _require(cond, msg: str) -> None:
    if not cond:
        raise ValueError(msg)


def _check_tensor(t, name: str, *, cuda: bool, dtypes, dim=None, shape=None, min_shape=None,
                  numel=None, contiguous=False, unit_stride=False) -> None:
    """t must be a tensor on the stated side (CUDA or host) with one of `dtypes`; optional
    exact rank, exact or minimum shape, exact element count, contiguity, and unit stride in
    its last dimension (empty tensors pass the layout checks)."""
    _require(t is not None and hasattr(t, "data_ptr") and hasattr(t, "dtype"),
             f"{name}: expected a torch tensor")
    _require(bool(t.is_cuda) == cuda, f"{name}: expected a {'CUDA' if cuda else 'host (CPU)'} tensor")
    _require(t.dtype in dtypes, f"{name}: dtype {t.dtype}, expected one of {list(dtypes)}")
    if dim is not None:
        _require(t.dim() == dim, f"{name}: {t.dim()} dimensions, expected {dim}")
    if shape is not None:
        _require(tuple(t.shape) == tuple(shape), f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if min_shape is not None:
        _require(t.dim() == len(min_shape) and all(a >= b for a, b in zip(t.shape, min_shape)),
                 f"{name}: shape {tuple(t.shape)}, expected at least {tuple(min_shape)}")
    if numel is not None:
        _require(t.numel() == numel, f"{name}: {t.numel()} elements, expected {numel}")
    if contiguous:
        _require(t.numel() == 0 or t.is_contiguous(), f"{name}: expected a contiguous tensor")
    if unit_stride:
        _require(t.numel() == 0 or t.stride(-1) == 1, f"{name}: last dimension must have stride 1")


def _src_dtypes():
    import torch
    return (torch.float32, torch.bfloat16, torch.float16)


def _index_dtypes():
    """Tap index tensors: int16 holding the uint16 indices (all < 2048), or uint16."""
    import torch
    return tuple(t for t in (torch.int16, getattr(torch, "uint16", None)) if t is not None)


def _src_extent(src, length):
    """(S, ld, L) of a [S][ld] source batch rendered over its first L samples."""
    S = src.shape[0]
    ld = src.stride(0) if S > 1 else src.shape[1]
    L = src.shape[1] if length is None else int(length)
    _require(0 <= L <= src.shape[1], f"length {L} outside the source rows' {src.shape[1]} samples")
    return S, ld, L


# ---------------------------------------------------------------------------------------
# same-name wrappers
# ---------------------------------------------------------------------------------------
def hrir_version() -> int:
    return load_library().hrir_version()


def hrir_create(device: int = 0) -> int:
    lib = load_library()
    h = _vp()
    rc = lib.hrir_create(ctypes.byref(h), device)
    if rc != HRIR_OK:
        raise HRIRError(rc, lib.hrir_last_error(None).decode())
    return h.value


def hrir_destroy(ctx) -> None:
    load_library().hrir_destroy(ctx)


def hrir_last_error(ctx) -> str:
    return load_library().hrir_last_error(ctx).decode()


def hrir_sync(ctx, stream=None) -> int:
    """Returns the status (does not raise) so callers can test device-side flags."""
    return load_library().hrir_sync(ctx, _stream_handle(stream))


def hrir_selftest_wait_timeout(ctx, stream=None) -> int:
    """Enqueue the failure-path self-test (a bounded device wait that expires after 1 s); the
    next hrir_sync returns HRIR_ETIMEDOUT."""
    return load_library().hrir_selftest_wait_timeout(ctx, _stream_handle(stream))


def hrir_topk_pack(ctx, g, k: int, idx=None, w=None, nnz=None, stream=None):
    """g: CUDA float32 [..., refl_len].  Returns (idx, w, nnz) CUDA tensors: idx is int16
    holding the uint16 indices (all < 2048, so the values read the same), w float32, nnz
    uint8."""
    import torch
    _check_tensor(g, "g", cuda=True, dtypes=(torch.float32,), contiguous=True)
    _require(g.dim() >= 1 and int(k) >= 0, "g needs a last (filter) dimension and k >= 0")
    refl_len = g.shape[-1]
    lead = tuple(g.shape[:-1])
    rows = int(np.prod(lead)) if lead else 1
    if idx is None:
        idx = torch.empty(lead + (k,), dtype=torch.int16, device=g.device)   # uint16 payload
    _check_tensor(idx, "idx", cuda=True, dtypes=_index_dtypes(), numel=rows * k, contiguous=True)
    if w is None:
        w = torch.empty(lead + (k,), dtype=torch.float32, device=g.device)
    _check_tensor(w, "w", cuda=True, dtypes=(torch.float32,), numel=rows * k, contiguous=True)
    if nnz is None:
        nnz = torch.empty(lead, dtype=torch.uint8, device=g.device)
    _check_tensor(nnz, "nnz", cuda=True, dtypes=(torch.uint8,), numel=rows, contiguous=True)
    rc = load_library().hrir_topk_pack(ctx, rows, refl_len, k, g.data_ptr(), idx.data_ptr(),
                                       w.data_ptr(), nnz.data_ptr(), _stream_handle(stream))
    _check(ctx, rc)
    return idx, w, nnz


def hrir_load_filters(ctx, tap_idx, tap_w, tap_nnz, refl_len: int, res, fft_size: int = 0):
    """Host numpy arrays: tap_idx uint16 [n_dirs][2][k_max], tap_w float32, tap_nnz uint8
    [n_dirs][2], res float32 [2][Lf]."""
    raw = np.asarray(tap_idx)
    _require(raw.ndim == 3, f"tap_idx: shape {raw.shape}, expected [n_dirs][n_ears][k_max]")
    if raw.dtype != np.uint16 and raw.size:
        _require(np.issubdtype(raw.dtype, np.integer) and raw.min() >= 0 and raw.max() <= 0xFFFF,
                 "tap_idx: indices must be integers in [0, 65535]")
    tap_idx = np.ascontiguousarray(raw, dtype=np.uint16)
    tap_w = np.ascontiguousarray(tap_w, dtype=np.float32)
    tap_nnz = np.ascontiguousarray(tap_nnz, dtype=np.uint8)
    res = np.ascontiguousarray(res, dtype=np.float32)
    n_dirs, n_ears, k_max = tap_idx.shape
    _require(tap_w.shape == tap_idx.shape, f"tap_w: shape {tap_w.shape}, expected {tap_idx.shape}")
    _require(tap_nnz.shape == (n_dirs, n_ears), f"tap_nnz: shape {tap_nnz.shape}, expected {(n_dirs, n_ears)}")
    _require(res.ndim == 2 and res.shape[0] == n_ears, f"res: shape {res.shape}, expected [{n_ears}][Lf]")
    rc = load_library().hrir_load_filters(
        ctx, n_dirs, n_ears, refl_len, k_max, tap_idx.ctypes.data, tap_w.ctypes.data,
        tap_nnz.ctypes.data, res.shape[1], res.ctypes.data, fft_size)
    _check(ctx, rc)
    _RES_LEN[ctx] = res.shape[1]
    _REFL_LEN[ctx] = int(refl_len)


def hrir_out_len(ctx, length: int, full: bool = True) -> int:
    return load_library().hrir_out_len(ctx, length, int(full))


def hrir_render_batch(ctx, src, dirs, mode="sparse", full=True, length=None, out=None,
                      stream=None):
    """src: CUDA [S][ld] float32/bfloat16/float16; dirs: CUDA int32 [S].
    Returns out: CUDA float32 [2][out_len] (or the given buffer)."""
    import torch
    _check_tensor(src, "src", cuda=True, dtypes=_src_dtypes(), dim=2, unit_stride=True)
    S, ld, L = _src_extent(src, length)
    _check_tensor(dirs, "dirs", cuda=True, dtypes=(torch.int32,), contiguous=True)
    _require(dirs.numel() >= S, f"dirs: {dirs.numel()} entries for {S} sources")
    out_len = hrir_out_len(ctx, L, full)
    if out is None:
        out = torch.empty((2, max(out_len, 1)), dtype=torch.float32, device=src.device)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(2, out_len),
                  unit_stride=True)
    rc = load_library().hrir_render_batch(
        ctx, S, L, ld, _dtype_code(src), src.data_ptr(), dirs.data_ptr(),
        MODES[mode] if isinstance(mode, str) else int(mode), int(full), out.data_ptr(),
        out.stride(0), _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :out_len]


def hrir_render_batch_host(ctx, src, dirs, mode="sparse", full=True, length=None, out=None,
                           stream=None):
    """src: CPU tensor [S][ld] (pinned for speed); dirs: CPU int32 [S].  Synchronous; returns
    a CPU float32 [2][out_len] tensor."""
    import torch
    _check_tensor(src, "src", cuda=False, dtypes=_src_dtypes(), dim=2, unit_stride=True)
    S, ld, L = _src_extent(src, length)
    _check_tensor(dirs, "dirs", cuda=False, dtypes=(torch.int32,))
    dirs = dirs.contiguous()
    _require(dirs.numel() >= S, f"dirs: {dirs.numel()} entries for {S} sources")
    out_len = hrir_out_len(ctx, L, full)
    if out is None:
        out = torch.empty((2, max(out_len, 1)), dtype=torch.float32,
                          pin_memory=src.is_pinned())
    _check_tensor(out, "out", cuda=False, dtypes=(torch.float32,), min_shape=(2, out_len),
                  unit_stride=True)
    rc = load_library().hrir_render_batch_host(
        ctx, S, L, ld, _dtype_code(src), src.data_ptr(), dirs.data_ptr(),
        MODES[mode] if isinstance(mode, str) else int(mode), int(full), out.data_ptr(),
        out.stride(0), _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :out_len]


def hrir_render_batch_noalloc(ctx, src, dirs, out, mode="sparse", full=True, length=None,
                              stream=None):
    """The allocation-free variant of hrir_render_batch: the caller passes every buffer,
    including `out` (CUDA float32 [2][>= out_len]); the library uses its fixed 32 MiB device
    scratch array and allocates nothing.  Returns out[:, :out_len]."""
    import torch
    _check_tensor(src, "src", cuda=True, dtypes=_src_dtypes(), dim=2, unit_stride=True)
    S, ld, L = _src_extent(src, length)
    _check_tensor(dirs, "dirs", cuda=True, dtypes=(torch.int32,), contiguous=True)
    _require(dirs.numel() >= S, f"dirs: {dirs.numel()} entries for {S} sources")
    out_len = hrir_out_len(ctx, L, full)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(2, out_len),
                  unit_stride=True)
    rc = load_library().hrir_render_batch_noalloc(
        ctx, S, L, ld, _dtype_code(src), src.data_ptr(), dirs.data_ptr(),
        MODES[mode] if isinstance(mode, str) else int(mode), int(full), out.data_ptr(),
        out.stride(0), _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :out_len]


def hrir_stream_open(ctx, block: int, max_slots: int, pool_bytes: int, stream=None) -> None:
    _check(ctx, load_library().hrir_stream_open(ctx, block, max_slots, pool_bytes,
                                                _stream_handle(stream)))


def hrir_stream_admit(ctx, req_id: int, session: int, src, direction: int) -> int:
    """src: host float32 samples (numpy array or CPU tensor; must stay alive until the
    source's upload has landed -- page-locked buffers are read asynchronously).  Returns the
    status: HRIR_OK, or HRIR_EBUSY / HRIR_ENOMEM when the request was not admitted now.
    Other errors raise."""
    if hasattr(src, "data_ptr"):
        import torch
        _check_tensor(src, "src", cuda=False, dtypes=(torch.float32,), contiguous=True)
        ptr, n = src.data_ptr(), src.numel()
    else:
        _require(isinstance(src, np.ndarray) and src.dtype == np.float32 and src.flags.c_contiguous,
                 "src: expected a contiguous float32 numpy array or CPU tensor")
        ptr, n = src.ctypes.data, src.size
    rc = load_library().hrir_stream_admit(ctx, int(req_id), int(session), ptr, int(n),
                                          int(direction))
    if rc not in (HRIR_OK, HRIR_EBUSY, HRIR_ENOMEM):
        _check(ctx, rc)
    return rc


class _StepBuffers:
    def __init__(self, max_slots):
        self.done = (ctypes.c_int64 * max_slots)()
        self.out = ctypes.POINTER(ctypes.c_float)()
        self.sess = ctypes.POINTER(ctypes.c_int64)()
        self.n_out = ctypes.c_int()
        self.n_done = ctypes.c_int()


def hrir_stream_step(ctx, bufs: "_StepBuffers", block: int):
    """One step.  Returns (blocks, sessions, done): blocks is a float32 view [n][2][block] of
    the library's output buffer (valid until the next step), sessions an int64 array [n] (the
    session of each block row), done a list of the finished request ids."""
    lib = load_library()
    rc = lib.hrir_stream_step(ctx, ctypes.byref(bufs.out), ctypes.byref(bufs.sess),
                              ctypes.byref(bufs.n_out), bufs.done, ctypes.byref(bufs.n_done))
    _check(ctx, rc)
    n = bufs.n_out.value
    if n:
        blocks = np.ctypeslib.as_array(bufs.out, shape=(n, 2, block))
        sessions = np.ctypeslib.as_array(bufs.sess, shape=(n,)).copy()
    else:
        blocks, sessions = np.zeros((0, 2, block), np.float32), np.zeros(0, np.int64)
    return blocks, sessions, list(bufs.done[:bufs.n_done.value])


def hrir_stream_stats(ctx):
    a, p, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(ctx, load_library().hrir_stream_stats(ctx, ctypes.byref(a), ctypes.byref(p),
                                                 ctypes.byref(u)))
    return a.value, p.value, u.value


def hrir_stream_close(ctx) -> None:
    _check(ctx, load_library().hrir_stream_close(ctx))


class Stream:
    """Block stream on a Renderer (continuous batching of sources into sessions)."""

    def __init__(self, renderer: "Renderer", block: int, max_slots: int, pool_bytes: int,
                 stream=None):
        self.r = renderer
        self.block = block
        self.max_slots = max_slots
        hrir_stream_open(renderer.ctx, block, max_slots, pool_bytes, stream)
        self.bufs = _StepBuffers(max_slots)

    def admit(self, req_id, session, src, direction) -> int:
        return hrir_stream_admit(self.r.ctx, req_id, session, src, direction)

    def step(self):
        return hrir_stream_step(self.r.ctx, self.bufs, self.block)

    def stats(self):
        return hrir_stream_stats(self.r.ctx)

    def close(self):
        hrir_stream_close(self.r.ctx)


def hrir_mlp_param_count(refl_len: int) -> int:
    return load_library().hrir_mlp_param_count(refl_len)


def hrir_mlp_act_stride(refl_len: int) -> int:
    return load_library().hrir_mlp_act_stride(refl_len)


def _f32_cuda(t, shape=None, name="tensor"):
    import torch
    _check_tensor(t, name, cuda=True, dtypes=(torch.float32,), shape=shape, contiguous=True)
    return t.data_ptr()


def hrir_mlp_forward(ctx, dirs, params, refl_len: int, out=None, acts=None, stream=None):
    """dirs: CUDA float32 [n][3] (az, el, ear = -1/+1); params: CUDA float32 [param_count].
    Returns out [n][refl_len] (and fills acts [n][act_stride] when given)."""
    import torch
    n = dirs.shape[0]
    if out is None:
        out = torch.empty((n, refl_len), dtype=torch.float32, device=dirs.device)
    rc = load_library().hrir_mlp_forward(
        ctx, n, _f32_cuda(dirs, (n, 3)), refl_len,
        _f32_cuda(params, (hrir_mlp_param_count(refl_len),)), _f32_cuda(out, (n, refl_len)),
        _f32_cuda(acts, (n, hrir_mlp_act_stride(refl_len))) if acts is not None else None,
        _stream_handle(stream))
    _check(ctx, rc)
    return out


def hrir_mlp_forward_bf16(ctx, dirs, params, refl_len: int, out=None, stream=None):
    """Tensor-core (BF16) inference of the network: returns out [n][refl_len] (CUDA)."""
    import torch
    n = dirs.shape[0]
    if out is None:
        out = torch.empty((n, refl_len), dtype=torch.float32, device=dirs.device)
    rc = load_library().hrir_mlp_forward_bf16(
        ctx, n, _f32_cuda(dirs, (n, 3)), refl_len,
        _f32_cuda(params, (hrir_mlp_param_count(refl_len),)), _f32_cuda(out, (n, refl_len)),
        _stream_handle(stream))
    _check(ctx, rc)
    return out


def hrir_mlp_backward(ctx, dirs, params, acts, out, target, refl_len: int, grads=None,
                      loss=None, stream=None):
    """Gradient of L = 1/(2n) sum ||out - target||^2; returns (grads, loss) CUDA tensors."""
    import torch
    n = dirs.shape[0]
    P = hrir_mlp_param_count(refl_len)
    if grads is None:
        grads = torch.empty(P, dtype=torch.float32, device=dirs.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=dirs.device)
    rc = load_library().hrir_mlp_backward(
        ctx, n, _f32_cuda(dirs, (n, 3)), refl_len, _f32_cuda(params, (P,)),
        _f32_cuda(acts, (n, hrir_mlp_act_stride(refl_len))), _f32_cuda(out, (n, refl_len)),
        _f32_cuda(target, (n, refl_len)), _f32_cuda(grads, (P,)), _f32_cuda(loss),
        _stream_handle(stream))
    _check(ctx, rc)
    return grads, loss


def hrir_mlp_adam(ctx, params, grads, m, v, step: int, lr: float, beta1=0.9, beta2=0.999,
                  eps=1e-8, stream=None) -> None:
    n = params.numel()
    rc = load_library().hrir_mlp_adam(ctx, n, _f32_cuda(params), _f32_cuda(grads, (n,)),
                                      _f32_cuda(m, (n,)), _f32_cuda(v, (n,)), int(step),
                                      float(lr), float(beta1), float(beta2), float(eps),
                                      _stream_handle(stream))
    _check(ctx, rc)


def hrir_render_moving(ctx, src, tap_idx, tap_w, tap_nnz, seg_len: int, full=True, length=None,
                       out=None, stream=None):
    """src: CUDA float32 [S][ld]; tap tables CUDA [S][n_seg][2][k] (idx int16 holding uint16,
    w float32) and nnz uint8 [S][n_seg][2].  Returns out CUDA float32 [2][out_len]."""
    import torch
    _check_tensor(src, "src", cuda=True, dtypes=(torch.float32,), dim=2, unit_stride=True)
    S, ld, L = _src_extent(src, length)
    _check_tensor(tap_idx, "tap_idx", cuda=True, dtypes=_index_dtypes(), dim=4, contiguous=True)
    n_seg, k = tap_idx.shape[1], tap_idx.shape[3]
    _check_tensor(tap_idx, "tap_idx", cuda=True, dtypes=_index_dtypes(), shape=(S, n_seg, 2, k))
    _check_tensor(tap_w, "tap_w", cuda=True, dtypes=(torch.float32,), shape=(S, n_seg, 2, k),
                  contiguous=True)
    _check_tensor(tap_nnz, "tap_nnz", cuda=True, dtypes=(torch.uint8,), shape=(S, n_seg, 2),
                  contiguous=True)
    out_len = hrir_out_len(ctx, L, full)
    if out is None:
        out = torch.empty((2, max(out_len, 1)), dtype=torch.float32, device=src.device)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(2, out_len),
                  unit_stride=True)
    rc = load_library().hrir_render_moving(
        ctx, S, L, ld, src.data_ptr(), n_seg, int(seg_len), k, tap_idx.data_ptr(),
        tap_w.data_ptr(), tap_nnz.data_ptr(), int(full), out.data_ptr(), out.stride(0),
        _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :out_len]


def hrir_resonance_per_source(ctx, src, full=True, length=None, out=None, stream=None):
    """src: CUDA bfloat16/float16 [S][ld].  Returns u: CUDA float32 [S][2][out_len] with
    u[s, e] = y_s * f_e (the loaded resonance), computed on the tensor cores."""
    import torch
    _check_tensor(src, "src", cuda=True, dtypes=(torch.bfloat16, torch.float16), dim=2,
                  unit_stride=True)
    S, ld, L = _src_extent(src, length)
    res_len = _res_len(ctx)
    out_len = (L + res_len - 1 if L > 0 else 0) if full else L
    if out is None:
        out = torch.empty((S, 2, max((out_len + 3) // 4 * 4, 4)), dtype=torch.float32,
                          device=src.device)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(S, 2, out_len),
                  unit_stride=True)
    _require(out.numel() == 0 or out.stride(0) == 2 * out.stride(1),
             "out: the two ears of a source must be adjacent rows ([S][2][len] layout)")
    rc = load_library().hrir_resonance_per_source(ctx, S, L, ld, _dtype_code(src), src.data_ptr(),
                                                  int(full), out.data_ptr(), out.stride(1),
                                                  _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :, :out_len]


def _filter_rows(X, name="X"):
    """(n_dirs, n_ears, M) of a CUDA float32 [n_dirs][n_ears][M] HRIR array."""
    import torch
    _check_tensor(X, name, cuda=True, dtypes=(torch.float32,), dim=3, contiguous=True)
    _require(1 <= X.shape[1] <= 2, f"{name}: {X.shape[1]} ears, expected 1 or 2")
    return X.shape[0], X.shape[1], X.shape[2]


def hrir_factorize(ctx, X, G, refl_len: int, iters: int = 50, normalise: bool = True, f=None,
                   trace=None, stream=None):
    """Algorithm 1 on the device.  X: CUDA float32 [n_dirs][n_ears][M]; G: CUDA float32
    [n_dirs][n_ears][Lg], the non-negative start, overwritten with the result.  Returns
    (f [n_ears][Lf], trace [n_ears][iters + 1]) CUDA tensors."""
    import torch
    n_dirs, n_ears, M = _filter_rows(X)
    Lf = M - int(refl_len) + 1
    _require(Lf >= 1, f"refl_len {refl_len} longer than the HRIRs ({M})")
    _require(int(iters) >= 1, f"iters {iters} < 1")
    _check_tensor(G, "G", cuda=True, dtypes=(torch.float32,), shape=(n_dirs, n_ears, refl_len),
                  contiguous=True)
    if f is None:
        f = torch.empty((n_ears, Lf), dtype=torch.float32, device=X.device)
    _check_tensor(f, "f", cuda=True, dtypes=(torch.float32,), shape=(n_ears, Lf), contiguous=True)
    if trace is None:
        trace = torch.empty((n_ears, int(iters) + 1), dtype=torch.float32, device=X.device)
    _check_tensor(trace, "trace", cuda=True, dtypes=(torch.float32,), shape=(n_ears, int(iters) + 1),
                  contiguous=True)
    rc = load_library().hrir_factorize(ctx, n_dirs, n_ears, M, int(refl_len), X.data_ptr(),
                                       G.data_ptr(), f.data_ptr(), trace.data_ptr(), int(iters),
                                       int(normalise), _stream_handle(stream))
    _check(ctx, rc)
    return f, trace


def hrir_sparsify(ctx, X, f, refl_len: int, lam: float, sigma: float = 0.0, thresh: float = 1e-4,
                  G=None, nnz=None, stream=None):
    """Eq. 14 per (direction, ear) with f fixed, D = I (sigma <= 0) or D_W(sigma); entries
    <= thresh dropped.  Returns (G [n_dirs][n_ears][Lg], nnz int32 [n_dirs][n_ears])."""
    import torch
    n_dirs, n_ears, M = _filter_rows(X)
    Lf = M - int(refl_len) + 1
    _require(Lf >= 1, f"refl_len {refl_len} longer than the HRIRs ({M})")
    _check_tensor(f, "f", cuda=True, dtypes=(torch.float32,), shape=(n_ears, Lf), contiguous=True)
    if G is None:
        G = torch.empty((n_dirs, n_ears, int(refl_len)), dtype=torch.float32, device=X.device)
    _check_tensor(G, "G", cuda=True, dtypes=(torch.float32,), shape=(n_dirs, n_ears, refl_len),
                  contiguous=True)
    if nnz is None:
        nnz = torch.empty((n_dirs, n_ears), dtype=torch.int32, device=X.device)
    _check_tensor(nnz, "nnz", cuda=True, dtypes=(torch.int32,), shape=(n_dirs, n_ears),
                  contiguous=True)
    rc = load_library().hrir_sparsify(ctx, n_dirs, n_ears, M, int(refl_len), X.data_ptr(),
                                      f.data_ptr(), float(lam), float(sigma), float(thresh),
                                      G.data_ptr(), nnz.data_ptr(), _stream_handle(stream))
    _check(ctx, rc)
    return G, nnz


def hrir_render_precomputed(ctx, u, dirs, full=True, length=None, out=None, stream=None):
    """u: CUDA float32 [S][2][u_ld] (u[s, e] = y_s * f_e, e.g. from hrir_resonance_per_source);
    dirs: CUDA int32 [n_views][S].  Returns out CUDA float32 [n_views][2][out_len]: each view
    mixes u through its directions' reflection taps (no resonance added)."""
    import torch
    _check_tensor(u, "u", cuda=True, dtypes=(torch.float32,), dim=3, unit_stride=True)
    S = u.shape[0]
    _require(u.shape[1] == 2, f"u: {u.shape[1]} ears, expected 2")
    _require(S == 0 or u.stride(0) == 2 * u.stride(1),
             "u: the two ears of a source must be adjacent rows ([S][2][len] layout)")
    u_ld = u.stride(1) if S else u.shape[2]
    L = u.shape[2] if length is None else int(length)
    _require(0 <= L <= u.shape[2], f"length {L} outside u's {u.shape[2]} samples")
    _check_tensor(dirs, "dirs", cuda=True, dtypes=(torch.int32,), dim=2, contiguous=True)
    _require(dirs.shape[1] == S, f"dirs: {dirs.shape[1]} sources per view, expected {S}")
    V = dirs.shape[0]
    out_len = (L + _refl_len(ctx) - 1 if L > 0 else 0) if full else L
    if out is None:
        out = torch.empty((V, 2, max(out_len, 1)), dtype=torch.float32, device=u.device)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(V, 2, out_len),
                  unit_stride=True)
    _require(V == 0 or out.stride(0) >= 2 * out.stride(1), "out: views overlap")
    rc = load_library().hrir_render_precomputed(
        ctx, S, L, u_ld, u.data_ptr(), V, dirs.data_ptr(), int(full), out.data_ptr(),
        out.stride(1) if V else max(out_len, 1), out.stride(0) if V else 2 * max(out_len, 1),
        _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :, :out_len]


def hrir_render_reflections(ctx, src, dirs, full=True, length=None, z=None, stream=None):
    """The reflection mix of a source set (sparse taps alone, no resonance).  src: CUDA
    [S][ld] float32/bfloat16/float16; dirs: CUDA int32 [S].  Returns z: CUDA float32
    [2][z_len] (or the given buffer), z_len = len + Lg - 1 (full) or len."""
    import torch
    _check_tensor(src, "src", cuda=True, dtypes=_src_dtypes(), dim=2, unit_stride=True)
    S, ld, L = _src_extent(src, length)
    _check_tensor(dirs, "dirs", cuda=True, dtypes=(torch.int32,), contiguous=True)
    _require(dirs.numel() >= S, f"dirs: {dirs.numel()} entries for {S} sources")
    z_len = (L + _refl_len(ctx) - 1 if L > 0 else 0) if full else L
    if z is None:
        z = torch.empty((2, max(z_len, 1)), dtype=torch.float32, device=src.device)
    _check_tensor(z, "z", cuda=True, dtypes=(torch.float32,), min_shape=(2, z_len), unit_stride=True)
    rc = load_library().hrir_render_reflections(
        ctx, S, L, ld, _dtype_code(src), src.data_ptr(), dirs.data_ptr(), int(full), z.data_ptr(),
        z.stride(0), _stream_handle(stream))
    _check(ctx, rc)
    return z[:, :z_len]


def hrir_apply_resonance(ctx, z, full=True, length=None, out=None, stream=None):
    """out_e = f_e * sum_c z[c, e] for z: CUDA float32 [n_parts][2][ld] (the reflection mixes of
    disjoint source sets, added in part order) or [2][ld] (one part); `length` samples of each
    (default: all).  Returns out: CUDA float32 [2][out_len], out_len = length + Lf - 1 (full)
    or length."""
    import torch
    _check_tensor(z, "z", cuda=True, dtypes=(torch.float32,), unit_stride=True)
    device = z.device
    if z.dim() == 2:
        z = z.unsqueeze(0)
    _require(z.dim() == 3 and z.shape[1] == 2, f"z: shape {tuple(z.shape)}, expected [n_parts][2][len]")
    P = z.shape[0]
    _require(P >= 1, "z: at least one part")
    _require(P == 1 or z.stride(0) == 2 * z.stride(1),
             "z: the parts must be [n_parts][2][ld] with the two ears adjacent")
    Lz = z.shape[2] if length is None else int(length)
    _require(0 <= Lz <= z.shape[2], f"length {Lz} outside z's {z.shape[2]} samples")
    out_len = (Lz + _res_len(ctx) - 1 if Lz > 0 else 0) if full else Lz
    if out is None:
        out = torch.empty((2, max(out_len, 1)), dtype=torch.float32, device=device)
    _check_tensor(out, "out", cuda=True, dtypes=(torch.float32,), min_shape=(2, out_len),
                  unit_stride=True)
    rc = load_library().hrir_apply_resonance(
        ctx, P, Lz, z.stride(1), z.data_ptr(), int(full), out.data_ptr(), out.stride(0),
        _stream_handle(stream))
    _check(ctx, rc)
    return out[:, :out_len]


_RES_LEN = {}
_REFL_LEN = {}


def _refl_len(ctx) -> int:
    return _REFL_LEN[ctx]


def _res_len(ctx) -> int:
    return _RES_LEN[ctx]


def hrir_set_timing(ctx, enable: bool) -> None:
    _check(ctx, load_library().hrir_set_timing(ctx, int(enable)))


def hrir_kernel_times(ctx, reset: bool = True):
    """{kernel family name: (milliseconds, launches)} accumulated since the last reset."""
    ms = (ctypes.c_double * HRIR_K_COUNT)()
    n = (ctypes.c_int64 * HRIR_K_COUNT)()
    _check(ctx, load_library().hrir_kernel_times(ctx, ms, n, int(reset)))
    return {KERNEL_NAMES.get(i, str(i)): (ms[i], n[i]) for i in range(HRIR_K_COUNT) if n[i]}


class Renderer:
    """Owns one hrir_ctx; convenience layer over the same-name functions above."""

    def __init__(self, device: int = 0):
        self.ctx = hrir_create(device)
        self.device = device

    def close(self):
        if self.ctx:
            hrir_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_filters(self, tap_idx, tap_w, tap_nnz, refl_len, res, fft_size=0):
        hrir_load_filters(self.ctx, tap_idx, tap_w, tap_nnz, refl_len, res, fft_size)

    def topk_pack(self, g, k, stream=None):
        return hrir_topk_pack(self.ctx, g, k, stream=stream)

    def render(self, src, dirs, mode="sparse", full=True, length=None, out=None, stream=None):
        return hrir_render_batch(self.ctx, src, dirs, mode, full, length, out, stream)

    def render_reflections(self, src, dirs, full=True, length=None, z=None, stream=None):
        return hrir_render_reflections(self.ctx, src, dirs, full, length, z, stream)

    def apply_resonance(self, z, full=True, length=None, out=None, stream=None):
        return hrir_apply_resonance(self.ctx, z, full, length, out, stream)

    def render_host(self, src, dirs, mode="sparse", full=True, length=None, out=None,
                    stream=None):
        return hrir_render_batch_host(self.ctx, src, dirs, mode, full, length, out, stream)

    def sync(self, stream=None) -> int:
        return hrir_sync(self.ctx, stream)

    def out_len(self, length, full=True):
        return hrir_out_len(self.ctx, length, full)

    def set_timing(self, enable=True):
        hrir_set_timing(self.ctx, enable)

    def kernel_times(self, reset=True):
        return hrir_kernel_times(self.ctx, reset)
