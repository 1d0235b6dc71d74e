"""The oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 CPU restatements of what the sparse factorized HRIR rendering path
computes (Luo, Zotkin & Duraiswami, "Sparse Head-Related Impulse Response for Efficient
Direct Convolution").  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  It shares no code with the CUDA library and never
imports it; the CUDA library never imports this package.

Contents
  * ``hrir_oracle.c`` (loaded through ctypes): direct convolution (Sec. I, footnote 2),
    sparse-filter convolution, the DFT and a radix-2 FFT, FFT convolution (footnote 3),
    the three binaural renderers of Eqs. 1-2 and top-K tap selection.
  * ``factorize.py``: the Toeplitz-constrained semi-NMF of Sec. III (Eqs. 3-13,
    Algorithm 1), the L1-NNLS sparsification (Eq. 14, Eq. 16) and the error metrics
    (Eq. 17).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrir_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U16 = ctypes.POINTER(ctypes.c_uint16)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile hrir_oracle.c with gcc into oracle/_build/liboracle.so (no CUDA involved)."""
    import platform
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stamp = os.path.join(_BUILD_DIR, "ARCH")
    same_arch = os.path.exists(stamp) and open(stamp).read() == platform.machine()
    stale = (not same_arch) or (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_conv_direct.argtypes = [_D, _i64, _D, _i64, _D]
            lib.orc_conv_direct.restype = None
            lib.orc_conv_sparse.argtypes = [_I32, _D, _int, _D, _i64, _i64, _D]
            lib.orc_conv_sparse.restype = None
            lib.orc_dft.argtypes = [_D, _D, _i64, _int, _D, _D]
            lib.orc_dft.restype = None
            lib.orc_fft.argtypes = [_D, _D, _i64, _int]
            lib.orc_fft.restype = _int
            lib.orc_conv_fft.argtypes = [_D, _i64, _D, _i64, _D]
            lib.orc_conv_fft.restype = _int
            render_args = [_int, _i64, _F, _i64, _I32, _int, _int, _U16, _F, _U8, _int, _int, _F]
            lib.orc_render_sparse.argtypes = render_args + [_int, _D, _i64]
            lib.orc_render_sparse.restype = _int
            lib.orc_render_dense.argtypes = render_args + [_D, _i64]
            lib.orc_render_dense.restype = _int
            lib.orc_render_fft.argtypes = render_args + [_D, _i64]
            lib.orc_render_fft.restype = _int
            lib.orc_render_sparse_at.argtypes = render_args + [ctypes.POINTER(ctypes.c_int64),
                                                               _i64, _D]
            lib.orc_render_sparse_at.restype = _int
            lib.orc_topk.argtypes = [_F, _int, _int, _int, _U16, _F, _U8]
            lib.orc_topk.restype = _int
            _lib = lib
    return _lib


def _p(a: np.ndarray, ptr):
    return a.ctypes.data_as(ptr)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------
# convolution primitives
# ---------------------------------------------------------------------------------------
def conv_direct(x, y) -> np.ndarray:
    """Direct convolution, Sec. I footnote 2 (0-based): out[n] = sum_j x[j] y[n-j]."""
    x, y = _f64(x), _f64(y)
    if x.size == 0 or y.size == 0:
        return np.zeros(0)
    out = np.empty(x.size + y.size - 1)
    _load().orc_conv_direct(_p(x, _D), x.size, _p(y, _D), y.size, _p(out, _D))
    return out


def conv_sparse(idx, w, y, refl_len: int) -> np.ndarray:
    """Convolution of y with the length-refl_len filter whose only non-zeros are w at idx."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    w, y = _f64(w), _f64(y)
    assert idx.shape == w.shape
    if y.size == 0:
        return np.zeros(0)
    out = np.empty(y.size + refl_len - 1)
    _load().orc_conv_sparse(_p(idx, _I32), _p(w, _D), idx.size, _p(y, _D), y.size, refl_len,
                            _p(out, _D))
    return out


def dft(x, inverse: bool = False) -> np.ndarray:
    """O(P^2) DFT by its definition (sign -1 forward, 1/P on the inverse)."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real), _f64(x.imag)
    ore, oim = np.empty_like(re), np.empty_like(im)
    _load().orc_dft(_p(re, _D), _p(im, _D), re.size, int(inverse), _p(ore, _D), _p(oim, _D))
    return ore + 1j * oim


def fft(x, inverse: bool = False) -> np.ndarray:
    """Radix-2 FFT (power-of-two length) with the same conventions as dft()."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.array(x.real, dtype=np.float64), np.array(x.imag, dtype=np.float64)
    rc = _load().orc_fft(_p(re, _D), _p(im, _D), re.size, int(inverse))
    if rc != 0:
        raise ValueError("fft length must be a power of two")
    return re + 1j * im


def conv_fft(x, y) -> np.ndarray:
    """FFT convolution, Sec. I footnote 3, on a power-of-two grid >= |x|+|y|-1."""
    x, y = _f64(x), _f64(y)
    if x.size == 0 or y.size == 0:
        return np.zeros(0)
    out = np.empty(x.size + y.size - 1)
    rc = _load().orc_conv_fft(_p(x, _D), x.size, _p(y, _D), y.size, _p(out, _D))
    if rc != 0:
        raise MemoryError("orc_conv_fft failed")
    return out


# ---------------------------------------------------------------------------------------
# binaural rendering (Eqs. 1-2)
# ---------------------------------------------------------------------------------------
def _render_common(y, dirs, tap_idx, tap_w, tap_nnz, res):
    y = np.asarray(y)
    if y.dtype != np.float32:
        raise TypeError("sources are FP32 (dequantise 16-bit sources before calling)")
    if y.ndim != 2:
        raise ValueError("y must be [S][ld]")
    dirs = np.ascontiguousarray(dirs, dtype=np.int32)
    tap_idx = np.ascontiguousarray(tap_idx, dtype=np.uint16)
    tap_w = np.ascontiguousarray(tap_w, dtype=np.float32)
    tap_nnz = np.ascontiguousarray(tap_nnz, dtype=np.uint8)
    res = np.ascontiguousarray(res, dtype=np.float32)
    n_dirs, n_ears, k_max = tap_idx.shape
    assert n_ears == 2 and tap_w.shape == tap_idx.shape and tap_nnz.shape == (n_dirs, 2)
    assert res.ndim == 2 and res.shape[0] == 2
    y = np.ascontiguousarray(y)
    return y, dirs, tap_idx, tap_w, tap_nnz, res, n_dirs, k_max


def _render(fn_name, y, length, dirs, tap_idx, tap_w, tap_nnz, refl_len, res, order=None):
    y, dirs, tap_idx, tap_w, tap_nnz, res, n_dirs, k_max = _render_common(
        y, dirs, tap_idx, tap_w, tap_nnz, res)
    S, ld = y.shape
    L = int(ld if length is None else length)
    assert 0 <= L <= ld and dirs.shape == (S,)
    res_len = res.shape[1]
    H = res_len + refl_len - 1
    n_out = L + H - 1
    out = np.zeros((2, max(n_out, 1)))
    lib = _load()
    args = [S, L, _p(y, _F), ld, _p(dirs, _I32), n_dirs, k_max, _p(tap_idx, _U16),
            _p(tap_w, _F), _p(tap_nnz, _U8), refl_len, res_len, _p(res, _F)]
    if order is not None:
        args.append(int(order))
    args += [_p(out, _D), out.shape[1]]
    rc = getattr(lib, fn_name)(*args)
    if rc != 0:
        raise ValueError(f"{fn_name} rejected its arguments (rc={rc})")
    return out[:, :n_out] if L > 0 else np.zeros((2, 0))


def render_sparse(y, dirs, tap_idx, tap_w, tap_nnz, refl_len, res, length=None, order=0):
    """out_e = sum_s (y_s * g_{dir s, e}) * f_e  (order 0) or (y_s * f_e) * g  (order 1).

    y [S][ld] FP32 (first ``length`` samples used), taps [n_dirs][2][k_max], res [2][Lf].
    Returns FP64 [2][L+H-1], H = Lf + refl_len - 1."""
    return _render("orc_render_sparse", y, length, dirs, tap_idx, tap_w, tap_nnz, refl_len, res,
                   order=order)


def render_dense(y, dirs, tap_idx, tap_w, tap_nnz, refl_len, res, length=None):
    """Same quantity as render_sparse, by direct convolution with the dense HRIR f*g."""
    return _render("orc_render_dense", y, length, dirs, tap_idx, tap_w, tap_nnz, refl_len, res)


def render_fft(y, dirs, tap_idx, tap_w, tap_nnz, refl_len, res, length=None):
    """Same quantity as render_sparse, by FFT convolution with the dense HRIR f*g."""
    return _render("orc_render_fft", y, length, dirs, tap_idx, tap_w, tap_nnz, refl_len, res)


def render_at(y, dirs, tap_idx, tap_w, tap_nnz, refl_len, res, positions, length=None):
    """The mix of render_sparse evaluated only at the given output positions ([2][n_pos]),
    straight from the cascade definition; cost independent of the source length."""
    y, dirs, tap_idx, tap_w, tap_nnz, res, n_dirs, k_max = _render_common(
        y, dirs, tap_idx, tap_w, tap_nnz, res)
    S, ld = y.shape
    L = int(ld if length is None else length)
    pos = np.ascontiguousarray(positions, dtype=np.int64)
    out = np.zeros((2, max(pos.size, 1)))
    rc = _load().orc_render_sparse_at(
        S, L, _p(y, _F), ld, _p(dirs, _I32), n_dirs, k_max, _p(tap_idx, _U16), _p(tap_w, _F),
        _p(tap_nnz, _U8), refl_len, res.shape[1], _p(res, _F),
        pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pos.size, _p(out, _D))
    if rc != 0:
        raise ValueError(f"orc_render_sparse_at rejected its arguments (rc={rc})")
    return out[:, :pos.size]


def dense_hrirs(tap_idx, tap_w, tap_nnz, refl_len, res) -> np.ndarray:
    """Dense HRIRs x_{d,e} = f_e * g_{d,e} (Eq. 1) in FP64, [n_dirs][2][H]."""
    tap_idx = np.asarray(tap_idx)
    n_dirs, _, _ = tap_idx.shape
    res = np.asarray(res, dtype=np.float64)
    H = res.shape[1] + refl_len - 1
    out = np.zeros((n_dirs, 2, H))
    for d in range(n_dirs):
        for e in range(2):
            g = np.zeros(refl_len)
            k = int(tap_nnz[d][e])
            np.add.at(g, np.asarray(tap_idx[d, e, :k], dtype=np.int64),
                      np.asarray(tap_w[d, e, :k], dtype=np.float64))
            out[d, e] = conv_direct(res[e], g)
    return out


def topk(g, k: int):
    """Top-k tap selection of non-negative FP32 rows g[..., refl_len].

    Returns (idx uint16 [..., k], w float32 [..., k], nnz uint8 [...]): the k largest
    strictly positive entries (larger value first, smaller index on ties), stored in
    ascending index order and padded with (0, 0.0)."""
    g = np.ascontiguousarray(g, dtype=np.float32)
    lead = g.shape[:-1]
    refl_len = g.shape[-1]
    rows = int(np.prod(lead)) if lead else 1
    idx = np.zeros(lead + (k,), dtype=np.uint16)
    w = np.zeros(lead + (k,), dtype=np.float32)
    nnz = np.zeros(lead, dtype=np.uint8)
    rc = _load().orc_topk(_p(g, _F), rows, refl_len, k, _p(idx, _U16), _p(w, _F), _p(nnz, _U8))
    if rc != 0:
        raise ValueError(f"orc_topk rejected its arguments (rc={rc})")
    return idx, w, nnz


# ---------------------------------------------------------------------------------------
# moving sources: per-segment reflection filters, output-domain linear crossfade
# ---------------------------------------------------------------------------------------
def _sparse_at(y, idx, w, k, n0, n1):
    """(y * g)[n] for n in [n0, n1) with g given by its k taps (zero outside y)."""
    L = y.size
    n = np.arange(n0, n1)
    acc = np.zeros(n.size)
    for t in range(k):
        m = n - int(idx[t])
        ok = (m >= 0) & (m < L)
        acc[ok] += float(w[t]) * y[m[ok]]
    return acc


def render_moving(y, tap_idx, tap_w, tap_nnz, seg_len: int, refl_len: int, res, length=None):
    """Binaural mix of moving sources (Eqs. 1-2 with a direction per segment).

    y [S][ld] FP32; tap tables [S][n_seg][2][k] give the reflection filter g_{s,j,e} of
    source s in segment j (samples [j seg_len, (j+1) seg_len)).  The reflection output of a
    source at output sample n in segment j is the linear crossfade
        z[n] = (1 - a) (y * g_{j-1})[n] + a (y * g_j)[n],   a = (n - j seg_len + 1) / seg_len
    for 1 <= j < n_seg; segment 0 uses g_0 alone and every n >= n_seg seg_len (the filter
    tails) uses g_{n_seg-1} alone.  Then out_e = f_e * sum_s z_{s,e}.  FP64 [2][L+H-1]."""
    y = np.asarray(y)
    if y.dtype != np.float32:
        raise TypeError("sources are FP32")
    S, ld = y.shape
    L = int(ld if length is None else length)
    tap_idx, tap_w, tap_nnz = np.asarray(tap_idx), np.asarray(tap_w), np.asarray(tap_nnz)
    n_seg = tap_idx.shape[1]
    assert tap_idx.shape[:3] == (S, n_seg, 2) and tap_nnz.shape == (S, n_seg, 2)
    res = np.asarray(res, dtype=np.float64)
    n_z = L + refl_len - 1
    if L == 0:
        return np.zeros((2, 0))
    z = np.zeros((2, n_z))
    for s in range(S):
        ys = y[s, :L].astype(np.float64)
        for j in range(max(n_seg, (n_z + seg_len - 1) // seg_len)):
            n0, n1 = j * seg_len, min((j + 1) * seg_len, n_z)
            if n0 >= n1:
                break
            jj = min(j, n_seg - 1)
            for e in range(2):
                cur = _sparse_at(ys, tap_idx[s, jj, e], tap_w[s, jj, e], int(tap_nnz[s, jj, e]), n0, n1)
                if 1 <= j < n_seg:
                    prev = _sparse_at(ys, tap_idx[s, j - 1, e], tap_w[s, j - 1, e],
                                      int(tap_nnz[s, j - 1, e]), n0, n1)
                    a = (np.arange(n0, n1) - n0 + 1) / seg_len
                    cur = (1.0 - a) * prev + a * cur
                z[e, n0:n1] += cur
    return np.stack([conv_direct(res[e], z[e]) for e in range(2)])
