"""Seeded synthetic inputs for the rendering path (sources, directions, filters).

This module only draws random inputs with the shapes and value distributions of the
workloads; it holds none of the rendering arithmetic.  Both the CUDA path's tests and the
oracle's tests take their inputs from here.  Everything is numpy and deterministic given
the seed.

Workloads (the paper measures on the CIPIC HRTF set -- 1250 directions, 200-tap HRIRs,
Sec. IV-A -- which is not available here; these generators stand in for it with the same
shapes):
  * tiny:    1 source x 44100 samples N(0,1); one direction; per-ear 32-tap resonance
             exp(-n/6) N(0,1) normalised to unit L2; 200-tap reflection with 16 taps at
             distinct uniform positions (first tap at 0), weights Exp(1) exp(-n/60).
  * batched: S sources x L samples of AR(1) noise (coefficient 0.95, stationary start),
             directions uniform over a 25 x 50 azimuth/elevation grid (1250 directions),
             dense non-negative reflection rows with `n_refl` reflections each, from
             which the K-tap tables are selected by top-K.
"""
from __future__ import annotations

import numpy as np

N_AZ, N_EL = 25, 50
N_DIRS = N_AZ * N_EL          # 1250
REFL_LEN = 200                # reflection filter length Lg
RES_LEN = 32                  # resonance filter length Lf


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def az_el_grid():
    """Synthetic direction grid: 25 azimuths x 50 elevations (radians), row-major [az][el]."""
    az = np.linspace(-80.0, 80.0, N_AZ)
    el = np.linspace(-45.0, 230.0, N_EL)
    A, E = np.meshgrid(az, el, indexing="ij")
    return np.deg2rad(A.ravel()), np.deg2rad(E.ravel())


def resonance(rng: np.random.Generator, res_len: int = RES_LEN, n_ears: int = 2) -> np.ndarray:
    """Per-ear resonance f_e[n] = exp(-n/6) N(0,1), scaled to unit L2 norm; float32 [ears][Lf]."""
    n = np.arange(res_len)
    f = np.exp(-n / 6.0)[None, :] * rng.standard_normal((n_ears, res_len))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    return f.astype(np.float32)


def reflection_row(rng: np.random.Generator, n_taps: int, refl_len: int = REFL_LEN) -> np.ndarray:
    """One dense non-negative reflection row with n_taps non-zeros at distinct positions
    (position 0 always present), weights Exp(1) exp(-n/60); float32 [refl_len]."""
    n_taps = min(n_taps, refl_len)
    pos = np.concatenate([[0], 1 + rng.choice(refl_len - 1, size=n_taps - 1, replace=False)])
    g = np.zeros(refl_len, dtype=np.float64)
    g[pos] = rng.exponential(1.0, size=pos.size) * np.exp(-pos / 60.0)
    return g.astype(np.float32)


def reflection_bank(rng: np.random.Generator, n_dirs: int = N_DIRS, n_refl: int = 48,
                    refl_len: int = REFL_LEN, n_ears: int = 2) -> np.ndarray:
    """Dense reflection rows for every (direction, ear): float32 [n_dirs][ears][refl_len]."""
    G = np.zeros((n_dirs, n_ears, refl_len), dtype=np.float32)
    for d in range(n_dirs):
        for e in range(n_ears):
            G[d, e] = reflection_row(rng, n_refl, refl_len)
    return G


def sources_white(rng: np.random.Generator, S: int, L: int, ld: int | None = None,
                  dtype=np.float32) -> np.ndarray:
    """S x ld array whose first L columns are N(0,1) samples; columns >= L are zero."""
    ld = L if ld is None else ld
    y = np.zeros((S, ld), dtype=dtype)
    y[:, :L] = rng.standard_normal((S, L), dtype=np.float32)
    return y


def sources_ar1(rng: np.random.Generator, S: int, L: int, ld: int | None = None,
                coef: float = 0.95, out: np.ndarray | None = None,
                chunk: int = 32) -> np.ndarray:
    """AR(1) 'pink-ish' noise: y[0] = e[0] / sqrt(1 - coef^2), y[n] = coef y[n-1] + e[n],
    e ~ N(0,1).  float32 [S][ld] (columns >= L are zero).  Written into `out` if given."""
    import scipy.signal
    ld = L if ld is None else ld
    if out is None:
        out = np.zeros((S, ld), dtype=np.float32)
    else:
        assert out.shape == (S, ld) and out.dtype == np.float32
        if ld > L:
            out[:, L:] = 0.0
    if L == 0:
        return out
    # the filter gives y[0] = e[0] + zi: zi = e[0] (1/sqrt(1-c^2) - 1) makes y[0] have the
    # stationary variance 1/(1-c^2)
    zi_scale = 1.0 / np.sqrt(1.0 - coef * coef) - 1.0
    for s0 in range(0, S, chunk):
        s1 = min(S, s0 + chunk)
        e = rng.standard_normal((s1 - s0, L), dtype=np.float32)
        zi = (zi_scale * e[:, :1]).astype(np.float32)
        y, _ = scipy.signal.lfilter([1.0], [1.0, -coef], e, axis=1, zi=zi)
        out[s0:s1, :L] = y.astype(np.float32)
    return out


def directions(rng: np.random.Generator, S: int, n_dirs: int = N_DIRS) -> np.ndarray:
    return rng.integers(0, n_dirs, size=S).astype(np.int32)


def tiny_config(seed: int = 1, L: int = 44100):
    """1 source x L samples, 1 direction, K = 16 of 200 reflection taps, 32-tap resonance.

    Returns dict(y [1][L] f32, dirs [1] i32, G [1][2][200] f32 dense rows, res [2][32])."""
    rng = rng_for(seed)
    y = sources_white(rng, 1, L)
    res = resonance(rng)
    G = np.stack([reflection_row(rng, 16), reflection_row(rng, 16)])[None]
    return dict(y=y, dirs=np.zeros(1, np.int32), G=G, res=res, k=16)


def batched_config(S: int = 1024, L: int = 480000, seed: int = 2, ld: int | None = None,
                   n_dirs: int = N_DIRS, n_refl: int = 48, out: np.ndarray | None = None):
    """S sources x L samples AR(1) noise, directions uniform over n_dirs, dense reflection
    rows with n_refl non-zeros (top-K selects the K-tap tables), 32-tap resonance."""
    rng = rng_for(seed)
    res = resonance(rng)
    G = reflection_bank(rng, n_dirs, n_refl)
    dirs = directions(rng, S, n_dirs)
    y = sources_ar1(rng, S, L, ld, out=out)
    return dict(y=y, dirs=dirs, G=G, res=res)


# ---------------------------------------------------------------------------------------
# synthetic HRIR sets for the learned filters (stand-ins for measured HRIR databases)
# ---------------------------------------------------------------------------------------
def hrir_set_params(seed: int, n_refl: int = 10, refl_len: int = REFL_LEN,
                    res_len: int = RES_LEN) -> dict:
    """Parameters of one seeded synthetic HRIR set.

    Per ear: a 32-tap resonance (as `resonance`).  Reflections k = 0..n_refl-1, k = 0 being
    the direct path at delay 0: base delay d0_k, delay swing a_k with phase p_k, gain
    c0_k with a gain swing of up to 40% and phase q_k.  The right ear mirrors the azimuth."""
    rng = rng_for(seed)
    res = resonance(rng, res_len)
    d0 = np.concatenate([[0.0], np.sort(rng.uniform(8.0, refl_len - 40.0, n_refl - 1))])
    amp = np.concatenate([[0.0], rng.uniform(0.5, 4.0, n_refl - 1)])
    return dict(res=res, d0=d0, amp=amp, phase=rng.uniform(0, 2 * np.pi, n_refl),
                gain=np.concatenate([[1.0], rng.uniform(0.15, 0.6, n_refl - 1)]),
                gswing=rng.uniform(0.0, 0.4, n_refl), gphase=rng.uniform(0, 2 * np.pi, n_refl),
                refl_len=refl_len)


def hrir_set_reflections(p: dict, az, el, ear) -> np.ndarray:
    """Non-negative reflection rows [n][refl_len] at arbitrary directions (radians; ear 0
    left, 1 right): each reflection is a two-tap linear-interpolation pulse at its delay
    d0 + a cos(az' - p) cos(el), az' = az (left) or -az (right)."""
    az = np.asarray(az, dtype=np.float64)
    el = np.asarray(el, dtype=np.float64)
    ear = np.asarray(ear)
    azs = np.where(ear == 0, az, -az)
    n = az.size
    Lg = p["refl_len"]
    g = np.zeros((n, Lg))
    rows = np.arange(n)
    for k in range(p["d0"].size):
        d = p["d0"][k] + p["amp"][k] * np.cos(azs - p["phase"][k]) * np.cos(el)
        d = np.clip(d, 0.0, Lg - 1.001)
        c = p["gain"][k] * (1.0 + p["gswing"][k] * np.cos(azs - p["gphase"][k]) * np.cos(el)) \
            * np.exp(-d / 60.0)
        i0 = np.floor(d).astype(np.int64)
        fr = d - i0
        np.add.at(g, (rows, i0), c * (1.0 - fr))
        np.add.at(g, (rows, i0 + 1), c * fr)
    return g


def hrir_set_at(p: dict, az, el, ear) -> np.ndarray:
    """HRIRs [n][H] (H = Lf + Lg - 1) at arbitrary directions: the resonance of the ear
    followed by its reflections, scaled to absolute sum 1 (the paper's HRIR preprocessing
    normalises every HRIR that way).  Data generation only: this stands in for measured
    HRIRs, it is not part of the rendering path."""
    g = hrir_set_reflections(p, az, el, ear)
    ear = np.asarray(ear)
    res = p["res"].astype(np.float64)
    H = res.shape[1] + g.shape[1] - 1
    x = np.zeros((g.shape[0], H))
    for i in range(g.shape[0]):
        x[i] = np.convolve(res[int(ear[i])], g[i])
    return x / np.sum(np.abs(x), axis=1, keepdims=True)


def hrir_set(seed: int, **kw):
    """One synthetic HRIR set on the 25 x 50 grid: (X [1250][2][H], az [1250], el [1250],
    params)."""
    p = hrir_set_params(seed, **kw)
    az, el = az_el_grid()
    n = az.size
    X = np.stack([hrir_set_at(p, az, el, np.full(n, e)) for e in range(2)], axis=1)
    return X, az, el, p


def trajectories(rng: np.random.Generator, S: int, n_seg: int):
    """Moving-source directions per (source, segment): each source starts at a uniform
    direction in the grid's azimuth/elevation range and moves at a constant random velocity
    of at most 0.5 degrees per segment in each angle, reflected at the range's edges.
    Returns (az, el) radians [S][n_seg]."""
    az_lo, az_hi = np.deg2rad(-80.0), np.deg2rad(80.0)
    el_lo, el_hi = np.deg2rad(-45.0), np.deg2rad(230.0)
    az0 = rng.uniform(az_lo, az_hi, S)
    el0 = rng.uniform(el_lo, el_hi, S)
    vaz = rng.uniform(-1.0, 1.0, S) * np.deg2rad(0.5)     # per segment (~90 deg/s at 48 kHz)
    vel = rng.uniform(-1.0, 1.0, S) * np.deg2rad(0.5)
    t = np.arange(n_seg)[None, :]
    az = az0[:, None] + vaz[:, None] * t
    el = el0[:, None] + vel[:, None] * t
    # reflect at the range edges
    span_a, span_e = az_hi - az_lo, el_hi - el_lo
    az = az_lo + span_a - np.abs(np.mod(az - az_lo, 2 * span_a) - span_a)
    el = el_lo + span_e - np.abs(np.mod(el - el_lo, 2 * span_e) - span_e)
    return az, el
