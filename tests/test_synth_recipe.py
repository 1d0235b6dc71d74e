"""The seeded input generators follow the stated input recipe (shapes, supports, value
distributions, structure); they hold none of the rendering arithmetic."""
import math

import numpy as np
import pytest

from paper_1502_03162_gb300 import synth


def test_direction_grid():
    az, el = synth.az_el_grid()
    assert az.shape == el.shape == (1250,)
    assert np.isclose(np.rad2deg(az).min(), -80) and np.isclose(np.rad2deg(az).max(), 80)
    assert np.isclose(np.rad2deg(el).min(), -45) and np.isclose(np.rad2deg(el).max(), 230)
    assert len(set(zip(np.round(az, 9), np.round(el, 9)))) == 1250


def test_resonance_unit_norm_and_envelope():
    f = synth.resonance(synth.rng_for(0))
    assert f.shape == (2, 32) and f.dtype == np.float32
    assert np.allclose(np.linalg.norm(f.astype(np.float64), axis=1), 1.0, atol=1e-6)
    # exp(-n/6) envelope: over many draws the energy of the tail is tiny
    fs = np.stack([synth.resonance(synth.rng_for(s)) for s in range(200)]).astype(np.float64)
    e = np.mean(fs ** 2, axis=(0, 1))
    assert e[:8].sum() > 0.9 and e[24:].sum() < 1e-3


@pytest.mark.parametrize("n_taps", [1, 16, 48, 200])
def test_reflection_row_support(n_taps):
    rng = synth.rng_for(n_taps)
    for _ in range(20):
        g = synth.reflection_row(rng, n_taps)
        assert g.shape == (200,) and g.dtype == np.float32
        assert np.all(g >= 0)
        nz = np.flatnonzero(g)
        assert nz[0] == 0 and nz.size == n_taps   # distinct positions, tap 0 always present


def test_reflection_bank_shape_and_determinism():
    G = synth.reflection_bank(synth.rng_for(4), n_dirs=10, n_refl=48)
    assert G.shape == (10, 2, 200)
    assert np.all((G > 0).sum(axis=2) == 48)
    assert np.array_equal(G, synth.reflection_bank(synth.rng_for(4), n_dirs=10, n_refl=48))


def test_ar1_sources_are_stationary_with_the_stated_coefficient():
    S, L, ld, c = 64, 20000, 20008, 0.95
    y = synth.sources_ar1(synth.rng_for(7), S, L, ld, coef=c)
    assert y.shape == (S, ld) and y.dtype == np.float32
    assert np.all(y[:, L:] == 0)
    x = y[:, :L].astype(np.float64)
    var = 1.0 / (1.0 - c * c)
    # stationary from the first sample: the variance at n = 0 is already 1 / (1 - c^2)
    assert abs(np.mean(x[:, 0] ** 2) / var - 1.0) < 0.4
    assert abs(np.mean(x ** 2) / var - 1.0) < 0.05
    r1 = np.mean(x[:, 1:] * x[:, :-1]) / np.mean(x ** 2)
    assert abs(r1 - c) < 0.005
    # innovations y[n] - c y[n-1] are N(0, 1)
    e = x[:, 1:] - c * x[:, :-1]
    assert abs(e.mean()) < 0.01 and abs(e.std() - 1.0) < 0.01
    # writing into a caller's buffer gives the same samples
    out = np.full((S, ld), 7.0, np.float32)
    synth.sources_ar1(synth.rng_for(7), S, L, ld, coef=c, out=out)
    assert np.array_equal(out, y)


def test_directions_uniform_over_the_grid():
    d = synth.directions(synth.rng_for(9), 200000)
    assert d.dtype == np.int32 and d.min() == 0 and d.max() == 1249
    counts = np.bincount(d, minlength=1250)
    assert counts.min() > 100 and counts.max() < 230      # 160 expected per direction


def test_trajectories_stay_in_range_and_move_slowly():
    S, n_seg = 300, 375
    az, el = synth.trajectories(synth.rng_for(11), S, n_seg)
    assert az.shape == el.shape == (S, n_seg)
    eps = 1e-12
    assert np.all(az >= math.radians(-80) - eps) and np.all(az <= math.radians(80) + eps)
    assert np.all(el >= math.radians(-45) - eps) and np.all(el <= math.radians(230) + eps)
    step = np.maximum(np.abs(np.diff(az, axis=1)), np.abs(np.diff(el, axis=1)))
    assert np.all(step <= math.radians(0.5) + 1e-12)


def test_hrir_set_structure():
    p = synth.hrir_set_params(3)
    az = np.array([0.3, -1.0, 0.0])
    el = np.array([0.1, 0.4, -0.6])
    for ear in (0, 1):
        g = synth.hrir_set_reflections(p, az, el, np.full(3, ear))
        assert g.shape == (3, 200) and np.all(g >= 0)
        x = synth.hrir_set_at(p, az, el, np.full(3, ear))
        assert x.shape == (3, 231)
        assert np.allclose(np.abs(x).sum(axis=1), 1.0)
    # the right ear mirrors the azimuth of the left
    gl = synth.hrir_set_reflections(p, -az, el, np.zeros(3, int))
    gr = synth.hrir_set_reflections(p, az, el, np.ones(3, int))
    assert np.allclose(gl, gr)
    # the direct path (reflection 0) sits at delay 0 with gain 1 before the swing
    g0 = synth.hrir_set_reflections(dict(p, d0=p["d0"][:1], amp=p["amp"][:1], phase=p["phase"][:1],
                                         gain=p["gain"][:1], gswing=np.zeros(1),
                                         gphase=p["gphase"][:1]), az, el, np.zeros(3, int))
    assert np.allclose(g0[:, 0], 1.0) and np.allclose(g0[:, 1:], 0.0)
