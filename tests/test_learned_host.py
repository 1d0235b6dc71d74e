"""Host-side pieces of the learned-filter layer that need no GPU: the parameter layout the C
ABI reports, the initial weights, the network's input rows and the nearest-grid fallback
(the method without the network)."""
import math

import numpy as np
import pytest

import oracle.mlp as omlp


@pytest.fixture(scope="module")
def learned():
    from paper_1502_03162_gb300 import build, hrir, learned
    build.build()
    hrir.load_library()
    return learned


@pytest.mark.parametrize("refl_len", [1, 33, 200, 256, 2048])
def test_param_count_agrees_with_the_oracle_layout(learned, refl_len):
    from paper_1502_03162_gb300 import hrir
    assert hrir.hrir_mlp_param_count(refl_len) == omlp.param_count(refl_len)


def test_param_count_rejects_bad_lengths(learned):
    from paper_1502_03162_gb300 import hrir
    assert hrir.hrir_mlp_param_count(0) == 0
    assert hrir.hrir_mlp_param_count(2049) == 0


def test_initial_weights(learned):
    refl_len, mean = 200, 0.0137
    p = learned.init_params(refl_len, seed=5, target_mean=mean)
    assert p.dtype == np.float32
    layers = omlp.unpack(p.astype(np.float64), refl_len)
    sizes = learned.layer_sizes(refl_len)
    for i, (W, b) in enumerate(layers):
        fan_in = sizes[i]
        bound = 1.0 / math.sqrt(fan_in)
        assert W.shape == (sizes[i + 1], fan_in)
        if i < len(layers) - 1:
            assert np.all(np.abs(W) <= bound) and np.all(np.abs(b) <= bound)
        else:
            assert np.all(np.abs(W) <= 0.1 * bound + 1e-7)
            # softplus(bias) is the mean target tap, so an all-zero last hidden layer outputs it
            assert np.allclose(np.log1p(np.exp(b)), mean, rtol=1e-5)
    assert np.array_equal(p, learned.init_params(refl_len, seed=5, target_mean=mean))
    assert not np.array_equal(p, learned.init_params(refl_len, seed=6, target_mean=mean))


def test_direction_rows_order_and_ear_sign(learned):
    az = np.array([0.1, 1.2, -2.0])
    el = np.array([0.0, 0.5, -0.7])
    rows = learned.direction_rows(az, el)
    assert rows.shape == (6, 3) and rows.dtype == np.float32
    for d in range(3):
        for e, sign in ((0, -1.0), (1, 1.0)):
            assert np.allclose(rows[2 * d + e], [az[d], el[d], sign])
    one = learned.direction_rows(az, el, ears=(1,))
    assert np.allclose(one[:, 2], 1.0) and np.allclose(one[:, 0], az)


def test_nearest_grid_tables(learned):
    rng = np.random.default_rng(3)
    n_dirs, k = 40, 4
    gaz = rng.uniform(-math.pi, math.pi, n_dirs)
    gel = rng.uniform(-1.2, 1.2, n_dirs)
    idx = rng.integers(0, 200, (n_dirs, 2, k)).astype(np.uint16)
    w = rng.random((n_dirs, 2, k)).astype(np.float32)
    nnz = rng.integers(0, k + 1, (n_dirs, 2)).astype(np.uint8)
    # queries exactly at grid directions pick those directions
    qi, qw, qn, nn = learned.nearest_grid_tables(gaz, gel, idx, w, nnz, gaz[None, :], gel[None, :])
    assert np.array_equal(nn[0], np.arange(n_dirs))
    assert np.array_equal(qi[0], idx) and np.array_equal(qw[0], w) and np.array_equal(qn[0], nnz)
    # an azimuth one full turn away is the same direction
    _, _, _, nn2 = learned.nearest_grid_tables(gaz, gel, idx, w, nnz, (gaz + 2 * math.pi)[None, :],
                                               gel[None, :])
    assert np.array_equal(nn2[0], np.arange(n_dirs))
    # brute force: the smallest great-circle angle
    qaz = rng.uniform(-math.pi, math.pi, (5, 7))
    qel = rng.uniform(-1.4, 1.4, (5, 7))
    _, _, _, nn3 = learned.nearest_grid_tables(gaz, gel, idx, w, nnz, qaz, qel)
    for s in range(5):
        for j in range(7):
            ang = [math.acos(max(-1.0, min(1.0, math.sin(qel[s, j]) * math.sin(gel[d]) +
                                           math.cos(qel[s, j]) * math.cos(gel[d]) *
                                           math.cos(qaz[s, j] - gaz[d]))))
                   for d in range(n_dirs)]
            assert nn3[s, j] == int(np.argmin(ang))
