"""Shared helpers of the GPU parity tests (inputs from synth, references from the oracle)."""
import numpy as np

import oracle
from paper_1502_03162_gb300 import synth

# FP32 GPU path vs FP64 oracle: max-abs error <= 1e-5 x RMS(out), per ear.
TOL = 1e-5


def tables(rng, n_dirs, k, refl_len=200, res_len=32, n_refl=48):
    G = synth.reflection_bank(rng, n_dirs, n_refl=n_refl, refl_len=refl_len)
    idx, w, nnz = oracle.topk(G, k)
    res = synth.resonance(rng, res_len)
    return G, idx, w, nnz, res


def max_err_over_rms(out, ref):
    """[2] array of max|out - ref| / RMS(ref) per ear."""
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    r = []
    for e in range(2):
        rms = np.sqrt(np.mean(ref[e] ** 2))
        r.append(np.max(np.abs(out[e] - ref[e])) / rms if ref.shape[1] else 0.0)
    return np.array(r)


def assert_close(out, ref, tol=TOL, what=""):
    err = max_err_over_rms(out, ref)
    assert np.all(err <= tol), f"{what}: max err / RMS = {err} > {tol}"
    return err
