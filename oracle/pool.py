"""The oracle's renderers run over source slices in worker processes.

TEST INFRASTRUCTURE ONLY (part of the oracle).  The binaural mix is linear in the sources
(Eq. 2 summed over sources), so the mix of a batch is the sum of the mixes of contiguous
source slices.  ``SlicedRenderer`` renders each slice with the plain FP64 oracle in its own
spawned process (safe after CUDA was initialised in the parent) and sums the slices' mixes
in FP64 in slice order.  It adds no arithmetic of its own beyond that sum.
"""
from __future__ import annotations

import os
import time

import numpy as np


def _part(job):
    """Worker: render sources [s0, s1) of the shared batch with one of the oracle's renderers."""
    from multiprocessing import shared_memory
    import oracle
    name, shape, s0, s1, L, mode, dirs, idx, w, nnz, refl_len, res = job
    shm = shared_memory.SharedMemory(name=name)
    try:
        y = np.ndarray(shape, dtype=np.float32, buffer=shm.buf)[s0:s1]
        fn = {"sparse": oracle.render_sparse, "dense": oracle.render_dense,
              "fft": oracle.render_fft}[mode]
        return fn(np.ascontiguousarray(y), dirs[s0:s1], idx, w, nnz, refl_len, res, length=L)
    finally:
        shm.close()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class SlicedRenderer:
    """Holds a source batch y [S][ld] (FP32) in shared memory and a pool of spawned workers.

    run(n_src, L, mode, workers) renders the first n_src sources over L samples with
    oracle.render_<mode> split into `workers` contiguous slices and returns (wall seconds,
    FP64 mix [2][L + H - 1])."""

    def __init__(self, y, dirs, idx, w, nnz, refl_len, res, cores=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import oracle
        oracle.build()
        y = np.asarray(y)
        if y.dtype != np.float32 or y.ndim != 2:
            raise TypeError("y must be a 2-D float32 array")
        self.cores = int(cores or host_cores())
        self.shm = shared_memory.SharedMemory(create=True, size=max(y.nbytes, 1))
        self.y = np.ndarray(y.shape, dtype=np.float32, buffer=self.shm.buf)
        self.y[:] = y
        self.tables = (np.ascontiguousarray(dirs, np.int32), np.ascontiguousarray(idx, np.uint16),
                       np.ascontiguousarray(w, np.float32), np.ascontiguousarray(nnz, np.uint8),
                       int(refl_len), np.ascontiguousarray(res, np.float32))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.run(min(self.cores, y.shape[0]), min(2000, y.shape[1]), "sparse")   # warm every worker

    def set_tables(self, idx, w, nnz):
        """Render with other tap tables (same directions, Lg and resonance)."""
        dirs, _, _, _, refl_len, res = self.tables
        self.tables = (dirs, np.ascontiguousarray(idx, np.uint16), np.ascontiguousarray(w, np.float32),
                       np.ascontiguousarray(nnz, np.uint8), refl_len, res)

    def run(self, n_src, L, mode="sparse", workers=None):
        dirs, idx, w, nnz, refl_len, res = self.tables
        workers = max(1, min(workers or self.cores, n_src))
        cuts = [n_src * i // workers for i in range(workers + 1)]
        jobs = [(self.shm.name, self.y.shape, cuts[i], cuts[i + 1], L, mode, dirs, idx, w, nnz,
                 refl_len, res) for i in range(workers)]
        t = time.perf_counter()
        parts = self.pool.map(_part, jobs, chunksize=1)
        out = parts[0].copy()
        for p in parts[1:]:
            out += p
        return time.perf_counter() - t, out

    def close(self):
        self.pool.close()
        self.pool.join()
        del self.y
        self.shm.close()
        self.shm.unlink()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
