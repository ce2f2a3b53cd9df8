"""Run the FP64 oracle's step on all host cores, for the CPU baseline.

TEST INFRASTRUCTURE ONLY: used by the benchmark's CPU-baseline leg and its
reference arm; never by the library.  No arithmetic of the method lives here:
each worker applies the oracle's own functions (oracle.gridpull) unchanged to
one chunk of a sample, and the parent only splits the work and times it.

Chunks are written by the parent to a scratch directory as .npy files before
the timed phases, so a worker only maps its chunk and computes.  Workers are
separate processes started with the "spawn" method, each with one BLAS thread.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

from . import gridpull as o

_POINTS = None


def _init(points_path: str):
    global _POINTS
    _POINTS = np.load(points_path, mmap_mode="r")


def _nn(path: str):
    """Brute-force NN(q) of one chunk of queries over the whole cloud."""
    q = np.load(path)
    t = time.perf_counter()
    o.nearest_point(q, np.asarray(_POINTS), chunk=_chunk(len(_POINTS)))
    return time.perf_counter() - t


def _chunk(J: int) -> int:
    """Queries per brute-force block: about 4e7 distances (a few hundred MB)."""
    return int(max(8, min(512, 4e7 // max(J, 1))))


def _nn_idx(path: str):
    """Brute-force NN(q) indices of one chunk of queries."""
    return o.nearest_point(np.load(path), np.asarray(_POINTS), chunk=_chunk(len(_POINTS)))


def _sigma(args):
    path, k = args
    idx = np.load(path)
    return o.knn_sigma(np.asarray(_POINTS), k, idx=idx, chunk=8)


def _terms(args):
    """Sampler + the query terms and their gradient for one chunk."""
    path, occ_path, R, M1, weights, seed = args
    z = np.load(path)
    pos, j = z["pos"], z["j"]
    sig = np.zeros(len(_POINTS))
    sig[z["sig_idx"]] = z["sig_val"]
    store = o.SparseValues(z["keys"], z["vals"])
    occ = np.load(occ_path, mmap_mode="r")
    t = time.perf_counter()
    q, jj = o.sample_queries(np.asarray(_POINTS), sig, seed, 0, pos)
    q = q.astype(np.float32)
    s = np.asarray(_POINTS)[j]
    member = lambda c: o.in_dilated_band(c, occ, M1, R, keys_sorted=True)
    o.query_terms(store, R, member, q, s, weights[1], weights[2], with_grad=True)
    return time.perf_counter() - t


def _tv(args):
    path, R, n_tv = args
    z = np.load(path)
    store = o.SparseValues(z["keys"], z["vals"])
    t = time.perf_counter()
    o.tv_term(store, R, z["tv"], True, n_tv)
    return time.perf_counter() - t


def _adam(args):
    path, lr = args
    z = np.load(path)
    t = time.perf_counter()
    o.adam(z["d"], z["g"], z["m"], z["v"], 3, lr)
    return time.perf_counter() - t


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class OraclePool:
    """A spawn-started process pool over the host's cores, each worker holding
    the cloud (memory-mapped from ``points_path``)."""

    def __init__(self, points_path: str, cores: int | None = None):
        self.cores = cores or host_cores()
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_init, initargs=(points_path,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def close(self):
        self.pool.close()
        self.pool.join()

    def timed_map(self, fn, items):
        """Wall time of running fn over items on every core."""
        t = time.perf_counter()
        self.pool.map(fn, items, chunksize=1)
        return time.perf_counter() - t

    def sigma(self, idx_paths, k):
        return np.concatenate(self.pool.map(_sigma, [(p, k) for p in idx_paths], chunksize=1))

    def nn(self, paths):
        return self.timed_map(_nn, paths)

    def nn_indices(self, paths):
        """Brute-force NN indices of the chunks, in order."""
        return np.concatenate(self.pool.map(_nn_idx, paths, chunksize=1))

    def terms(self, items):
        return self.timed_map(_terms, items)

    def tv(self, items):
        return self.timed_map(_tv, items)

    def adam(self, items):
        return self.timed_map(_adam, items)
