"""The oracle's sort-based forms evaluated with the coordinates spread over
host processes.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests, the
package's ``smoke()`` check and the benchmark's CPU-baseline and reference
legs use it; the library never imports it.

Algorithm 2 (Section 2) handles the d coordinates independently and sums
their contributions ("summing over all i in [d]"); the l1 gradient and the
odd-p form of Theorem "odd_p" are likewise a sum (or a column) per
coordinate.  So each worker process runs the serial oracle function itself
(``oracle.l1_sort``, ``oracle.l1_grad_sort``, ``oracle.lpp_odd_sort``) on a
contiguous block of coordinates, and the parent adds the blocks' results in
block order.  Nothing here re-implements the method: the only change from
the serial call is the grouping of the final sum over coordinates (exact for
integer inputs, a rounding-level difference in FP64).

Workers are started with the ``spawn`` method (a pool forked from a process
that has touched the GPU can hang); the arrays travel through shared memory.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

import oracle


def default_workers(d: int) -> int:
    return max(1, min(d, os.cpu_count() or 1))


def _blocks(d: int, workers: int):
    w = max(1, min(workers, d))
    edges = np.linspace(0, d, w + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


class _Shared:
    """A numpy array in a named shared-memory segment."""

    def __init__(self, shape, dtype, src=None):
        dtype = np.dtype(dtype)
        nbytes = max(1, int(np.prod(shape)) * dtype.itemsize)
        self.shm = shared_memory.SharedMemory(create=True, size=nbytes)
        self.array = np.ndarray(shape, dtype=dtype, buffer=self.shm.buf)
        if src is not None:
            self.array[...] = src
        self.spec = (self.shm.name, tuple(shape), dtype.str)

    def close(self):
        del self.array
        self.shm.close()
        self.shm.unlink()


def _attach(spec):
    name, shape, dtype = spec
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf)


def _work(job):
    kind, lo, hi, slot, specs, extra = job
    handles = [_attach(s) for s in specs]
    try:
        arrays = [a for _, a in handles]
        if kind == "l1_sort":
            X, Z, out = arrays
            out[slot] = oracle.l1_sort(X[:, lo:hi], Z)
        elif kind == "lpp_odd_sort":
            X, Z, out = arrays
            out[slot] = oracle.lpp_odd_sort(X[:, lo:hi], Z, extra)
        elif kind == "l1_grad_sort":
            X, W, Z, G = arrays
            G[:, lo:hi] = oracle.l1_grad_sort(X[:, lo:hi], W, Z)
        else:
            raise ValueError(kind)
        del arrays
    finally:
        for shm, a in handles:
            del a
            shm.close()
    return None


def _result_dtype(X, Z):
    return np.int64 if (np.issubdtype(X.dtype, np.integer) and np.issubdtype(Z.dtype, np.integer)) \
        else np.float64


def executor(workers: int) -> ProcessPoolExecutor:
    """A spawned worker pool that callers may pass to several calls (an
    executor, not a Pool: a worker that dies raises instead of being replaced
    forever)."""
    return ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def _run(jobs, pool=None):
    if pool is not None:
        list(pool.map(_work, jobs))
    elif len(jobs) == 1:
        _work(jobs[0])
    else:
        with executor(len(jobs)) as ex:
            list(ex.map(_work, jobs))


def _product(kind, X, Z, extra, workers, pool=None):
    X = np.asarray(X)
    Z = np.asarray(Z)
    if X.ndim == 1:
        X = X[:, None]
    squeeze = Z.ndim == 1
    if squeeze:
        Z = Z[:, None]
    n, d = X.shape
    k = Z.shape[1]
    blocks = _blocks(d, workers or default_workers(d))
    rt = _result_dtype(X, Z)
    sx = _Shared(X.shape, X.dtype, X)
    sz = _Shared(Z.shape, Z.dtype, Z)
    so = _Shared((len(blocks), n, k), rt)
    try:
        jobs = [(kind, lo, hi, s, [sx.spec, sz.spec, so.spec], extra)
                for s, (lo, hi) in enumerate(blocks)]
        _run(jobs, pool)
        out = so.array[0].copy()
        for s in range(1, len(blocks)):
            out += so.array[s]
    finally:
        for sh in (sx, sz, so):
            sh.close()
    return out[:, 0] if squeeze else out


def l1_sort(X, Z, workers: int | None = None, pool=None) -> np.ndarray:
    """``oracle.l1_sort`` (Algorithms 1 and 2) with blocks of coordinates on
    separate processes (a fresh pool, or ``pool`` from ``executor()``); the
    blocks' products are added in block order."""
    return _product("l1_sort", X, Z, None, workers, pool)


def lpp_odd_sort(X, Z, p: int, workers: int | None = None) -> np.ndarray:
    """``oracle.lpp_odd_sort`` (odd p, Theorem "odd_p") with blocks of
    coordinates on separate processes."""
    if p % 2 == 0:
        raise ValueError("p must be odd")
    return _product("lpp_odd_sort", X, Z, int(p), workers)


def l1_grad_sort(X, W, Z, workers: int | None = None) -> np.ndarray:
    """``oracle.l1_grad_sort`` with blocks of coordinates on separate
    processes; column c of the gradient depends on coordinate c alone."""
    X = np.asarray(X)
    if X.ndim == 1:
        X = X[:, None]
    W = np.asarray(W)
    Z = np.asarray(Z)
    if W.ndim == 1:
        W = W[:, None]
    if Z.ndim == 1:
        Z = Z[:, None]
    n, d = X.shape
    integer = all(np.issubdtype(a.dtype, np.integer) for a in (X, W, Z))
    rt = np.int64 if integer else np.float64
    blocks = _blocks(d, workers or default_workers(d))
    sx, sw, sz = (_Shared(a.shape, a.dtype, a) for a in (X, W, Z))
    sg = _Shared((n, d), rt)
    try:
        jobs = [("l1_grad_sort", lo, hi, 0, [sx.spec, sw.spec, sz.spec, sg.spec], None)
                for lo, hi in blocks]
        _run(jobs)
        G = sg.array.copy()
    finally:
        for sh in (sx, sw, sz, sg):
            sh.close()
    return G
