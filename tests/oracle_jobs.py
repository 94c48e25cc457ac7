"""The oracle's full B of the full-size workloads, computed in background
processes while the GPU tests run.

The oracle is single-threaded and takes from under a minute (1M x 100 bp) to
several minutes (2M ragged reads) per workload, so the tests that compare the
GPU's B with it element by element start every oracle job as soon as pytest
has collected them (``start``), each in its own process, and wait for the
result only when they need it (``result``).  The processes are started with
``spawn``, never forked from a process that has touched the GPU.  Each job
generates its workload itself from the seeds, exactly as the test does, and
writes B to a temporary ``.npy`` file; nothing here computes any part of the
method.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

# workload name -> a function of no arguments returning (reads, offsets, alphabet)


def _short():
    import readgen
    w = readgen.short()
    return w.reads, w.offsets, w.alphabet


def _batched():
    import readgen
    w = readgen.batched()
    return w.reads, w.offsets, w.alphabet


def _long():
    import readgen
    w = readgen.long()
    return w.reads, w.offsets, w.alphabet


def _serving_20():
    import readgen
    resident, requests = readgen.serving_scaled(20)
    return concat_in_order([(resident.reads, resident.offsets)] + list(requests)) + (b"ACGT",)


WORKLOADS = {"short": _short, "batched": _batched, "long": _long, "serving_20": _serving_20}


def concat_in_order(sets):
    """(reads, offsets) of several read sets one after the other (the read
    ids the GPU assigns when they are appended in this order)."""
    reads = np.concatenate([np.asarray(r, np.uint8) for r, _ in sets])
    lens = np.concatenate([np.diff(np.asarray(o, np.uint64).astype(np.int64)) for _, o in sets])
    off = np.zeros(len(lens) + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    return reads, off


def _job(name: str, path: str) -> str:
    import oracle
    reads, off, alphabet = WORKLOADS[name]()
    B = oracle.bwt(reads, off, alphabet)
    np.save(path, B)
    return path


_pool = None
_pending = {}
_dir = None


def start(names) -> None:
    """Starts the oracle jobs of `names` (at most one process each)."""
    global _pool, _dir
    names = [n for n in names if n not in _pending]
    if not names:
        return
    import oracle
    oracle.build()  # compile once here, not in every child
    if _pool is None:
        _dir = tempfile.mkdtemp(prefix="sbwt_oracle_")
        _pool = mp.get_context("spawn").Pool(processes=len(WORKLOADS))
    for n in names:
        _pending[n] = _pool.apply_async(_job, (n, os.path.join(_dir, n + ".npy")))


def result(name: str, timeout: float = 3600.0) -> np.ndarray:
    """The oracle's B of workload `name` (starting its job if needed)."""
    start([name])
    return np.load(_pending[name].get(timeout=timeout), mmap_mode="r")


def stop() -> None:
    """Ends every job and removes the results."""
    global _pool
    if _pool is not None:
        _pool.terminate()
        _pool.join()
        _pool = None
    _pending.clear()
    if _dir and os.path.isdir(_dir):
        for f in os.listdir(_dir):
            os.remove(os.path.join(_dir, f))
        os.rmdir(_dir)
