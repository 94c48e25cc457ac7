"""GB300 set-bwte: incremental BWT / FM-index construction of read sets.

Python binding of ``libsbwt.so`` (the C ABI declared in ``include/sbwt.h``).
It only marshals arguments: every step of the path (packing, ConstructSA,
B_int, ComputeRanks, the g[SA_int] gather, Insert, rank queries) runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or was not built for this GPU, importing works but every call raises.

The functions carry the C names (``sbwt_create``, ``sbwt_append``, ...);
:class:`SetBWT` wraps a handle for convenience.  Host arrays are numpy
arrays (or raw addresses of pinned host memory); device arrays are raw
device addresses (e.g. ``torch.Tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsbwt.so")

SBWT_OK = 0
SBWT_EINVAL = -1
SBWT_ENOMEM = -2
SBWT_ERANGE = -3
SBWT_EDEVICE = -4
SBWT_ENOTSUP = -5
SBWT_EBUSY = -6
SBWT_ETIMEDOUT = -7
SBWT_EIO = -8

SBWT_STAGE_SA = 0
SBWT_STAGE_BINT = 1
SBWT_STAGE_G = 2
SBWT_STAGE_GSA = 3

#: every symbol include/sbwt.h declares, in header order
EXPORTS = (
    "sbwt_create", "sbwt_create_ex", "sbwt_append", "sbwt_prepend", "sbwt_append_device", "sbwt_get_bwt", "sbwt_rank",
    "sbwt_rank_batch", "sbwt_count", "sbwt_memory", "sbwt_size", "sbwt_reset", "sbwt_destroy", "sbwt_strerror",
    "sbwt_get_stream", "sbwt_set_capture", "sbwt_get_stage", "sbwt_set_profiling", "sbwt_set_profiling_only",
    "sbwt_get_kernel_stats", "sbwt_reset_kernel_stats", "sbwt_set_graph_replay", "sbwt_measure_bandwidth",
    "sbwt_set_block_overlap", "sbwt_autotune_block_suffixes", "sbwt_set_tile_shapes", "sbwt_get_tile_shapes",
    "sbwt_autotune_tile_shapes", "sbwt_autotune", "sbwt_serve_start", "sbwt_submit",
    "sbwt_wait", "sbwt_serve_stop", "sbwt_save", "sbwt_load", "sbwt_bwt_noalloc",
)

#: most suffixes (reads + one terminator each) sbwt_bwt_noalloc accepts
SBWT_NOALLOC_MAX_SUFFIXES = 1 << 18


class SbwtError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class sbwt_options(ctypes.Structure):
    _fields_ = [("index_bits", ctypes.c_uint32), ("block_suffixes", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int32), ("host_tier", ctypes.c_uint32),
                ("occ_sampling", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 6)]


class sbwt_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile libsbwt.so in-tree (nvcc, sm_103a)."""
    from . import _build
    return _build.build()


def load() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1410_0562_gb300.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P, U64, I, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
        sig = {
            "sbwt_create": ([ctypes.c_char_p, SZ, ctypes.POINTER(P)], I),
            "sbwt_create_ex": ([ctypes.c_char_p, SZ, ctypes.POINTER(sbwt_options), ctypes.POINTER(P)], I),
            "sbwt_append": ([P, P, P, U64], I),
            "sbwt_prepend": ([P, P, P, U64], I),
            "sbwt_append_device": ([P, P, P, U64], I),
            "sbwt_get_bwt": ([P, P, U64, ctypes.POINTER(U64)], I),
            "sbwt_rank": ([P, ctypes.c_uint8, U64, ctypes.POINTER(U64)], I),
            "sbwt_rank_batch": ([P, P, P, U64, P], I),
            "sbwt_count": ([P, P, P, U64, P], I),
            "sbwt_size": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64)], I),
            "sbwt_memory": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64)], I),
            "sbwt_reset": ([P], I),
            "sbwt_destroy": ([P], None),
            "sbwt_strerror": ([I], ctypes.c_char_p),
            "sbwt_get_stream": ([P, ctypes.POINTER(P)], I),
            "sbwt_set_capture": ([P, I], I),
            "sbwt_get_stage": ([P, I, P, U64, ctypes.POINTER(U64)], I),
            "sbwt_set_profiling": ([P, I], I),
            "sbwt_set_profiling_only": ([P, ctypes.c_char_p], I),
            "sbwt_get_kernel_stats": ([P, ctypes.POINTER(sbwt_kernel_stat), I, ctypes.POINTER(I)], I),
            "sbwt_reset_kernel_stats": ([P], I),
            "sbwt_set_graph_replay": ([P, I], I),
            "sbwt_set_block_overlap": ([P, I], I),
            "sbwt_set_tile_shapes": ([P, P], I),
            "sbwt_get_tile_shapes": ([P, P], I),
            "sbwt_autotune_tile_shapes": ([P, P, P, U64, P, I, P, P], I),
            "sbwt_measure_bandwidth": ([P, P], I),
            "sbwt_autotune_block_suffixes": ([P, P, P, U64, P, I, ctypes.POINTER(U64), P], I),
            "sbwt_autotune": ([P, P, P, U64, P, I, P, I, ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_uint32), P],
                              I),
            "sbwt_serve_start": ([P, U64], I),
            "sbwt_submit": ([P, P, P, U64, ctypes.POINTER(U64)], I),
            "sbwt_wait": ([P, U64, U64, ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_double)], I),
            "sbwt_serve_stop": ([P], I),
            "sbwt_save": ([P, ctypes.c_char_p], I),
            "sbwt_load": ([ctypes.c_char_p, SZ, ctypes.POINTER(sbwt_options), ctypes.POINTER(P)], I),
            "sbwt_bwt_noalloc": ([ctypes.c_char_p, P, P, U64, P, U64, ctypes.POINTER(U64), P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def strerror(code: int) -> str:
    return load().sbwt_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != SBWT_OK:
        raise SbwtError(rc, what)


def _host_ptr(a, dtype):
    """(pointer, keepalive) for a numpy array or a raw host address."""
    if isinstance(a, int):
        return ctypes.c_void_p(a), None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


# ---- the C ABI, one Python function per entry point ----------------------

def sbwt_create(alphabet: bytes = b"ACGT", hbm_budget: int = 0):
    h = ctypes.c_void_p()
    _check(load().sbwt_create(alphabet, hbm_budget, ctypes.byref(h)), "sbwt_create")
    return h


def sbwt_save(h, path) -> None:
    """Writes the committed index to the file `path`."""
    _check(load().sbwt_save(h, os.fsencode(path)), "sbwt_save")


def sbwt_load(path, hbm_budget: int = 0, index_bits: int = 0, block_suffixes: int = 0, stream: int = 0,
              device: int = -1, host_tier: int = 0, occ_sampling: int = 0):
    """A new index handle built from a file written by sbwt_save."""
    opt = sbwt_options(index_bits, block_suffixes, stream or None, device, host_tier, occ_sampling)
    out = ctypes.c_void_p()
    _check(load().sbwt_load(os.fsencode(path), hbm_budget, ctypes.byref(opt), ctypes.byref(out)), "sbwt_load")
    return out


def sbwt_create_ex(alphabet: bytes = b"ACGT", hbm_budget: int = 0, index_bits: int = 0, block_suffixes: int = 0,
                   stream: int = 0, device: int = -1, host_tier: int = 0, occ_sampling: int = 0):
    opt = sbwt_options(index_bits, block_suffixes, stream or None, device, host_tier, occ_sampling)
    h = ctypes.c_void_p()
    _check(load().sbwt_create_ex(alphabet, hbm_budget, ctypes.byref(opt), ctypes.byref(h)), "sbwt_create_ex")
    return h


def sbwt_append(h, reads, offsets, m: int | None = None):
    rp, rk = _host_ptr(reads, np.uint8)
    op, ok = _host_ptr(offsets, np.uint64)
    if m is None:
        m = len(ok) - 1
    _check(load().sbwt_append(h, rp, op, m), "sbwt_append")


def sbwt_prepend(h, reads, offsets, m: int | None = None):
    rp, rk = _host_ptr(reads, np.uint8)
    op, ok = _host_ptr(offsets, np.uint64)
    if m is None:
        m = len(ok) - 1
    _check(load().sbwt_prepend(h, rp, op, m), "sbwt_prepend")


def sbwt_append_device(h, d_reads: int, d_offsets: int, m: int):
    _check(load().sbwt_append_device(h, ctypes.c_void_p(d_reads), ctypes.c_void_p(d_offsets), m),
           "sbwt_append_device")


def sbwt_size(h):
    n, m = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().sbwt_size(h, ctypes.byref(n), ctypes.byref(m)), "sbwt_size")
    return n.value, m.value


def sbwt_memory(h):
    """(HBM bytes, host-tier bytes) the index holds."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().sbwt_memory(h, ctypes.byref(a), ctypes.byref(b)), "sbwt_memory")
    return a.value, b.value


def sbwt_get_bwt(h) -> np.ndarray:
    n, _ = sbwt_size(h)
    out = np.zeros(max(n, 1), dtype=np.uint8)
    got = ctypes.c_uint64()
    _check(load().sbwt_get_bwt(h, ctypes.c_void_p(out.ctypes.data), n, ctypes.byref(got)), "sbwt_get_bwt")
    return out[: got.value]


def sbwt_rank(h, c: int, k: int) -> int:
    out = ctypes.c_uint64()
    _check(load().sbwt_rank(h, c, k, ctypes.byref(out)), "sbwt_rank")
    return out.value


def sbwt_rank_batch(h, cs, ks) -> np.ndarray:
    cs = np.ascontiguousarray(cs, dtype=np.uint8)
    ks = np.ascontiguousarray(ks, dtype=np.uint64)
    out = np.zeros(max(len(ks), 1), dtype=np.uint64)
    _check(load().sbwt_rank_batch(h, ctypes.c_void_p(cs.ctypes.data), ctypes.c_void_p(ks.ctypes.data), len(ks),
                                  ctypes.c_void_p(out.ctypes.data)), "sbwt_rank_batch")
    return out[: len(ks)]


def sbwt_count(h, patterns) -> np.ndarray:
    """Occurrences of each pattern (a list of bytes) in the indexed reads."""
    data = b"".join(patterns)
    offs = np.zeros(len(patterns) + 1, dtype=np.uint64)
    np.cumsum([len(p) for p in patterns], out=offs[1:])
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, np.uint8)
    out = np.zeros(max(len(patterns), 1), dtype=np.uint64)
    _check(load().sbwt_count(h, ctypes.c_void_p(buf.ctypes.data), ctypes.c_void_p(offs.ctypes.data),
                             len(patterns), ctypes.c_void_p(out.ctypes.data)), "sbwt_count")
    return out[: len(patterns)]


def sbwt_reset(h):
    _check(load().sbwt_reset(h), "sbwt_reset")


def sbwt_destroy(h):
    load().sbwt_destroy(h)


def sbwt_get_stream(h) -> int:
    s = ctypes.c_void_p()
    _check(load().sbwt_get_stream(h, ctypes.byref(s)), "sbwt_get_stream")
    return s.value or 0


def sbwt_set_capture(h, on: bool):
    _check(load().sbwt_set_capture(h, int(on)), "sbwt_set_capture")


_STAGE_DTYPE = {SBWT_STAGE_SA: np.uint32, SBWT_STAGE_BINT: np.uint8, SBWT_STAGE_G: np.uint64,
                SBWT_STAGE_GSA: np.uint64}


def sbwt_get_stage(h, stage: int) -> np.ndarray:
    cnt = ctypes.c_uint64()
    rc = load().sbwt_get_stage(h, stage, None, 0, ctypes.byref(cnt))
    if rc not in (SBWT_OK, SBWT_ERANGE):
        _check(rc, "sbwt_get_stage")
    dt = _STAGE_DTYPE[stage]
    out = np.zeros(max(cnt.value, 1), dtype=dt)
    _check(load().sbwt_get_stage(h, stage, ctypes.c_void_p(out.ctypes.data), out.nbytes, ctypes.byref(cnt)),
           "sbwt_get_stage")
    return out[: cnt.value]


def sbwt_set_profiling(h, on: bool):
    _check(load().sbwt_set_profiling(h, int(on)), "sbwt_set_profiling")


def sbwt_set_profiling_only(h, kernel: str):
    _check(load().sbwt_set_profiling_only(h, kernel.encode()), "sbwt_set_profiling_only")


def sbwt_get_kernel_stats(h) -> list:
    n = ctypes.c_int()
    _check(load().sbwt_get_kernel_stats(h, None, 0, ctypes.byref(n)), "sbwt_get_kernel_stats")
    arr = (sbwt_kernel_stat * max(n.value, 1))()
    _check(load().sbwt_get_kernel_stats(h, arr, n.value, ctypes.byref(n)), "sbwt_get_kernel_stats")
    return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "ms": float(arr[i].ms),
             "bytes": float(arr[i].bytes)} for i in range(n.value)]


def sbwt_reset_kernel_stats(h):
    _check(load().sbwt_reset_kernel_stats(h), "sbwt_reset_kernel_stats")


class sbwt_bandwidth(ctypes.Structure):
    _fields_ = [("h2d_gbs", ctypes.c_double), ("d2h_gbs", ctypes.c_double), ("host_random_gbs", ctypes.c_double),
                ("hbm_random_gbs", ctypes.c_double)]


def sbwt_measure_bandwidth(h) -> dict:
    """H2D / D2H copy GB/s over the host link and random 32-byte read GB/s
    from pinned host memory and from HBM, on the index's device."""
    b = sbwt_bandwidth()
    _check(load().sbwt_measure_bandwidth(h, ctypes.byref(b)), "sbwt_measure_bandwidth")
    return {"h2d_GBps": b.h2d_gbs, "d2h_GBps": b.d2h_gbs, "host_random_32B_GBps": b.host_random_gbs,
            "hbm_random_32B_GBps": b.hbm_random_gbs}


class sbwt_tile_shapes(ctypes.Structure):
    _fields_ = [("insert_threads", ctypes.c_uint32), ("rank_segment", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


def sbwt_set_tile_shapes(h, insert_threads: int = 0, rank_segment: int = 0):
    _check(load().sbwt_set_tile_shapes(h, ctypes.byref(sbwt_tile_shapes(insert_threads, rank_segment))),
           "sbwt_set_tile_shapes")


def sbwt_get_tile_shapes(h):
    t = sbwt_tile_shapes()
    _check(load().sbwt_get_tile_shapes(h, ctypes.byref(t)), "sbwt_get_tile_shapes")
    return t.insert_threads, t.rank_segment


def sbwt_autotune_tile_shapes(h, d_reads: int, d_offsets: int, m: int, candidates=None):
    """Returns ((insert_threads, rank_segment) kept, {shape: ms}); candidates
    is a list of (insert_threads, rank_segment) pairs, None for the defaults."""
    n = len(candidates) if candidates is not None else 0
    arr = (sbwt_tile_shapes * max(n, 1))(*[sbwt_tile_shapes(a, b) for a, b in (candidates or [])])
    ms = np.zeros(max(n, 5), dtype=np.float64)
    best = sbwt_tile_shapes()
    _check(load().sbwt_autotune_tile_shapes(h, ctypes.c_void_p(d_reads), ctypes.c_void_p(d_offsets), m,
                                            arr if n else None, n, ctypes.byref(best),
                                            ctypes.c_void_p(ms.ctypes.data)), "sbwt_autotune_tile_shapes")
    shapes = candidates if n else [(0, 256), (256, 256), (512, 256), (0, 512), (0, 1024)]
    return (best.insert_threads, best.rank_segment), {tuple(c): float(t) for c, t in zip(shapes, ms)}


def sbwt_set_block_overlap(h, on: bool):
    _check(load().sbwt_set_block_overlap(h, int(on)), "sbwt_set_block_overlap")


def sbwt_set_graph_replay(h, on: bool):
    _check(load().sbwt_set_graph_replay(h, int(on)), "sbwt_set_graph_replay")


def sbwt_autotune_block_suffixes(h, d_reads: int, d_offsets: int, m: int, candidates=None):
    """Returns (best M, {M: ms}) after timing each candidate block size."""
    cands = np.ascontiguousarray(candidates if candidates is not None else
                                 [1 << 22, 1 << 23, 1 << 24, 1 << 25, 1 << 26, 1 << 27], dtype=np.uint64)
    ms = np.zeros(len(cands), dtype=np.float64)
    best = ctypes.c_uint64()
    _check(load().sbwt_autotune_block_suffixes(h, ctypes.c_void_p(d_reads), ctypes.c_void_p(d_offsets), m,
                                               ctypes.c_void_p(cands.ctypes.data), len(cands), ctypes.byref(best),
                                               ctypes.c_void_p(ms.ctypes.data)), "sbwt_autotune_block_suffixes")
    return best.value, {int(c): float(t) for c, t in zip(cands, ms)}


def sbwt_autotune(h, d_reads: int, d_offsets: int, m: int, block_suffixes=None, samplings=None):
    """Returns (best M, best occurrence sampling, {(sampling, M): ms}) after
    timing every pair of candidates; the index keeps the best pair."""
    Ms = np.ascontiguousarray(block_suffixes if block_suffixes is not None else
                              [1 << 22, 1 << 23, 1 << 24, 1 << 25, 1 << 26, 1 << 27], dtype=np.uint64)
    Ss = np.ascontiguousarray(samplings if samplings is not None else [64, 128, 256], dtype=np.uint32)
    ms = np.zeros(len(Ms) * len(Ss), dtype=np.float64)
    best_m, best_s = ctypes.c_uint64(), ctypes.c_uint32()
    _check(load().sbwt_autotune(h, ctypes.c_void_p(d_reads), ctypes.c_void_p(d_offsets), m,
                                ctypes.c_void_p(Ms.ctypes.data), len(Ms), ctypes.c_void_p(Ss.ctypes.data), len(Ss),
                                ctypes.byref(best_m), ctypes.byref(best_s), ctypes.c_void_p(ms.ctypes.data)),
           "sbwt_autotune")
    times = {(int(s_), int(m_)): float(ms[i * len(Ms) + j]) for i, s_ in enumerate(Ss) for j, m_ in enumerate(Ms)}
    return best_m.value, best_s.value, times


def sbwt_bwt_noalloc(alphabet: bytes, reads, offsets, stream: int = 0) -> np.ndarray:
    """B of a small read set computed without any device allocation (for
    callers whose device memory is owned by someone else); at most
    SBWT_NOALLOC_MAX_SUFFIXES suffixes."""
    rp, rk = _host_ptr(reads, np.uint8)
    op, ok = _host_ptr(offsets, np.uint64)
    m = len(ok) - 1
    n = int(ok[-1]) + m
    out = np.zeros(max(n, 1), dtype=np.uint8)
    got = ctypes.c_uint64()
    _check(load().sbwt_bwt_noalloc(alphabet, rp, op, m, ctypes.c_void_p(out.ctypes.data), n, ctypes.byref(got),
                                   ctypes.c_void_p(stream or None)), "sbwt_bwt_noalloc")
    return out[: got.value]


def sbwt_serve_start(h, max_batch_bases: int = 0):
    _check(load().sbwt_serve_start(h, max_batch_bases), "sbwt_serve_start")


def sbwt_submit(h, reads, offsets) -> int:
    rp, rk = _host_ptr(reads, np.uint8)
    op, ok = _host_ptr(offsets, np.uint64)
    t = ctypes.c_uint64()
    _check(load().sbwt_submit(h, rp, op, len(ok) - 1, ctypes.byref(t)), "sbwt_submit")
    return t.value


def sbwt_wait(h, ticket: int, timeout_us: int = 600_000_000):
    """(status, first read id, latency ms); status is an SBWT_* code."""
    first, lat = ctypes.c_uint64(), ctypes.c_double()
    rc = load().sbwt_wait(h, ticket, timeout_us, ctypes.byref(first), ctypes.byref(lat))
    return rc, first.value, lat.value


def sbwt_serve_stop(h):
    _check(load().sbwt_serve_stop(h), "sbwt_serve_stop")


class SetBWT:
    """An index handle: ``SetBWT(b"ACGT").append(reads, offsets).bwt()``."""

    def __init__(self, alphabet: bytes = b"ACGT", hbm_budget: int = 0, index_bits: int = 0,
                 block_suffixes: int = 0, stream: int = 0, device: int = -1, host_tier: int = 0,
                 occ_sampling: int = 0):
        self.alphabet = alphabet
        self._h = sbwt_create_ex(alphabet, hbm_budget, index_bits, block_suffixes, stream, device, host_tier,
                                 occ_sampling)

    @classmethod
    def load(cls, path, hbm_budget: int = 0, index_bits: int = 0, block_suffixes: int = 0, stream: int = 0,
             device: int = -1, host_tier: int = 0, occ_sampling: int = 0) -> "SetBWT":
        """An index read from a file that save() wrote."""
        self = cls.__new__(cls)
        self._h = sbwt_load(path, hbm_budget, index_bits, block_suffixes, stream, device, host_tier, occ_sampling)
        self.alphabet = None
        return self

    def save(self, path) -> "SetBWT":
        sbwt_save(self._h, path)
        return self

    @property
    def handle(self):
        return self._h

    def append(self, reads, offsets, m: int | None = None) -> "SetBWT":
        sbwt_append(self._h, reads, offsets, m)
        return self

    def prepend(self, reads, offsets, m: int | None = None) -> "SetBWT":
        """The reads go before every read already in the index."""
        sbwt_prepend(self._h, reads, offsets, m)
        return self

    def append_device(self, d_reads: int, d_offsets: int, m: int) -> "SetBWT":
        sbwt_append_device(self._h, d_reads, d_offsets, m)
        return self

    def bwt(self) -> np.ndarray:
        return sbwt_get_bwt(self._h)

    def rank(self, c, k: int) -> int:
        return sbwt_rank(self._h, c if isinstance(c, int) else ord(c), k)

    def rank_batch(self, cs, ks) -> np.ndarray:
        return sbwt_rank_batch(self._h, cs, ks)

    def count(self, patterns) -> np.ndarray:
        return sbwt_count(self._h, patterns)

    def size(self):
        return sbwt_size(self._h)

    def reset(self):
        sbwt_reset(self._h)

    def close(self):
        if self._h is not None:
            sbwt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
