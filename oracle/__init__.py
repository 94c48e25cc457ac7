"""CPU oracle for set-bwte (arXiv 1410.0562) -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
shares no code with it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, compiled with
gcc into ``liboracle.so`` next to it).  This module only marshals numpy
arrays into it.  Every function cites the passage of the paper it follows:

* :func:`bwt` -- Section 2, Eq. 1 with the terminator order
  ``$_0 < ... < $_{m-1} < c_1``: sort all suffixes of
  ``T = S_0 $_0 ... S_{m-1} $_{m-1}`` by direct comparison and read
  ``B[i] = T[(SA[i]-1) mod n]``.
* :func:`rank` -- Eq. 2, by counting.
* :func:`block_sa`, :func:`block_bint` -- Algorithm 1, ConstructSA and
  ``B(S_jk, SA_int)``.
* :func:`block_g_direct` -- the number of old suffixes below each block
  suffix (the quantity of Lemma 1, Section 4), by binary search.
* :func:`block_g_lemma1` -- Algorithm 2 (ComputeRanks) with Lemma 1 and the
  start value ``i := m_ext``.
* :func:`insert` -- Insert (Algorithm 1, Section 5) as a stable merge.
* :func:`setbwte` -- Algorithm 1 over given block boundaries.
* :func:`lf_invert`, :func:`lf_invert_sampled` -- recover the reads from B
  by LF steps.
* :func:`count` -- occurrences of a pattern, by direct comparison.
* :func:`row_of_suffix`, :func:`bwt_symbol_of_suffix` -- one suffix's row and
  B symbol, for sampled checks at large sizes.

Every function here is pinned by tests that do not reuse it: brute-force
rotation sorting, textbook BWTs, a hand-derived two-block example,
invariants and the block-partition identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
EINVAL = -1
ENOMEM = -2


def build_planted(plant: int, out_path: str) -> str:
    """Compile a copy of the oracle with deliberate mistake ``plant`` (see
    ORACLE_PLANT in oracle.c) into ``out_path``; used only by the tests that
    show the pins catch such mistakes."""
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", f"-DORACLE_PLANT={plant}", "-o",
                           out_path, _SRC])
    return out_path


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (plain -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _declare(lib):
    P = ctypes.c_void_p
    U64 = ctypes.c_uint64
    I = ctypes.c_int
    lib.oracle_bwt.argtypes = [P, P, U64, P, I, P]
    lib.oracle_bwt.restype = I
    lib.oracle_rank.argtypes = [P, U64, ctypes.c_uint8, U64]
    lib.oracle_rank.restype = U64
    lib.oracle_block_sa.argtypes = [P, P, U64, U64, P]
    lib.oracle_block_sa.restype = I
    lib.oracle_block_bint.argtypes = [P, P, U64, U64, P, U64, P]
    lib.oracle_block_bint.restype = I
    lib.oracle_block_g_direct.argtypes = [P, P, U64, U64, P]
    lib.oracle_block_g_direct.restype = I
    lib.oracle_block_g_lemma1.argtypes = [P, U64, P, P, U64, U64, P, I, P]
    lib.oracle_block_g_lemma1.restype = I
    lib.oracle_insert.argtypes = [P, U64, P, P, U64, P]
    lib.oracle_insert.restype = I
    lib.oracle_setbwte.argtypes = [P, P, U64, P, I, P, U64, P]
    lib.oracle_setbwte.restype = I
    lib.oracle_setbwte_reverse.argtypes = [P, P, U64, P, I, P, U64, P]
    lib.oracle_setbwte_reverse.restype = I
    lib.oracle_lf_invert.argtypes = [P, U64, U64, P, I, P, U64, P]
    lib.oracle_lf_invert.restype = I
    lib.oracle_lf_invert_sampled.argtypes = [P, U64, U64, P, I, P, U64, P]
    lib.oracle_lf_invert_sampled.restype = I
    lib.oracle_count.argtypes = [P, P, U64, P, U64]
    lib.oracle_count.restype = U64
    lib.oracle_row_of_suffix.argtypes = [P, P, U64, U64, U64]
    lib.oracle_row_of_suffix.restype = U64
    lib.oracle_bwt_symbol_of_suffix.argtypes = [P, P, U64, U64]
    lib.oracle_bwt_symbol_of_suffix.restype = ctypes.c_uint8
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIBRARY names another build of oracle.c (the planted-
            # mistake builds, in the tests that run the pins against them)
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIBRARY") or build())
            _declare(lib)
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8).copy()
    return np.ascontiguousarray(a, dtype=np.uint8)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with code {rc}")


def num_suffixes(offsets) -> int:
    offsets = _u64(offsets)
    return int(offsets[-1]) + (len(offsets) - 1)


def bwt(reads, offsets, alphabet: bytes = b"ACGT") -> np.ndarray:
    """B of the set, one byte per row ('$' for every terminator); Eq. 1."""
    reads, offsets, alpha = _u8(reads), _u64(offsets), _u8(alphabet)
    m = len(offsets) - 1
    out = np.zeros(max(num_suffixes(offsets), 1), dtype=np.uint8)
    _check(_load().oracle_bwt(_ptr(reads), _ptr(offsets), m, _ptr(alpha), len(alpha), _ptr(out)), "oracle_bwt")
    return out[: num_suffixes(offsets)]


def rank(B, c: int, k: int) -> int:
    """rank(c, k, B) = number of c among B[0..k) (Eq. 2)."""
    B = _u8(B)
    return int(_load().oracle_rank(_ptr(B), len(B), c, k))


def block_bounds_positions(offsets, j0: int, j1: int) -> int:
    offsets = _u64(offsets)
    return int(offsets[j1] - offsets[j0]) + (j1 - j0)


def block_sa(reads, offsets, j0: int, j1: int) -> np.ndarray:
    """SA_int of the block of reads [j0, j1), as block-local positions."""
    reads, offsets = _u8(reads), _u64(offsets)
    n = block_bounds_positions(offsets, j0, j1)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(_load().oracle_block_sa(_ptr(reads), _ptr(offsets), j0, j1, _ptr(out)), "oracle_block_sa")
    return out[:n]


def block_bint(reads, offsets, j0: int, j1: int, sa) -> np.ndarray:
    """B_int of the block: the symbol before each SA_int suffix ('$' at a read start)."""
    reads, offsets, sa = _u8(reads), _u64(offsets), _u64(sa)
    out = np.zeros(max(len(sa), 1), dtype=np.uint8)
    _check(_load().oracle_block_bint(_ptr(reads), _ptr(offsets), j0, j1, _ptr(sa), len(sa), _ptr(out)),
           "oracle_block_bint")
    return out[: len(sa)]


def block_g_direct(reads, offsets, j0: int, j1: int) -> np.ndarray:
    """g[t] = number of suffixes of reads [0, j0) smaller than block suffix t."""
    reads, offsets = _u8(reads), _u64(offsets)
    n = block_bounds_positions(offsets, j0, j1)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(_load().oracle_block_g_direct(_ptr(reads), _ptr(offsets), j0, j1, _ptr(out)), "oracle_block_g_direct")
    return out[:n]


def block_g_lemma1(B_ext, reads, offsets, j0: int, j1: int, alphabet: bytes = b"ACGT") -> np.ndarray:
    """g by Algorithm 2 (ComputeRanks, Lemma 1) over the given B_ext."""
    B_ext, reads, offsets, alpha = _u8(B_ext), _u8(reads), _u64(offsets), _u8(alphabet)
    n = block_bounds_positions(offsets, j0, j1)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    _check(_load().oracle_block_g_lemma1(_ptr(B_ext), len(B_ext), _ptr(reads), _ptr(offsets), j0, j1,
                                         _ptr(alpha), len(alpha), _ptr(out)), "oracle_block_g_lemma1")
    return out[:n]


def insert(B_ext, bint, g_sa) -> np.ndarray:
    """Insert: new symbol i on row g_sa[i]+i, old rows in order around them."""
    B_ext, bint, g_sa = _u8(B_ext), _u8(bint), _u64(g_sa)
    out = np.zeros(max(len(B_ext) + len(bint), 1), dtype=np.uint8)
    _check(_load().oracle_insert(_ptr(B_ext), len(B_ext), _ptr(bint), _ptr(g_sa), len(bint), _ptr(out)),
           "oracle_insert")
    return out[: len(B_ext) + len(bint)]


def setbwte(reads, offsets, bounds, alphabet: bytes = b"ACGT", reverse: bool = False) -> np.ndarray:
    """Algorithm 1 over block boundaries 0 = bounds[0] < ... < bounds[K] = m;
    reverse=True runs the blocks from the last to the first, each going
    before the reads already inserted (Algorithm 2 then starts at i := 0)."""
    reads, offsets, alpha, bounds = _u8(reads), _u64(offsets), _u8(alphabet), _u64(bounds)
    m = len(offsets) - 1
    n = num_suffixes(offsets)
    out = np.zeros(max(n, 1), dtype=np.uint8)
    fn = _load().oracle_setbwte_reverse if reverse else _load().oracle_setbwte
    _check(fn(_ptr(reads), _ptr(offsets), m, _ptr(alpha), len(alpha), _ptr(bounds), len(bounds) - 1, _ptr(out)),
           "oracle_setbwte")
    return out[:n]


def lf_invert(B, m: int, alphabet: bytes = b"ACGT"):
    """Recover (reads, offsets) from B by LF steps; raises on an inconsistent B."""
    B, alpha = _u8(B), _u8(alphabet)
    reads = np.zeros(max(len(B), 1), dtype=np.uint8)
    offsets = np.zeros(m + 1, dtype=np.uint64)
    _check(_load().oracle_lf_invert(_ptr(B), len(B), m, _ptr(alpha), len(alpha), _ptr(reads), len(reads),
                                    _ptr(offsets)), "oracle_lf_invert")
    return reads[: int(offsets[-1])], offsets


def lf_invert_sampled(B, m: int, alphabet: bytes = b"ACGT"):
    """lf_invert with rank counts every 64 rows (for large B)."""
    B, alpha = _u8(B), _u8(alphabet)
    reads = np.zeros(max(len(B), 1), dtype=np.uint8)
    offsets = np.zeros(m + 1, dtype=np.uint64)
    _check(_load().oracle_lf_invert_sampled(_ptr(B), len(B), m, _ptr(alpha), len(alpha), _ptr(reads), len(reads),
                                            _ptr(offsets)), "oracle_lf_invert_sampled")
    return reads[: int(offsets[-1])], offsets


def count(reads, offsets, pattern: bytes) -> int:
    """Occurrences of `pattern` in the reads, overlapping ones included."""
    reads, offsets, pat = _u8(reads), _u64(offsets), _u8(pattern)
    return int(_load().oracle_count(_ptr(reads), _ptr(offsets), len(offsets) - 1, _ptr(pat), len(pat)))


def row_of_suffix(reads, offsets, r: int, p: int) -> int:
    """Row of suffix (read r, offset p) among all suffixes of the set."""
    reads, offsets = _u8(reads), _u64(offsets)
    return int(_load().oracle_row_of_suffix(_ptr(reads), _ptr(offsets), len(offsets) - 1, r, p))


def bwt_symbol_of_suffix(reads, offsets, r: int, p: int) -> int:
    """The byte B holds on the row of suffix (r, p) (Eq. 1 for one suffix)."""
    reads, offsets = _u8(reads), _u64(offsets)
    return int(_load().oracle_bwt_symbol_of_suffix(_ptr(reads), _ptr(offsets), r, p))
