"""The 2-bit Insert kernel (Section 5's stable merge) run on the CPU.

The text of ``insert_kernel`` and of the dictionary layout it writes is cut
out of csrc/insert.cu and csrc/sbwt_internal.cuh and compiled for the host
with tests/emu/cuda_emu.h (one thread per GPU thread, warp intrinsics and CTA
barriers emulated, every array between inaccessible pages).  Its output
dictionary is compared, word by word, with the oracle's Insert (new symbol
i on row g_sa[i] + i, the old rows in order around them) packed into the
same layout here: per 64-row part the low-bit, high-bit and terminator
planes, per occurrence block of 64, 128 or 256 rows the 16-bit counters
relative to the superblock, and the per-superblock totals.  The merge does not need a
BWT, so old rows, new symbols and the non-decreasing g_sa are drawn at
random, sparse, dense and clustered.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "insert_emulation.cpp")

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
SUPER_ROWS = 1 << 16


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("insemu")
    ins = open(os.path.join(CSRC, "insert.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "dict.inc").write_text(_cut(hdr, "constexpr int kOccShift = 6;",
                                     "// rank(c, i) within i's superblock: the block counter"))
    (d / "scan.inc").write_text(_cut(hdr, "struct SumOp {", "// Launch bookkeeping"))
    kern = _cut(ins, "constexpr int kThreads = 256;", "// ------------------------------------------------"
                                                      "---------------------------\n// The same merge")
    (d / "insert.inc").write_text(kern)
    lib = d / "libinsemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64 = ctypes.c_void_p, ctypes.c_uint64
    L.emu_insert.argtypes = [P, U64, P, P, ctypes.c_int, U64, P, P, U64, P, P, ctypes.c_int]
    L.emu_insert.restype = ctypes.c_int
    L.emu_insert_in_place.argtypes = [P, U64, P, P, ctypes.c_int, U64, P, U64, P, P, ctypes.c_int, U64]
    L.emu_insert_in_place.restype = ctypes.c_int
    L.emu_spread_old.argtypes = [P, U64, P]
    L.emu_spread_old.restype = None
    return L


def pack_dict(B: np.ndarray, k: int = 1) -> np.ndarray:
    """B (bytes over ACGT and '$') in the 2-bit dictionary layout, as 64-bit
    words: blocks of 64 k rows, each the (lo, hi, terminator) planes of its
    64-row parts, then the counts of each code before the block within its
    superblock of 2^16 rows (16 bits per code)."""
    n = len(B)
    nb = n // (64 * k) + 1
    rows = nb * 64 * k
    lut = np.zeros(256, np.uint64)
    for c, v in CODE.items():
        lut[c] = v
    codes = np.zeros(rows, np.uint64)
    dollar = np.zeros(rows, np.uint64)
    codes[:n] = lut[B]
    dollar[:n] = B == ord("$")
    sh = np.arange(64).astype(np.uint64)
    parts = lambda x: np.bitwise_or.reduce(x.reshape(-1, 64) << sh, axis=1).reshape(nb, k)  # noqa: E731
    lo, hi, dm = parts(codes & np.uint64(1)), parts(codes >> np.uint64(1)), parts(dollar)
    counts = np.stack([((codes == c) & (dollar == 0)).reshape(nb, -1).sum(axis=1) for c in range(4)],
                      axis=1).astype(np.int64)
    excl = np.cumsum(counts, axis=0) - counts
    per_super = SUPER_ROWS // (64 * k)
    first = (np.arange(nb) // per_super) * per_super
    rel = (excl - excl[first]).astype(np.uint64)
    out = np.zeros((nb, 3 * k + 1), np.uint64)
    out[:, 0:3 * k:3], out[:, 1:3 * k:3], out[:, 2:3 * k:3] = lo, hi, dm
    out[:, 3 * k] = rel[:, 0] | (rel[:, 1] << np.uint64(16)) | (rel[:, 2] << np.uint64(32)) | (rel[:, 3] << np.uint64(48))
    return out.ravel()


def super_totals(B: np.ndarray) -> np.ndarray:
    nsb = (len(B) >> 16) + 1
    tot = np.zeros((nsb, 4), np.uint32)
    for s in range(nsb):
        chunk = B[s * SUPER_ROWS:(s + 1) * SUPER_ROWS]
        for c, v in CODE.items():
            tot[s, v] = np.count_nonzero(chunk == c)
    return tot.ravel()


def plan(gsa: np.ndarray, n_new: int) -> np.ndarray:
    """First new symbol of every superblock: |{i : g_sa[i] + i < S * 2^16}|."""
    nsb = (n_new >> 16) + 1
    r = gsa.astype(np.int64) + np.arange(len(gsa))
    return np.searchsorted(r, np.arange(nsb + 1) * SUPER_ROWS, side="left").astype(np.uint32)


def run(emu, B_ext, bint, gsa, width=4, ins_plan=None, k=1):
    n_ext, n_int = len(B_ext), len(bint)
    n_new = n_ext + n_int
    old = pack_dict(B_ext, k)
    codes = np.array([255 if b == ord("$") else CODE[int(b)] for b in bint], np.uint8)
    g = np.ascontiguousarray(gsa, np.uint32 if width == 4 else np.uint64)
    p = plan(gsa, n_new) if ins_plan is None else ins_plan
    nsb = (n_new >> 16) + 1
    new = np.zeros((n_new // (64 * k) + 1) * (3 * k + 1), np.uint64)
    tot = np.zeros(4 * nsb, np.uint32)
    err = ctypes.c_uint32(0)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_insert(ptr(old), n_ext, ptr(codes), ptr(g), width, n_int, ptr(p), ptr(new), n_new, ptr(tot),
                          ctypes.byref(err), k) == 0
    return new, tot, err.value


def random_case(rng, n_ext, n_int, kind, p_dollar=0.05):
    sym = np.frombuffer(b"ACGT", np.uint8)
    B_ext = rng.choice(sym, size=n_ext)
    B_ext[rng.random(n_ext) < p_dollar] = ord("$")
    bint = rng.choice(sym, size=n_int)
    bint[rng.random(n_int) < p_dollar] = ord("$")
    if kind == "uniform":
        gsa = np.sort(rng.integers(0, n_ext + 1, size=n_int))
    elif kind == "clustered":  # runs of equal g_sa: long runs of consecutive new rows
        anchors = np.sort(rng.integers(0, n_ext + 1, size=max(1, n_int // 200)))
        gsa = np.sort(rng.choice(anchors, size=n_int))
    else:  # every new symbol at one place
        gsa = np.full(n_int, int(rng.integers(0, n_ext + 1)))
    return B_ext.astype(np.uint8), bint.astype(np.uint8), gsa.astype(np.uint64)


def check(emu, B_ext, bint, gsa, width=4, k=1):
    new, tot, err = run(emu, B_ext, bint, gsa, width, k=k)
    expect = oracle.insert(B_ext, bint, gsa)
    assert err == 0
    want = pack_dict(expect, k)
    bad = np.nonzero(new != want)[0]
    assert len(bad) == 0, f"words differ at {bad[:8].tolist()} (block of {3 * k + 1} words)"
    assert np.array_equal(tot, super_totals(expect))


def test_worked_example(emu):
    """The two-read example of the readings: B_ext = C$A after read AC; read
    A adds B_int = A$ at g_sa = [1, 1]; the result is CA$$A."""
    check(emu, np.frombuffer(b"", np.uint8), np.frombuffer(b"C$A", np.uint8), np.zeros(3, np.uint64))
    check(emu, np.frombuffer(b"C$A", np.uint8), np.frombuffer(b"A$", np.uint8), np.array([1, 1], np.uint64))
    assert bytes(oracle.insert(b"C$A", b"A$", [1, 1])) == b"CA$$A"


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("n_ext,n_int,kind", [
    (0, 1, "uniform"), (0, 5000, "uniform"), (1, 1, "uniform"), (63, 2, "uniform"), (64, 64, "one"),
    (65, 200, "uniform"), (4095, 60, "uniform"), (4096, 9000, "clustered"), (3000, 3000, "one"),
    (70_000, 700, "uniform"), (70_000, 25_000, "clustered"), (65_536 - 100, 300, "uniform"),
    (20_000, 110_000, "uniform"),
])
def test_merge_matches_the_oracle(emu, n_ext, n_int, kind, k):
    rng = np.random.default_rng(n_ext * 7 + n_int)
    B_ext, bint, gsa = random_case(rng, n_ext, n_int, kind)
    check(emu, B_ext, bint, gsa, width=4 if (n_ext + n_int) % 2 else 8, k=k)


def test_inconsistent_plan_is_flagged_without_leaving_the_arrays(emu):
    """A g_sa that is not non-decreasing (impossible from ComputeRanks) puts
    two new symbols on one row or outside their superblock: the kernel flags
    bit 10 and every access stays inside the arrays (guard pages)."""
    rng = np.random.default_rng(9)
    B_ext, bint, gsa = random_case(rng, 5000, 800, "uniform")
    bad = gsa.copy()[::-1].copy()  # decreasing
    _, _, err = run(emu, B_ext, bint, bad)
    assert err & 1024
    # a plan that names more new symbols than there are
    p = plan(gsa, len(B_ext) + len(bint))
    p[-1] = len(bint) + 5
    _, _, err = run(emu, B_ext, bint, gsa, ins_plan=p)
    assert err & 1024


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("n_ext,n_int,kind,chunk", [
    (200_000, 3_000, "uniform", 1), (180_000, 90_000, "clustered", 2), (140_000, 5, "one", 1),
    (70_000, 200_000, "uniform", 1),
])
def test_in_place_merge_matches_the_oracle(emu, n_ext, n_int, kind, chunk, k):
    """The host tier's Insert rewrites the one dictionary in place, from the
    top superblock down in chunks, staging each chunk's old blocks first;
    chunks of one or two superblocks over dictionaries of three to five."""
    rng = np.random.default_rng(n_ext + n_int + chunk)
    B_ext, bint, gsa = random_case(rng, n_ext, n_int, kind)
    n_new = n_ext + n_int
    words = np.zeros((n_new // (64 * k) + 1) * (3 * k + 1), np.uint64)
    old = pack_dict(B_ext, k)
    words[: len(old)] = old
    codes = np.array([255 if b == ord("$") else CODE[int(b)] for b in bint], np.uint8)
    g = np.ascontiguousarray(gsa, np.uint32)
    p = plan(gsa, n_new)
    tot = np.zeros(4 * ((n_new >> 16) + 1), np.uint32)
    err = ctypes.c_uint32(0)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_insert_in_place(ptr(words), n_ext, ptr(codes), ptr(g), 4, n_int, ptr(p), n_new, ptr(tot),
                                   ctypes.byref(err), k, chunk) == 0
    expect = oracle.insert(B_ext, bint, gsa)
    assert err.value == 0
    bad = np.nonzero(words != pack_dict(expect, k))[0]
    assert len(bad) == 0, f"words differ at {bad[:8].tolist()}"
    assert np.array_equal(tot, super_totals(expect))


def test_spread_old_places_old_rows_in_order_around_the_new_ones(emu):
    """One output part: its old rows (the window's low 64 - k rows, on each
    of the three planes) fill the rows where F is clear, in order, and the
    rows of F stay empty -- for every k, so each of the three ways (opening
    rows one by one, the deposit network, placing the few old rows) is
    checked against a bit-by-bit reference."""
    rng = np.random.default_rng(77)
    inp = np.zeros(3, np.uint64)
    out = np.zeros(3, np.uint64)
    for k in list(range(65)) * 40:
        rows = rng.choice(64, size=k, replace=False)
        F = int(np.bitwise_or.reduce(np.left_shift(np.uint64(1), rows.astype(np.uint64)))) if k else 0
        inp[:] = rng.integers(0, 2**64, size=3, dtype=np.uint64)
        emu.emu_spread_old(inp.ctypes.data, F, out.ctypes.data)
        for plane in range(3):
            x, want, src = int(inp[plane]), 0, 0
            for p in range(64):
                if not (F >> p) & 1:
                    want |= ((x >> src) & 1) << p
                    src += 1
            assert int(out[plane]) == want, (k, plane, hex(F))
