"""Insert (Section 5) for the 4-bit dictionary (alphabets of 5 to 16
symbols) run on the CPU.

The 4-bit dictionary keeps one 64-byte block per 64 rows: the rows' codes
(the symbol's index in the alphabet, 4 bits each, row q at bits 4 (q mod 16)
of word q / 16, a terminator stored as code 0), a terminator mask, and
sixteen 12-bit counts of each code (terminators excluded) from the start of
the block's superblock of 4096 rows.  Insert places new symbol i on row
g_sa[i] + i and the old rows in order around them, and returns each
superblock's code totals.

Checked against the oracle's Insert, packed here into that layout, on random
cases: an empty old index, all new symbols on one row, runs of equal g_sa,
sizes at block and superblock edges, and both index widths.  The kernel's
text is cut out of the CUDA source and compiled for the host with
tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "insert_w_emulation.cpp")
ALPHA = b"ABCGKMNRSTWY"  # 12 symbols, in increasing byte order
SUPER_ROWS_W = 4096


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("inswemu")
    ins = open(os.path.join(CSRC, "insert.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "dict.inc").write_text(_cut(hdr, "constexpr int kOccShift = 6;",
                                     "// rank(c, i) within i's superblock: the block counter"))
    (d / "dictw.inc").write_text(_cut(hdr, "constexpr int kSuperShiftW = 12;",
                                      "// rank(c, i) within i's superblock for the wide dictionary."))
    assert "constexpr int kThreads = 256;" in ins
    (d / "threads.inc").write_text("constexpr int kThreads = 256;\n")
    (d / "insert_w.inc").write_text(_cut(ins, "__device__ __forceinline__ unsigned long long funnel_r(",
                                         "constexpr int kScanThreads = 256;"))
    lib = d / "libinswemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.emu_insert_w.argtypes = [P, U64, P, P, I, U64, P, U64, P, P]
    L.emu_insert_w.restype = I
    return L


def codes_of(B: np.ndarray) -> np.ndarray:
    lut = np.zeros(256, np.int64)
    for i, c in enumerate(ALPHA):
        lut[c] = i
    return lut[B]


def pack_dict_w(B: np.ndarray) -> np.ndarray:
    """B (bytes over ALPHA and '$') in the 4-bit layout: 8 words per block
    (sym[0..3], dmask, cnt[0..2])."""
    n = len(B)
    nb = (n >> 6) + 1
    rows = nb * 64
    codes = np.zeros(rows, np.int64)
    dollar = np.zeros(rows, bool)
    dollar[:n] = B == ord("$")
    codes[:n] = np.where(dollar[:n], 0, codes_of(B))
    out = np.zeros((nb, 8), np.uint64)
    c4 = codes.reshape(nb, 4, 16).astype(np.uint64)
    sh = (4 * np.arange(16)).astype(np.uint64)
    out[:, 0:4] = np.bitwise_or.reduce(c4 << sh, axis=2)
    out[:, 4] = np.bitwise_or.reduce(dollar.reshape(nb, 64).astype(np.uint64) << np.arange(64).astype(np.uint64),
                                     axis=1)
    per_block = np.stack([((codes == c) & ~dollar).reshape(nb, 64).sum(axis=1) for c in range(16)], axis=1)
    excl = np.cumsum(per_block, axis=0) - per_block
    first = (np.arange(nb) // 64) * 64
    rel = excl - excl[first]  # counts from the superblock's start, below 4096
    assert rel.max(initial=0) < 4096
    # the sixteen 12-bit counts as one 192-bit field per block
    for b in range(nb):
        f = 0
        for c in range(16):
            f |= int(rel[b, c]) << (12 * c)
        out[b, 5] = f & (2 ** 64 - 1)
        out[b, 6] = (f >> 64) & (2 ** 64 - 1)
        out[b, 7] = f >> 128
    return out.ravel()


def super_totals_w(B: np.ndarray) -> np.ndarray:
    nsb = ((len(B) >> 6) + 1 + 63) // 64
    codes = codes_of(B)
    dollar = B == ord("$")
    tot = np.zeros((nsb, 16), np.uint32)
    for s in range(nsb):
        sl = slice(s * SUPER_ROWS_W, (s + 1) * SUPER_ROWS_W)
        c, d = codes[sl], dollar[sl]
        for x in range(16):
            tot[s, x] = np.count_nonzero((c == x) & ~d)
    return tot.ravel()


def random_case(rng, n_ext, n_int, kind, p_dollar=0.05):
    sym = np.frombuffer(ALPHA, np.uint8)
    B_ext = rng.choice(sym, size=n_ext)
    B_ext[rng.random(n_ext) < p_dollar] = ord("$")
    bint = rng.choice(sym, size=n_int)
    bint[rng.random(n_int) < p_dollar] = ord("$")
    if kind == "uniform":
        gsa = np.sort(rng.integers(0, n_ext + 1, size=n_int))
    elif kind == "clustered":
        anchors = np.sort(rng.integers(0, n_ext + 1, size=max(1, n_int // 200)))
        gsa = np.sort(rng.choice(anchors, size=n_int))
    else:
        gsa = np.full(n_int, int(rng.integers(0, n_ext + 1)))
    return B_ext.astype(np.uint8), bint.astype(np.uint8), gsa.astype(np.uint64)


def check(emu, B_ext, bint, gsa, width):
    n_ext, n_int = len(B_ext), len(bint)
    n_new = n_ext + n_int
    old = pack_dict_w(B_ext)
    codes = np.where(bint == ord("$"), 255, codes_of(bint)).astype(np.uint8)
    g = np.ascontiguousarray(gsa, np.uint32 if width == 4 else np.uint64)
    nb_new = (n_new >> 6) + 1
    nsb = (nb_new + 63) // 64
    new = np.zeros(nb_new * 8, np.uint64)
    tot = np.zeros(16 * nsb, np.uint32)
    err = ctypes.c_uint32(0)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_insert_w(p(old), n_ext, p(codes), p(g), width, n_int, p(new), n_new, p(tot),
                            ctypes.byref(err)) == 0
    expect = oracle.insert(B_ext, bint, gsa)
    assert err.value == 0
    want = pack_dict_w(expect)
    bad = np.nonzero(new != want)[0]
    assert len(bad) == 0, f"words differ at {bad[:8].tolist()} (8 words per block)"
    assert np.array_equal(tot, super_totals_w(expect))


@pytest.mark.timeout(600)
@pytest.mark.parametrize("n_ext,n_int,kind", [
    (0, 1, "uniform"), (0, 3000, "uniform"), (1, 1, "uniform"), (63, 2, "uniform"), (64, 64, "one"),
    (65, 200, "uniform"), (4095, 60, "uniform"), (4096, 9000, "clustered"), (3000, 3000, "one"),
    (20_000, 700, "uniform"), (12_000, 9_000, "clustered"),
])
def test_merge_matches_the_oracle(emu, n_ext, n_int, kind):
    rng = np.random.default_rng(n_ext * 11 + n_int)
    B_ext, bint, gsa = random_case(rng, n_ext, n_int, kind)
    check(emu, B_ext, bint, gsa, 4 if (n_ext + n_int) % 2 else 8)
