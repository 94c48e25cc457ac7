"""Insert's superblock-counter scan (csrc/insert.cu) run on the CPU.

After Insert (Section 5) writes a dictionary, each superblock's per-code
totals become the 64-bit counters of the codes before it (an exclusive
prefix sum over superblocks, per code), and C[c] = m + the number of
symbols with a smaller code (the m terminators sort first: Lemma 1's C).
One CTA does it for up to 2048 superblocks; beyond that three kernels scan
256-superblock chunks, scan the chunk totals (and write C), and add the
chunk offsets.

Checked against numpy's prefix sums for both forms and both code counts (4
for 2-bit codes, 16 for 4-bit), with totals near 2^31 so that the 64-bit
carries matter, and a superblock count that leaves the last chunk ragged.
The kernels' text is cut out of the CUDA source and compiled for the host
with tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "super_emulation.cpp")


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("superemu")
    src = open(os.path.join(CSRC, "insert.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "scan.inc").write_text(_cut(hdr, "struct SumOp {", "// Launch bookkeeping"))
    (d / "super.inc").write_text(_cut(src, "constexpr int kScanThreads = 256;",
                                      "template <int kCodes>\nvoid super_scan("))
    lib = d / "libsuperemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.emu_super_scan.argtypes = [I, P, U64, U64, I, P, P]
    L.emu_super_scan.restype = I
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("codes,nsb,force", [(4, 1, 0), (4, 300, 0), (4, 2048, 0), (4, 300, 1), (4, 2049, 0),
                                             (4, 5000, 0), (4, 70_000, 0), (16, 777, 0), (16, 2600, 0)])
def test_counters_and_C_are_prefix_sums(emu, codes, nsb, force):
    rng = np.random.default_rng(codes * 10_000 + nsb + force)
    sb_tot = rng.integers(0, 1 << 31, size=(nsb, codes), dtype=np.int64).astype(np.uint32)
    sb_tot[rng.random((nsb, codes)) < 0.2] = 0
    m = 123_456_789_012
    sup = np.full((nsb, codes), 0xABCDEF, np.uint64)
    C = np.zeros(codes, np.uint64)
    flat = np.ascontiguousarray(sb_tot)
    assert emu.emu_super_scan(codes, _p(flat), nsb, m, force, _p(sup), _p(C)) == 0
    t = sb_tot.astype(np.uint64)
    want = np.cumsum(t, axis=0, dtype=np.uint64) - t
    assert np.array_equal(sup, want)
    totals = t.sum(axis=0, dtype=np.uint64)
    want_C = np.uint64(m) + np.concatenate([[0], np.cumsum(totals, dtype=np.uint64)[:-1]]).astype(np.uint64)
    assert np.array_equal(C, want_C)
    assert int(want[-1].max() + t[-1].max()) > (1 << 32) or nsb < 3  # the 64-bit carries were exercised
