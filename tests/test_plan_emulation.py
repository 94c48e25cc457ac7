"""The append planning (csrc/plan.cu) run on the CPU.

Algorithm 1 builds the index block by block, each block some whole reads of
about M suffixes.  Read j's first suffix sits at text position
offsets[j] + j (every read is followed by its terminator), so reads
[j, j') hold (offsets[j'] + j') - (offsets[j] + j) suffixes.  The planner
checks the offsets first (they start at 0, never decrease, and no read with
its terminator exceeds the largest block; it also finds the longest read),
then cuts the blocks greedily: whole reads while the block holds at most M
suffixes, a read longer than M alone.

Checked against that greedy cut written as a plain loop over reads, with
empty reads, reads longer than M, a table too small for every block, and
bad offsets.  The kernels' text is cut out of the CUDA source and compiled
for the host with tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "plan_emulation.cpp")


class PlanBlock(ctypes.Structure):
    _fields_ = [("j0", ctypes.c_uint64), ("j1", ctypes.c_uint64), ("base", ctypes.c_uint64),
                ("n_int", ctypes.c_uint64)]


class PlanSummary(ctypes.Structure):
    _fields_ = [("bad", ctypes.c_uint32), ("blocks", ctypes.c_uint32), ("max_len", ctypes.c_uint64),
                ("npos", ctypes.c_uint64)]


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("planemu")
    src = open(os.path.join(CSRC, "plan.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_kernels.cuh")).read()
    (d / "plan_types.inc").write_text(_cut(hdr, "struct PlanBlock {", "void launch_plan("))
    (d / "plan.inc").write_text(_cut(src, "constexpr int kThreads = 256;", "}  // namespace\n"))
    lib = d / "libplanemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    L.emu_plan.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                           ctypes.c_uint, ctypes.POINTER(PlanSummary)]
    L.emu_plan.restype = ctypes.c_int
    return L


def greedy(offsets, M):
    """Blocks (j0, j1, base, n_int) read by read."""
    m = len(offsets) - 1
    rpos = [int(offsets[j]) + j for j in range(m + 1)]
    out, j = [], 0
    while j < m:
        e = j + 1
        while e < m and rpos[e + 1] - rpos[j] <= M:
            e += 1
        out.append((j, e, rpos[j], rpos[e] - rpos[j]))
        j = e
    return out


def plan(emu, offsets, M, max_block=1 << 31, cap=8192):
    table = (PlanBlock * cap)()
    s = PlanSummary()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    assert emu.emu_plan(ctypes.c_void_p(off.ctypes.data), len(off) - 1, M, max_block, table, cap,
                        ctypes.byref(s)) == 0
    return s, [(b.j0, b.j1, b.base, b.n_int) for b in table[:min(cap, s.blocks)]]


@pytest.mark.parametrize("m,M,seed", [(0, 100, 1), (1, 100, 2), (700, 1000, 3), (5000, 64, 4), (3000, 50_000, 5),
                                      (3000, 10 ** 9, 6)])
def test_greedy_blocks_and_longest_read(emu, m, M, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 120, size=m)
    if m > 10:
        lens[::97] = 0
        lens[5] = 3 * M if M < 10_000 else 150  # a read longer than M: a block alone
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    s, blocks = plan(emu, offsets, M)
    assert s.bad == 0
    assert s.max_len == (int(lens.max()) if m else 0)
    assert s.npos == int(offsets[-1]) + m
    want = greedy(offsets, M)
    assert s.blocks == len(want) and blocks == want
    # every read in exactly one block, blocks in order
    assert all(b[1] == c[0] for b, c in zip(want, want[1:]))


def test_table_smaller_than_the_block_count(emu):
    offsets = np.concatenate([[0], np.cumsum(np.full(400, 50))]).astype(np.uint64)
    s, blocks = plan(emu, offsets, 100, cap=7)
    want = greedy(offsets, 100)
    assert s.blocks == len(want) > 7 and blocks == want[:7]


@pytest.mark.parametrize("case", ["nonzero_start", "decreasing", "too_long"])
def test_bad_offsets_are_flagged_and_plan_nothing(emu, case):
    offsets = np.concatenate([[0], np.cumsum(np.full(600, 30))]).astype(np.uint64)
    max_block = 1 << 31
    if case == "nonzero_start":
        offsets = offsets + np.uint64(5)
    elif case == "decreasing":
        offsets[300] = offsets[299] - np.uint64(1)
    else:
        max_block = 30  # a 30-symbol read and its terminator need 31
    s, _ = plan(emu, offsets, 100, max_block=max_block)
    assert s.bad == 1 and s.blocks == 0
