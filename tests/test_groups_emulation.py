"""The device-wide path's bookkeeping (csrc/suffix_sort.cu) run on the CPU.

Units too large for a CTA are sorted by one device-wide radix sort per
doubling round.  Around that sort, `sa_round_keys` gives each unsorted
member t the key (rank[t], rank[t + h]) (Larsson-Sadakane's doubling; t + h
past the block is an error).  After it, the group pass walks the sorted
list, whose element i sits on row act_pos_in[i] (rows increase along the
list).  A group is a maximal run of equal keys; in the initial list a key
that ends at its terminator (length field below 29) is a group of its own.
The pass writes SA[row] = t, sets rank[t] to the row of its group's first
element, and lists the members of groups with two or more elements, in
order, as the next round's members.  It works by reduce-then-scan over
chunks of whole tiles of 4096 elements.

Checked against those definitions in numpy, over several grids (chunks
holding one or more tiles, empty chunks) and a ragged last tile.  The
kernels' text is cut out of the CUDA source and compiled for the host with
tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "groups_emulation.cpp")
kH0 = 29
SENT = 0xABCDEF


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("groupsemu")
    src = open(os.path.join(CSRC, "suffix_sort.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "scan.inc").write_text(_cut(hdr, "struct SumOp {", "// Launch bookkeeping"))
    (d / "constants.inc").write_text(_cut(src, "constexpr int kThreads = 256;", "// Key geometry per code width"))
    (d / "groups.inc").write_text(_cut(src, "__global__ void __launch_bounds__(kThreads) sa_round_keys_kernel(",
                                       "constexpr size_t kLocalSortSmem"))
    lib = d / "libgroupsemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U32, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    L.emu_round_keys.argtypes = [P, U32, P, U32, U32, I, P, P, P, ctypes.c_uint]
    L.emu_groups.argtypes = [I, P, P, P, U32, U32, P, P, P, P, P, P, ctypes.c_uint]
    L.emu_round_keys.restype = I
    L.emu_groups.restype = I
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def test_round_keys(emu):
    rng = np.random.default_rng(1)
    n, h, bits = 50_000, 58, 16
    rank = rng.integers(0, 1 << bits, size=n).astype(np.uint32)
    act = rng.choice(n - h, size=9000, replace=False).astype(np.uint32)
    keys = np.zeros(act.size, np.uint64)
    vals = np.zeros(act.size, np.uint32)
    err = np.zeros(1, np.uint32)
    assert emu.emu_round_keys(_p(act), act.size, _p(rank), h, n, bits, _p(keys), _p(vals), _p(err), 5) == 0
    want = (rank[act].astype(np.uint64) << np.uint64(bits)) | rank[act + h].astype(np.uint64)
    assert err[0] == 0 and np.array_equal(keys, want) and np.array_equal(vals, act)
    # a member without h symbols after it is an error of the caller
    act[7] = n - 3
    assert emu.emu_round_keys(_p(act), act.size, _p(rank), h, n, bits, _p(keys), _p(vals), _p(err), 5) == 0
    assert err[0] & 4


def make_list(rng, cnt, init):
    """A key-sorted list with runs of equal keys, its elements on increasing
    rows (with gaps) and distinct suffixes t."""
    run = rng.geometric(0.35, size=cnt)  # run lengths, many of one element
    starts = np.cumsum(run)
    gid = np.searchsorted(starts, np.arange(cnt), side="right")
    base = np.cumsum(rng.integers(1, 50, size=gid.max() + 1)).astype(np.uint64)
    keys = base[gid] << np.uint64(5)
    if init:
        # the length field: terminated keys (below kH0) are groups of their own
        field = np.where(rng.random(gid.max() + 1) < 0.3, rng.integers(0, kH0, size=gid.max() + 1), kH0)
        keys |= field[gid].astype(np.uint64)
    else:
        keys |= np.uint64(kH0)
    n_block = cnt * 3 + 100
    rows = np.sort(rng.choice(n_block, size=cnt, replace=False)).astype(np.uint32)
    vals = rng.choice(n_block, size=cnt, replace=False).astype(np.uint32)
    return keys, vals, rows, n_block


def expected(keys, vals, rows, n_block, init):
    cnt = keys.size
    head = np.ones(cnt, bool)
    head[1:] = keys[1:] != keys[:-1]
    if init:
        head |= (keys & np.uint64(31)) < np.uint64(kH0)
    gstart = np.maximum.accumulate(np.where(head, np.arange(cnt), 0))
    end = np.ones(cnt, bool)
    end[:-1] = head[1:]
    single = head & end
    sa = np.full(n_block, SENT, np.uint32)
    rank = np.full(n_block, SENT, np.uint32)
    sa[rows] = vals
    rank[vals] = rows[gstart]
    keep = ~single
    return sa, rank, rows[keep], vals[keep]


@pytest.mark.timeout(600)
@pytest.mark.parametrize("init", [True, False])
@pytest.mark.parametrize("cnt,grid", [(1, 1), (4095, 2), (4097, 1), (23_000, 1), (23_000, 3), (23_000, 12)])
def test_group_pass(emu, init, cnt, grid):
    rng = np.random.default_rng(cnt * 7 + grid + init)
    keys, vals, rows, n_block = make_list(rng, cnt, init)
    sa = np.full(n_block, SENT, np.uint32)
    rank = np.full(n_block, SENT, np.uint32)
    pos_out = np.full(n_block, SENT, np.uint32)
    suf_out = np.full(n_block, SENT, np.uint32)
    cnt_out = np.zeros(1, np.uint32)
    err = np.zeros(1, np.uint32)
    assert emu.emu_groups(int(init), _p(keys), _p(vals), _p(rows), cnt, n_block, _p(sa), _p(rank), _p(pos_out),
                          _p(suf_out), _p(cnt_out), _p(err), grid) == 0
    w_sa, w_rank, w_pos, w_suf = expected(keys, vals, rows, n_block, init)
    assert err[0] == 0
    assert np.array_equal(sa, w_sa) and np.array_equal(rank, w_rank)
    k = int(cnt_out[0])
    assert k == w_pos.size
    assert np.array_equal(pos_out[:k], w_pos) and np.array_equal(suf_out[:k], w_suf)
    assert np.all(pos_out[k:] == SENT)
