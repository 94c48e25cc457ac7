"""The unit scan and the local-sort kernels of the suffix sort, run on the CPU.

The text of the warp-per-unit kernels and of the CTA-batch kernels that take
the units they leave is cut out of csrc/suffix_sort.cu and compiled for the
host with tests/emu/warp_emulation.cpp: one thread per GPU thread, warp
intrinsics and CTA barriers emulated, every array between inaccessible
pages.  Synthetic block layouts (buckets of every size class, units that
span windows, units of the device-wide path) are sorted and the output is
compared with the contract both kernels share:

* initial local sort: inside every local unit the long rows are ordered by
  (key, t); the j-th of them goes to the unit's j-th long row; rank[t] is
  the row of its group's head (equal keys whose length field is the
  unresolved value, else the suffix alone); the members of groups of two or
  more are listed in row order from the unit's first row of loc_act, and
  their count is the unit's count and is added to the block total;
* one round: inside every unit's member list the members are ordered by
  (rank[t], rank[t + h], t); a member at offset x of the old group headed by
  row H takes row H + x, its rank is H plus the offset of its new group's
  first member, and the members of new groups of two or more are listed
  again in order;
* the unit scan (one CTA over the window table): each unit's end (the next
  unit's start) and long count, the unit owning each window's first row,
  the offsets of the device-wide units (over 2048 long rows) in window
  order, zeroed counts and round counters.

The inputs keep the order the pipeline guarantees: inside a bucket (and
inside an old group) the entries are in t order.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "warp_emulation.cpp")

kNone = 0xFFFFFFFF
kFallback = 0xFFFFFFFE
kH0 = 29
kWindow = 1024
kLCap = 2048
kWChunk = 256


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("emu")
    src = open(os.path.join(CSRC, "suffix_sort.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    dyn = "extern __shared__ __align__(16) unsigned char smem[];"
    parts = {
        "constants.inc": _cut(src, "constexpr int kThreads = 256;", "// Key geometry per code width"),
        "scan.inc": _cut(hdr, "struct SumOp {", "// Launch bookkeeping"),
        "unit_scan.inc": _cut(src, "// kScanPer consecutive windows of one field", "// one spare slot per kLItems"),
        "cta_local.inc": _cut(src, "// one spare slot per kLItems", "// Warp-per-unit local sort."),
        "warp_local.inc": _cut(src, "// Warp-per-unit local sort.", "// The global-path list:"),
        "round_gather.inc": _cut(src, "// next-ranks of the local unsorted members",
                                 "// One round for the local units, a batch of units per CTA step"),
        "cta_round.inc": _cut(src, "// One round for the local units, a batch of units per CTA step",
                              "// One round for the local units of at most kWChunk"),
        "warp_round.inc": _cut(src, "// One round for the local units of at most kWChunk",
                               "__global__ void __launch_bounds__(kThreads) sa_round_keys_kernel("),
    }
    for name, text in parts.items():
        (d / name).write_text(text.replace(dyn, "unsigned char* smem = g_dyn_smem;"))
    lib = d / "libwarpemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    return ctypes.CDLL(str(lib))


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


# ---- initial local sort ----------------------------------------------------

def make_block(rng, n_target, seg_shift, p_short=0.15, max_bucket=16, p_big=0.0, big=(257, 600), p_unres=0.6,
               low_range=(1, 8), p_hugeshort=0.0):
    """Rows of a digit-sorted block: buckets in order, each all short or all
    long; long keys share their bucket bits above seg_shift; t in order
    inside a bucket."""
    is_long, keys, starts = [], [], []
    bucket = 1
    n = 0
    while n < n_target:
        u = rng.random()
        if u < p_hugeshort:
            size, kind = int(rng.integers(1100, 3000)), "short"
        elif u < p_hugeshort + p_short:
            size, kind = int(rng.integers(1, 6)), "short"
        elif u < p_hugeshort + p_short + p_big:
            size, kind = int(rng.integers(*big)), "long"
        else:
            size, kind = int(rng.integers(1, max_bucket + 1)), "long"
        starts.append(n)
        span = int(rng.integers(*low_range))
        for _ in range(size):
            if kind == "long":
                lenf = kH0 if rng.random() < p_unres else int(rng.integers(0, kH0))
                keys.append((bucket << seg_shift) | (int(rng.integers(0, span)) << 5) | lenf)
                is_long.append(True)
            else:
                keys.append(0)
                is_long.append(False)
        n += size
        bucket += 1
    t_of_row = rng.permutation(n).astype(np.uint32)
    bounds = starts + [n]
    for a, b in zip(bounds, bounds[1:]):
        t_of_row[a:b] = np.sort(t_of_row[a:b])
    return n, np.array(is_long), np.array(keys, dtype=np.uint64), starts, t_of_row


def build_units(n, is_long, keys, starts, t_of_row):
    """The window table and the long-row lists, as the unit kernels make them."""
    nwin = (n + kWindow - 1) // kWindow
    is_start = np.zeros(n + 1, bool)
    is_start[starts] = True
    beg = np.full(nwin, kNone, np.uint32)
    lcb = np.zeros(nwin, np.uint32)
    lct = np.zeros(nwin, np.uint32)
    ll_t = np.zeros(n, np.uint32)
    ll_row = np.zeros(n, np.uint32)
    ll_key = np.zeros(n, np.uint64)
    for w in range(nwin):
        lo, hi = w * kWindow, min(n, (w + 1) * kWindow)
        k, first, before = 0, None, 0
        for i in range(lo, hi):
            if first is None and is_start[i]:
                first, before = i, k
            if is_long[i]:
                ll_t[lo + k], ll_row[lo + k], ll_key[lo + k] = t_of_row[i], i, keys[i]
                k += 1
        beg[w] = kNone if first is None else first
        lcb[w] = k if first is None else before
        lct[w] = k
    nlong = np.zeros(nwin, np.uint32)
    lofs = np.full(nwin, kNone, np.uint32)
    unit_ws = [w for w in range(nwin) if beg[w] != kNone]
    cum = np.concatenate([[0], np.cumsum(is_long)])
    ends = {}
    for a, w in enumerate(unit_ws):
        end = int(beg[unit_ws[a + 1]]) if a + 1 < len(unit_ws) else n
        ends[w] = end
        nlong[w] = cum[end] - cum[beg[w]]
        if nlong[w] > kLCap:
            lofs[w] = 0  # the device-wide path
    return nwin, beg, lcb, lct, nlong, lofs, ll_t, ll_row, ll_key, ends


def expected_local(n, is_long, keys, t_of_row, beg, nlong, lofs, ends):
    sa, rank, loc = {}, {}, {}
    for w, end in ends.items():
        if lofs[w] != kNone or nlong[w] == 0:
            continue
        rows = [i for i in range(int(beg[w]), end) if is_long[i]]
        items = sorted((int(keys[i]), int(t_of_row[i])) for i in rows)
        heads = [p == 0 or k != items[p - 1][0] or (k & 31) < kH0 for p, (k, _) in enumerate(items)]
        act, head_row = [], None
        for p, (k, t) in enumerate(items):
            if heads[p]:
                head_row = rows[p]
            sa[rows[p]] = t
            rank[t] = head_row
            if not (heads[p] and (p + 1 == len(items) or heads[p + 1])):
                act.append(t)
        loc[w] = act
    return sa, rank, loc


LOCAL_CASES = [
    dict(seed=11, n_target=8000),                                   # short-read-like buckets
    dict(seed=12, n_target=16000, p_big=0.02),                      # buckets over a warp chunk
    dict(seed=13, n_target=16000, p_big=0.01, p_hugeshort=0.01),    # units spanning windows
    dict(seed=14, n_target=16000, max_bucket=300, low_range=(1, 2)),
    dict(seed=15, n_target=16000, p_big=0.005, big=(2500, 4000)),   # device-wide units
    dict(seed=16, n_target=12000, seg_shift=33, p_big=0.01),        # the 4-bit codes' shift
    dict(seed=17, n_target=6000, max_bucket=1, p_short=0.0),        # singletons only
]


@pytest.mark.timeout(600)
@pytest.mark.parametrize("use_warp", [1, 0])
@pytest.mark.parametrize("case", LOCAL_CASES)
def test_local_sort(emu, case, use_warp):
    case = dict(case)
    seg_shift = case.pop("seg_shift", 41)
    rng = np.random.default_rng(case.pop("seed"))
    n, is_long, keys, starts, t_of_row = make_block(rng, case.pop("n_target"), seg_shift, **case)
    nwin, beg, lcb, lct, nlong, lofs, ll_t, ll_row, ll_key, ends = build_units(n, is_long, keys, starts, t_of_row)
    cnt = np.zeros(nwin, np.uint32)
    sa = np.full(n, kNone, np.uint32)
    rank = np.full(n, kNone, np.uint32)
    loc_act = np.full(n, kNone, np.uint32)
    d_cnt = np.zeros(1, np.uint32)
    d_err = np.zeros(1, np.uint32)
    emu.emu_local_sort(ctypes.c_uint32(n), _p(ll_t), _p(ll_row), _p(ll_key), _p(beg), _p(lcb), _p(lct), _p(nlong),
                       _p(lofs), _p(cnt), ctypes.c_uint32(nwin), _p(sa), _p(rank), _p(loc_act), _p(d_cnt), _p(d_err),
                       ctypes.c_int(seg_shift), ctypes.c_uint(2), ctypes.c_uint(3), ctypes.c_int(use_warp))
    e_sa, e_rank, e_loc = expected_local(n, is_long, keys, t_of_row, beg, nlong, lofs, ends)
    bad_sa = [r for r, t in e_sa.items() if sa[r] != t]
    bad_rank = [t for t, r in e_rank.items() if rank[t] != r]
    assert not bad_sa and not bad_rank, (bad_sa[:5], bad_rank[:5])
    for w, act in e_loc.items():
        assert cnt[w] == len(act)
        assert list(loc_act[beg[w]:beg[w] + len(act)]) == act
    assert int(d_cnt[0]) == sum(len(a) for a in e_loc.values())
    assert d_err[0] == 0
    for w, end in ends.items():  # units of the device-wide path are left alone
        if lofs[w] != kNone:
            assert cnt[w] == 0 and np.all(sa[beg[w]:end] == kNone)


# ---- one unit-local round ----------------------------------------------------

def make_round(rng, nwin=24, p_unit=0.7, p_global=0.1, max_group=12, next_range=3, big_units=0.1):
    n = nwin * kWindow
    beg = np.full(nwin, kNone, np.uint32)
    lofs = np.full(nwin, kNone, np.uint32)
    cnt = np.zeros(nwin, np.uint32)
    loc_act = np.full(n, 0xABCDEF01, np.uint32)
    loc_next = np.zeros(n, np.uint32)
    rank = np.full(n, kNone, np.uint32)
    perm = rng.permutation(n).astype(np.uint32)
    used = 0
    units = {}
    for w in range(nwin - 1):  # the last window stays free: every row stays inside n
        if rng.random() > p_unit:
            continue
        b0 = w * kWindow + int(rng.integers(0, 200))
        beg[w] = b0
        if rng.random() < p_global:
            lofs[w] = 0
            continue
        target = int(rng.integers(300, 900)) if rng.random() < big_units else int(rng.integers(0, 256))
        row = b0 + int(rng.integers(0, 5))
        members = []
        while len(members) < target:
            s = min(int(rng.integers(2, max_group + 1)), target - len(members))
            if s < 2:
                break
            ts = np.sort(perm[used:used + s])  # the previous pass listed each group in t order
            used += s
            rank[ts] = row
            members.extend(int(t) for t in ts)
            row += s + int(rng.integers(0, 3))
        cnt[w] = len(members)
        loc_act[b0:b0 + len(members)] = members
        loc_next[b0:b0 + len(members)] = rng.integers(0, next_range, size=len(members))
        units[w] = members
    return n, beg, lofs, cnt, loc_act, loc_next, rank, units


ROUND_CASES = [dict(seed=1), dict(seed=2, max_group=40, next_range=2), dict(seed=3, next_range=1),
               dict(seed=4, next_range=1000), dict(seed=5, max_group=256, next_range=4, big_units=0.3)]


@pytest.mark.timeout(600)
@pytest.mark.parametrize("case", ROUND_CASES)
def test_round(emu, case):
    case = dict(case)
    rng = np.random.default_rng(case.pop("seed"))
    n, beg, lofs, cnt, loc_act, loc_next, rank, units = make_round(rng, **case)
    rank0 = rank.copy()
    e_sa, e_rank, e_loc = {}, {}, {}
    for w, members in units.items():
        if not members:
            continue
        b0 = int(beg[w])
        items = sorted(((int(rank0[t]) << 32) | int(loc_next[b0 + k]), t) for k, t in enumerate(members))
        act = []
        for p, (key, t) in enumerate(items):
            here = key >> 32
            of = p
            while of and items[of - 1][0] >> 32 == here:
                of -= 1
            hf = p
            while hf and items[hf - 1][0] == key:
                hf -= 1
            e_sa[here + p - of] = t
            e_rank[t] = here + hf - of
            if sum(1 for k2, _ in items if k2 == key) >= 2:
                act.append(t)
        e_loc[w] = act
    sa = np.full(n, kNone, np.uint32)
    d_cnt = np.zeros(1, np.uint32)
    d_err = np.zeros(1, np.uint32)
    d_left = np.zeros(1, np.uint32)
    nwin = len(beg)
    left = sum(1 for w in range(nwin) if beg[w] != kNone and lofs[w] == kNone and cnt[w] > kWChunk)
    emu.emu_round(_p(loc_act), _p(loc_next), _p(beg), _p(lofs), _p(cnt), ctypes.c_uint32(nwin), ctypes.c_uint32(n),
                  _p(rank), _p(sa), _p(d_cnt), _p(d_err), _p(d_left), ctypes.c_uint(2), ctypes.c_uint(3))
    assert d_err[0] == 0
    # the count the CTA kernel returns early on when it is zero
    assert int(d_left[0]) == left
    assert all(sa[r] == t for r, t in e_sa.items())
    assert all(rank[t] == r for t, r in e_rank.items())
    for w, act in e_loc.items():
        assert cnt[w] == len(act)
        assert list(loc_act[beg[w]:beg[w] + len(act)]) == act
    assert int(d_cnt[0]) == sum(len(a) for a in e_loc.values())


@pytest.mark.timeout(600)
@pytest.mark.parametrize("seed,grid", [(31, 1), (32, 3), (33, 7)])
def test_round_gather(emu, seed, grid):
    """Each local unit's members get the rank of the suffix h further on,
    in member order; other rows of loc_next stay as they were; a member
    whose t + h is past the block is flagged (bit 7 of the error word)."""
    rng = np.random.default_rng(seed)
    n, beg, lofs, cnt, loc_act, _, rank, _ = make_round(rng, nwin=40, big_units=0.2)
    h = 3
    if seed == 33:  # a member near the block end: no suffix h further on
        w0 = next(w for w in range(len(beg)) if beg[w] != kNone and lofs[w] == kNone and cnt[w] > 40)
        loc_act[beg[w0] + 37] = n - 2
    loc_next = np.full(n, 0xABCDEF, np.uint32)
    want = loc_next.copy()
    bad = False
    for w in range(len(beg)):
        if beg[w] == kNone or lofs[w] != kNone:
            continue
        for k in range(int(cnt[w])):
            t = int(loc_act[beg[w] + k])
            if t + h < n:
                want[beg[w] + k] = rank[t + h]
            else:
                want[beg[w] + k] = 0
                bad = True
    d_err = np.zeros(1, np.uint32)
    emu.emu_round_gather(_p(loc_act), _p(beg), _p(lofs), _p(cnt), ctypes.c_uint32(len(beg)), _p(rank),
                         ctypes.c_uint32(h), ctypes.c_uint32(n), _p(loc_next), _p(d_err), ctypes.c_uint(grid))
    assert np.array_equal(loc_next, want)
    assert bool(d_err[0] & 128) == bad and (d_err[0] & ~np.uint32(128)) == 0
    assert bad or seed != 33


# ---- the unit scan ------------------------------------------------------------

@pytest.mark.timeout(600)
@pytest.mark.parametrize("case", [dict(seed=21, n_target=30000), dict(seed=22, n_target=60000, p_big=0.01,
                                  big=(2500, 4000)), dict(seed=23, n_target=5000000, max_bucket=64, p_short=0.3),
                                  dict(seed=24, n_target=20000, p_hugeshort=0.02)])
def test_unit_scan(emu, case):
    """Unit ends, long counts, window owners and the offsets of the units
    of the device-wide path, from the window table of a block."""
    case = dict(case)
    rng = np.random.default_rng(case.pop("seed"))
    n, is_long, keys, starts, t_of_row = make_block(rng, case.pop("n_target"), 41, **case)
    nwin = (n + kWindow - 1) // kWindow
    is_start = np.zeros(n + 1, bool)
    is_start[starts] = True
    beg = np.full(nwin, kNone, np.uint32)
    lcb = np.zeros(nwin, np.uint32)
    lct = np.zeros(nwin, np.uint32)
    long_before = np.concatenate([[0], np.cumsum(is_long)])
    for w in range(nwin):
        lo, hi = w * kWindow, min(n, (w + 1) * kWindow)
        st = np.nonzero(is_start[lo:hi])[0]
        lct[w] = long_before[hi] - long_before[lo]
        if len(st):
            beg[w] = lo + st[0]
            lcb[w] = long_before[lo + st[0]] - long_before[lo]
        else:
            lcb[w] = lct[w]
    stride = (n // kWindow + 2 + 7) & ~7  # the device layout's words per field
    fields = np.zeros(8 * stride, np.uint32)
    fields[0:nwin] = beg
    fields[stride:stride + nwin] = lcb
    fields[2 * stride:2 * stride + nwin] = lct
    fields[6 * stride:6 * stride + nwin] = 7  # counts to be zeroed
    zero_slots = np.full(3 * 2, 9, np.uint32)
    left_slots = np.full(4, 9, np.uint32)
    d_large = np.zeros(1, np.uint32)
    emu.emu_unit_scan(_p(fields), ctypes.c_uint64(stride), ctypes.c_uint32(nwin), ctypes.c_uint32(n), _p(d_large),
                      _p(zero_slots), ctypes.c_int(3), ctypes.c_int(2), _p(left_slots), ctypes.c_int(3))
    end = fields[3 * stride:3 * stride + nwin]
    nlong = fields[4 * stride:4 * stride + nwin]
    lofs = fields[5 * stride:5 * stride + nwin]
    cnt = fields[6 * stride:6 * stride + nwin]
    owner = fields[7 * stride:7 * stride + nwin]
    unit_ws = [w for w in range(nwin) if beg[w] != kNone]
    off = 0
    last = None
    for w in range(nwin):
        if beg[w] != kNone:
            a = unit_ws.index(w)
            e = int(beg[unit_ws[a + 1]]) if a + 1 < len(unit_ws) else n
            nl = long_before[e] - long_before[beg[w]]
            assert end[w] == e and nlong[w] == nl
            if nl > kLCap:
                assert lofs[w] == off
                off += e - int(beg[w])
            else:
                assert lofs[w] == kNone
        else:
            assert end[w] == 0 and nlong[w] == 0 and lofs[w] == kNone
        # the unit whose rows include the window's first row
        assert owner[w] == (w if beg[w] == w * kWindow else last)
        if beg[w] != kNone:
            last = w
    assert int(d_large[0]) == off
    assert np.all(cnt == 0)
    assert list(zero_slots) == [0, 9, 0, 9, 0, 9]
    assert list(left_slots) == [0, 0, 0, 9]
