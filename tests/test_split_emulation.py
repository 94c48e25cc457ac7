"""The front of the bucket split (csrc/suffix_sort.cu) run on the CPU.

ConstructSA (Section 3) starts from one element per suffix t of the block:
its bucket number (the first P codes and min(len, P), numbered densely in
key order, bit 31 set for a short bucket, len < P), its key's length field
and t.  `sa_digit_keys` writes them and counts the first radix pass's digits
(bits 0..7) per chunk of whole 2048-element tiles.  After the elements are
sorted by bucket (stably: t order inside a bucket), `sa_unit_begin` walks
each window of 1024 rows.  A short suffix is final where it landed: its
bucket holds only equal strings, in t order, so SA[i] = t and rank[t] = i.
Each long row joins its window's list with its key; the window's first
bucket start and its long counts go to the unit table.

Checked against plain definitions on random reads with terminators (2-bit
codes, and 4-bit codes for 16 symbols): keys built symbol by symbol, bucket
numbers as the index of (p, l) among all valid pairs, counts by chunk, and
the window table from the sorted rows.  The kernels' text is cut out of
the CUDA source and compiled for the host with tests/emu/cuda_emu.h.  No
GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "split_emulation.cpp")
kH0 = 29
kShortFlag = 0x80000000
kDigitMask = (1 << 24) - 1
kNone = 0xFFFFFFFF
kWindow = 1024
TILE = 2048


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("splitemu")
    src = open(os.path.join(CSRC, "suffix_sort.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "radix_hdr.inc").write_text(_cut(hdr, "constexpr int kRadixBits = 8;", "size_t radix_temp_words(uint64_t cap);"))
    (d / "constants.inc").write_text(_cut(src, "constexpr int kThreads = 256;", "// Key geometry per code width"))
    (d / "keys.inc").write_text(_cut(src, "// Key geometry per code width",
                                     "// Element of block position t for the bucket split"))
    (d / "digit_keys.inc").write_text(_cut(src, "// Element of block position t for the bucket split",
                                           "// One warp per window of the digit-sorted array"))
    (d / "unit_begin.inc").write_text(_cut(src, "// One warp per window of the digit-sorted array",
                                           "// kScanPer consecutive windows of one field"))
    (d / "scan.inc").write_text(_cut(hdr, "struct SumOp {", "// Launch bookkeeping"))
    (d / "unit_scan.inc").write_text(_cut(src, "// kScanPer consecutive windows of one field",
                                          "// one spare slot per kLItems"))
    (d / "large_gather.inc").write_text(_cut(src, "// The global-path list:",
                                             "// next-ranks of the local unsorted members"))
    lib = d / "libsplitemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    L.emu_digit_keys.argtypes = [I, P, U64, P, U64, U32, U32, U32, U32, P, P, P, P]
    L.emu_unit_begin.argtypes = [I, P, U64, P, U32, U32, P, P, P, P, P, P, P, P, P, ctypes.c_uint]
    L.emu_digit_keys.restype = I
    L.emu_unit_begin.restype = I
    L.emu_large_chain.argtypes = [I, P, U64, P, U32, U32, U64, P, P, P, P, P, P, P, P]
    L.emu_large_chain.restype = I
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def pack(codes, kb):
    """Codes into 32-bit words, first code in the most significant bits."""
    per = 32 // kb
    words = np.zeros((codes.size + per - 1) // per, np.uint64)
    for j in range(per):
        part = codes[j::per].astype(np.uint64)
        words[:part.size] |= part << np.uint64(32 - kb * (j + 1))
    return words.astype(np.uint32)


def make_text(rng, kb, sigma, n_reads):
    """Reads of mixed lengths, a third of them copies of earlier ones (so
    buckets and keys repeat), each followed by a terminator."""
    H = 29 if kb == 2 else 14
    reads = []
    for _ in range(n_reads):
        if reads and rng.random() < 0.33:
            src = reads[int(rng.integers(0, len(reads)))]
            a = int(rng.integers(0, len(src) + 1))
            reads.append(src[a:])
        else:
            ln = int(rng.integers(0, 4 * H)) if rng.random() < 0.9 else int(rng.integers(0, 4))
            reads.append(rng.integers(0, sigma, size=ln))
    lens = np.array([r.size for r in reads])
    n = int(lens.sum() + lens.size)
    codes = rng.integers(0, sigma, size=n)  # the code at a terminator is arbitrary
    term = np.zeros(n, bool)
    ends = np.cumsum(lens + 1) - 1
    term[ends] = True
    starts = ends - lens
    for r, s in zip(reads, starts):
        codes[s:s + r.size] = r
    return codes, term


def keys_of(codes, term, kb):
    """Each suffix's key: its first H codes (zero at and past its terminator)
    and its length field, built symbol by symbol."""
    H = 29 if kb == 2 else 14
    n = codes.size
    idx = np.where(term, np.arange(n), n)
    next_term = np.minimum.accumulate(idx[::-1])[::-1]
    ln = next_term - np.arange(n)
    pad = np.concatenate([codes, np.zeros(H, codes.dtype)])
    key = np.zeros(n, np.uint64)
    for q in range(H):
        c = np.where(q < ln, pad[q:q + n], 0).astype(np.uint64)
        key = (key << np.uint64(kb)) | c
    field = np.where(ln < H, ln, kH0)
    return (key << np.uint64(5)) | field.astype(np.uint64), field, ln


def bucket_numbers(keys, field, kb, sigma, P):
    """Index of each key's bucket (p, l) among all valid buckets in key
    order (p, then l), with bit 31 set for l < P."""
    H = 29 if kb == 2 else 14
    codes = keys >> np.uint64(5)
    p = np.zeros(keys.size, np.int64)
    for q in range(P):
        c = ((codes >> np.uint64(kb * (H - 1 - q))) & np.uint64((1 << kb) - 1)).astype(np.int64)
        p = p * sigma + c
    l = np.minimum(field, P).astype(np.int64)
    vp, vl = [], []
    for ll in range(P + 1):
        x = np.arange(0, sigma ** P, sigma ** (P - ll), dtype=np.int64)
        vp.append(x)
        vl.append(np.full(x.size, ll, np.int64))
    valid = np.sort(np.concatenate(vp) * (P + 1) + np.concatenate(vl))
    code = p * (P + 1) + l
    at = np.searchsorted(valid, code)
    assert np.array_equal(valid[at], code), "a key fell in an invalid bucket"
    return at.astype(np.uint32) | np.where(l < P, kShortFlag, 0).astype(np.uint32)


def bucket_codes_for(sigma):
    P = 1
    while P + 1 <= 14 and sum(sigma ** k for k in range(P + 2)) <= 1 << 24:
        P += 1
    return P


CASES = [dict(kb=2, sigma=4, reads=500, seed=1, grids=(1, 3)),
         dict(kb=2, sigma=4, reads=900, seed=2, grids=(7, 40)),
         dict(kb=4, sigma=16, reads=700, seed=3, grids=(2, 5))]


@pytest.mark.timeout(900)
@pytest.mark.parametrize("case", CASES)
def test_digit_keys_and_unit_begin(emu, case):
    kb, sigma = case["kb"], case["sigma"]
    rng = np.random.default_rng(case["seed"])
    codes, term = make_text(rng, kb, sigma, case["reads"])
    n = codes.size
    assert n > 2 * TILE and n % TILE != 0
    P = 11 if kb == 2 else bucket_codes_for(sigma)
    text = pack(codes, kb)
    bits = np.zeros((n + 31) // 32, np.uint32)
    for j in np.nonzero(term)[0]:
        bits[j >> 5] |= np.uint32(1 << (j & 31))
    keys, field, _ = keys_of(codes, term, kb)
    digits = bucket_numbers(keys, field, kb, sigma, P)
    want_elems = (digits.astype(np.uint64) | (field.astype(np.uint64) << np.uint64(24))
                  | (np.arange(n, dtype=np.uint64) << np.uint64(32)))
    for grid in case["grids"]:
        elems = np.zeros(n, np.uint64)
        counts = np.full(grid * 256, 0xDEAD, np.uint32)
        totals = np.zeros(256, np.uint32)
        n_out = np.zeros(1, np.uint32)
        assert emu.emu_digit_keys(kb, _p(text), text.size, _p(bits), bits.size, n, sigma, P, grid, _p(elems),
                                  _p(counts), _p(totals), _p(n_out)) == 0
        assert int(n_out[0]) == n
        assert np.array_equal(elems, want_elems)
        ntiles = (n + TILE - 1) // TILE
        per = (ntiles + grid - 1) // grid
        chunk = (np.arange(n) // TILE) // per
        used = int(chunk.max()) + 1
        want = np.zeros((grid, 256), np.int64)
        np.add.at(want, (chunk, (digits & 255).astype(np.int64)), 1)
        got = counts.reshape(grid, 256).astype(np.int64)
        assert np.array_equal(got[:used], want[:used])
        assert np.all(got[used:] == 0xDEAD)  # chunks past the last tile are left alone
        assert np.array_equal(totals.astype(np.int64), want.sum(axis=0))

    # the elements sorted by bucket (stable: t order inside a bucket)
    order = np.argsort(want_elems & np.uint64(kDigitMask), kind="stable")
    srt = want_elems[order]
    d = (srt & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    t = (srt >> np.uint64(32)).astype(np.uint32)
    nwin = (n + kWindow - 1) // kWindow
    beg = np.full(nwin, 7, np.uint32)
    lcb = np.full(nwin, 7, np.uint32)
    lct = np.full(nwin, 7, np.uint32)
    sa = np.full(n, 0xABCD, np.uint32)
    rank = np.full(n, 0xABCD, np.uint32)
    slots = nwin * kWindow
    ll_t = np.full(slots, 0xABCD, np.uint32)
    ll_row = np.full(slots, 0xABCD, np.uint32)
    ll_key = np.full(slots, 0xABCD, np.uint64)
    d_err = np.zeros(1, np.uint32)
    assert emu.emu_unit_begin(kb, _p(text), text.size, _p(srt), n, nwin, _p(beg), _p(lcb), _p(lct), _p(sa),
                              _p(rank), _p(ll_t), _p(ll_row), _p(ll_key), _p(d_err), 3) == 0
    assert d_err[0] == 0
    short = (d & np.uint32(kShortFlag)) != 0
    bnd = np.ones(n, bool)
    bnd[1:] = ((d[1:] ^ d[:-1]) & np.uint32(kDigitMask)) != 0
    rows = np.arange(n)
    # short suffixes: final where they landed
    assert np.array_equal(sa[short], t[short])
    assert np.array_equal(rank[t[short]], rows[short].astype(np.uint32))
    assert np.all(sa[~short] == 0xABCD) and np.all(rank[t[~short]] == 0xABCD)
    for w in range(nwin):
        lo, hi = w * kWindow, min(n, (w + 1) * kWindow)
        b = np.nonzero(bnd[lo:hi])[0]
        lng = np.nonzero(~short[lo:hi])[0]
        assert lct[w] == lng.size
        if b.size:
            assert beg[w] == lo + b[0] and lcb[w] == np.count_nonzero(lng < b[0])
        else:
            assert beg[w] == kNone and lcb[w] == lng.size
        k = lng.size
        assert np.array_equal(ll_t[lo:lo + k], t[lo + lng])
        assert np.array_equal(ll_row[lo:lo + k], (lo + lng).astype(np.uint32))
        assert np.array_equal(ll_key[lo:lo + k], keys[t[lo + lng]])
        assert np.all(ll_t[lo + k:lo + kWindow] == 0xABCD)
    # a real mix: short and long suffixes in the sorted rows
    assert short.any() and (~short).any()


@pytest.mark.timeout(900)
def test_units_too_large_for_a_cta_are_listed_for_the_device_wide_path(emu):
    """Many copies of one read make units with more than 2048 long
    suffixes.  After the unit begin and the unit scan, the gather lists every
    row of each such unit, in row order, at the unit's offset: (key, t,
    row); the offsets are the units' sizes summed in unit order."""
    kb, sigma, P = 2, 4, 11
    rng = np.random.default_rng(8)
    rep = rng.integers(0, sigma, size=60)
    reads = [rep.copy() for _ in range(2600)] + [rng.integers(0, sigma, size=int(rng.integers(0, 90)))
                                                 for _ in range(600)]
    order = rng.permutation(len(reads))
    reads = [reads[i] for i in order]
    lens = np.array([r.size for r in reads])
    n = int(lens.sum() + lens.size)
    codes = rng.integers(0, sigma, size=n)
    term = np.zeros(n, bool)
    ends = np.cumsum(lens + 1) - 1
    term[ends] = True
    for r, s in zip(reads, ends - lens):
        codes[s:s + r.size] = r
    text = pack(codes, kb)
    keys, field, _ = keys_of(codes, term, kb)
    digits = bucket_numbers(keys, field, kb, sigma, P)
    elems = (digits.astype(np.uint64) | (field.astype(np.uint64) << np.uint64(24))
             | (np.arange(n, dtype=np.uint64) << np.uint64(32)))
    srt = elems[np.argsort(elems & np.uint64(kDigitMask), kind="stable")]
    d = (srt & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    t = (srt >> np.uint64(32)).astype(np.uint32)
    nwin = (n + kWindow - 1) // kWindow
    stride = (n // kWindow + 2 + 7) & ~7
    fields = np.zeros(8 * stride, np.uint32)
    sa = np.zeros(n, np.uint32)
    rank = np.zeros(n, np.uint32)
    lkeys = np.full(n, 0xABCD, np.uint64)
    lvals = np.full(n, 0xABCD, np.uint32)
    lpos = np.full(n, 0xABCD, np.uint32)
    d_large = np.zeros(1, np.uint32)
    d_err = np.zeros(1, np.uint32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_large_chain(kb, p(text), text.size, p(srt), n, nwin, stride, p(fields), p(sa), p(rank),
                               p(lkeys), p(lvals), p(lpos), p(d_large), p(d_err)) == 0
    assert d_err[0] == 0
    # units from the definitions: a unit is the buckets starting in a window
    bnd = np.ones(n, bool)
    bnd[1:] = ((d[1:] ^ d[:-1]) & np.uint32(kDigitMask)) != 0
    long_ = (d & np.uint32(kShortFlag)) == 0
    starts = [int(w * kWindow + np.nonzero(bnd[w * kWindow:(w + 1) * kWindow])[0][0])
              for w in range(nwin) if bnd[w * kWindow:(w + 1) * kWindow].any()]
    ends = starts[1:] + [n]
    off, want = 0, []
    for b, e in zip(starts, ends):
        if np.count_nonzero(long_[b:e]) > 2048:
            want.append((b, e, off))
            off += e - b
    assert want, "the data must hold a unit too large for a CTA"
    assert int(d_large[0]) == off
    lofs = fields[5 * stride:5 * stride + nwin]
    for b, e, o in want:
        assert lofs[b // kWindow] == o
        rows = np.arange(b, e)
        assert np.array_equal(lpos[o:o + e - b], rows.astype(np.uint32))
        assert np.array_equal(lvals[o:o + e - b], t[rows])
        assert np.array_equal(lkeys[o:o + e - b], keys[t[rows]])
    assert np.all(lpos[off:] == 0xABCD)
