"""ComputeRanks (Algorithm 2 with Lemma 1) run on the CPU: the per-read
kernel and the segmented kernel for long reads; and the gather that follows
it (B_int, g_sa = g[SA_int] and Insert's plan).

The text of both kernels and of the dictionary layout is cut out of
csrc/ranks.cu and csrc/sbwt_internal.cuh and compiled for the host with
tests/emu/cuda_emu.h (one thread per GPU thread, every array between
inaccessible pages).  The dictionary of the reads already indexed is packed
here from the oracle's B (bit planes, counters every 64, 128 or 256 rows,
superblock counters and C[] with the terminators counted), the new reads'
text in the append layout, and g is compared with the oracle's direct count
of smaller old suffixes for every position of the block.  The segmented
kernel starts each segment of 256 positions from a backward search whose
window doubles while it still occurs in B_ext; reads drawn from a short
genome make those windows repeat.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import readgen
from test_insert_emulation import CODE, pack_dict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "ranks_emulation.cpp")
SEG_ROWS = 256


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("rankemu")
    src = open(os.path.join(CSRC, "ranks.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "dict.inc").write_text("constexpr int kThreads = 256;\n" + _cut(
        hdr, "constexpr int kOccShift = 6;", "// ---------------------------------------------------------------------------\n// CTA-wide scans"))
    (d / "text.inc").write_text(_cut(hdr, "constexpr int kTextPadWords = 4;", "// Rank dictionary over B"))
    (d / "bint.inc").write_text(_cut(src, "// B_int[i]: the symbol before block suffix SA[i]",
                                     "// Algorithm 2, one thread per read:"))
    (d / "gather.inc").write_text(_cut(src, "// B_int and g_sa in one pass over SA_int",
                                       "// rank(c, k) queries, codes 0..kCodes-1"))
    (d / "queries.inc").write_text(_cut(src, "// rank(c, k) queries, codes 0..kCodes-1",
                                        "// The read-back of the 2-bit dictionary"))
    (d / "unpack.inc").write_text(_cut(src, "// The read-back of the 2-bit dictionary",
                                       "// The read-back for the 4-bit dictionary"))
    (d / "unpack_w.inc").write_text(_cut(src, "// The read-back for the 4-bit dictionary", "uint32_t alpha4_of("))
    kh = open(os.path.join(CSRC, "sbwt_kernels.cuh")).read()
    (d / "alphabet.inc").write_text(_cut(kh, "struct Alphabet16 {", "// pack.cu:"))
    kern = _cut(src, "// Algorithm 2, one thread per read:", "// B_int and g_sa in one pass over SA_int")
    kern = kern.replace("extern __shared__ unsigned long long s_raw[];", "unsigned long long* s_raw = g_dyn_smem;")
    (d / "ranks.inc").write_text(kern)
    lib = d / "librankemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    L.emu_compute_ranks.argtypes = [I, I, U32, U32, P, U64, P, U64, P, P, P, U64, U64, P, U64, P]
    L.emu_compute_ranks.restype = I
    L.emu_bint_gather.argtypes = [P, U64, P, U64, U64, P, P, U64, U32, P, P, P, U64, I]
    L.emu_bint_gather.restype = I
    L.emu_queries.argtypes = [I, P, P, P, U64, P, P, U64, P, P, U64, P, U64, P, U64, U64, P]
    L.emu_queries.restype = I
    L.emu_queries_w.argtypes = [P, P, P, U64, P, I, P, P, U64, P, P, U64, P, U64, P, U64, U64, P]
    L.emu_queries_w.restype = I
    L.emu_compute_ranks_w.argtypes = [I, I, U32, U32, P, U64, P, U64, P, P, P, U64, U64, P, U64, P]
    L.emu_compute_ranks_w.restype = I
    L.emu_bint_plain.argtypes = [P, U64, P, U64, U64, P, U32, P]
    L.emu_bint_plain.restype = I
    return L


def dictionary(B: np.ndarray, m: int, k: int):
    """Blocks, superblock counters and C[] of B (m terminators)."""
    words = pack_dict(B, k)
    nsb = (len(B) >> 16) + 1
    sup = np.zeros((nsb, 4), np.uint64)
    for s in range(1, nsb):
        chunk = B[: s << 16]
        sup[s] = [np.count_nonzero(chunk == c) for c in b"ACGT"]
    tot = [np.count_nonzero(B == c) for c in b"ACGT"]
    C = np.array([m, m + tot[0], m + tot[0] + tot[1], m + tot[0] + tot[1] + tot[2]], np.uint64)
    return words, sup.ravel(), C


def append_text(reads: np.ndarray, off: np.ndarray) -> np.ndarray:
    """2-bit codes of an append's positions (read j's symbol k at off[j] + j +
    k, a terminator after each read stored as code 0), 16 per word, MSB first,
    with four zero words of padding."""
    m = len(off) - 1
    npos = int(off[-1]) + m
    codes = np.zeros(npos, np.uint32)
    lut = np.zeros(256, np.uint32)
    for c, v in CODE.items():
        lut[c] = v
    pos = np.arange(int(off[-1])) + np.repeat(np.arange(m), np.diff(off.astype(np.int64)))
    codes[pos] = lut[reads]
    nw = (npos + 15) // 16
    padded = np.zeros(nw * 16, np.uint32)
    padded[:npos] = codes
    sh = (30 - 2 * np.arange(16)).astype(np.uint32)
    words = np.bitwise_or.reduce(padded.reshape(nw, 16) << sh, axis=1).astype(np.uint32)
    return np.concatenate([words, np.zeros(4, np.uint32)])


def run(emu, old_reads, old_off, new_reads, new_off, k=1, seg=False, seg_rows=SEG_ROWS):
    B = oracle.bwt(old_reads, old_off)
    m_ext = len(old_off) - 1
    words, sup, C = dictionary(B, m_ext, k)
    text = append_text(new_reads, new_off)
    nreads = len(new_off) - 1
    n_int = int(new_off[-1]) + nreads
    max_len = int(np.diff(new_off.astype(np.int64)).max())
    segs = max_len // seg_rows + 1
    g = np.zeros(max(n_int, 1), np.uint32)
    err = ctypes.c_uint32(0)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    off = np.ascontiguousarray(new_off, np.uint64)
    assert emu.emu_compute_ranks(k, int(seg), segs, seg_rows, ptr(text), len(text), ptr(off), nreads, ptr(words), ptr(sup),
                                 ptr(C), len(B), m_ext, ptr(g), n_int, ctypes.byref(err)) == 0
    return g[:n_int], err.value


def expected_g(old, new):
    reads = np.concatenate([old[0], new[0]])
    lens = np.concatenate([np.diff(old[1].astype(np.int64)), np.diff(new[1].astype(np.int64))])
    off = readgen.offsets_from_lengths(lens)
    m0 = len(old[1]) - 1
    return oracle.block_g_direct(reads, off, m0, len(off) - 1).astype(np.uint32)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_per_read_kernel_matches_direct_counts(emu, k):
    old = readgen.ragged_reads(400, 0, 120, seed=31, p_empty=0.03, p_repeat=0.05)
    new = readgen.ragged_reads(150, 0, 120, seed=32, p_empty=0.03, p_repeat=0.05)
    g, err = run(emu, *old, *new, k=k)
    assert err == 0
    assert np.array_equal(g, expected_g(old, new))


@pytest.mark.parametrize("k,seg_rows", [(1, 256), (4, 256), (1, 1024)])
@pytest.mark.parametrize("repeat", [True, False])
def test_segmented_kernel_matches_direct_counts(emu, k, seg_rows, repeat):
    """Long reads (513 to 3000 symbols) sampled from a genome: a 300-symbol
    unit repeated twelve times makes the backward-search windows occur in
    B_ext, so segments widen their window, up to the terminator's exact
    chain; a 100 kbp i.i.d. genome lets the first window settle most
    segments."""
    g_ = np.tile(readgen.genome(300, seed=300), 12) if repeat else readgen.genome(100_000, seed=1)
    old = readgen.sampled_reads(g_, 30, np.random.default_rng(1).integers(200, 3000, size=30), 0.01, seed=33)
    lens = np.random.default_rng(2).integers(600, 3000, size=12)
    lens[0] = 513  # just over the per-read limit: two segments and a partial third
    new = readgen.sampled_reads(g_, 12, lens, 0.01, seed=34)
    g, err = run(emu, *old, *new, k=k, seg=True, seg_rows=seg_rows)
    assert err == 0
    assert np.array_equal(g, expected_g(old, new))
    # the per-read kernel agrees on the same block
    g2, _ = run(emu, *old, *new, k=k, seg=False)
    assert np.array_equal(g2, g)


def test_segmented_kernel_against_an_empty_index(emu):
    """No old reads: every window's interval is empty at once (g = 0)."""
    empty = (np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    new = readgen.ragged_reads(6, 700, 1500, seed=35)
    g, err = run(emu, *empty, *new, seg=True)
    assert err == 0 and not np.any(g)


def term_bitmap(off: np.ndarray) -> np.ndarray:
    """Terminator bitmap of an append (bit t & 31 of word t >> 5 set at read
    j's terminator position off[j+1] + j), with two zero words of padding."""
    m = len(off) - 1
    npos = int(off[-1]) + m
    words = np.zeros((npos + 31) // 32 + 2, np.uint32)
    tpos = off[1:].astype(np.int64) + np.arange(m)
    np.bitwise_or.at(words, tpos >> 5, (np.uint32(1) << (tpos & 31).astype(np.uint32)).astype(np.uint32))
    return words


@pytest.mark.parametrize("n_reads,seed", [(40, 1), (173, 2)])
def test_gather_writes_bint_gsa_and_the_insert_plan(emu, n_reads, seed):
    """B_int[i] is the symbol before suffix SA[i] (a terminator where the
    suffix starts its read), g_sa[i] = g[SA[i]], and the plan entry of
    superblock S is the number of new symbols whose rows r_i = g_sa[i] + i
    lie below S 2^shift (here 64-row superblocks, so hundreds of entries),
    for blocks whose sizes are not multiples of a thread's four elements."""
    rng = np.random.default_rng(seed)
    reads, off = readgen.ragged_reads(n_reads, 0, 60, seed=seed + 10, p_empty=0.05)
    m = len(off) - 1
    n = int(off[-1]) + m
    text = append_text(reads, off)
    term = term_bitmap(off)
    sa = rng.permutation(n).astype(np.uint32)
    n_ext = 3 * n + 17
    gsa_want = np.sort(rng.integers(0, n_ext + 1, size=n)).astype(np.uint32)
    g = np.zeros(n, np.uint32)
    g[sa] = gsa_want
    shift = 6
    nsb = ((n_ext + n) >> shift) + 1
    bint = np.zeros(n, np.uint8)
    gsa = np.zeros(n, np.uint32)
    plan = np.full(nsb + 1, 0xDEADBEEF, np.uint32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_bint_gather(ptr(text), len(text), ptr(term), len(term), 0, ptr(sa), ptr(g), n, n, ptr(bint),
                               ptr(gsa), ptr(plan), nsb, shift) == 0
    codes = np.zeros(n, np.int64)
    lut = np.zeros(256, np.int64)
    for c, v in CODE.items():
        lut[c] = v
    pos = np.arange(int(off[-1])) + np.repeat(np.arange(m), np.diff(off.astype(np.int64)))
    codes[pos] = lut[reads]
    is_term = np.zeros(n, bool)
    is_term[off[1:].astype(np.int64) + np.arange(m)] = True
    t = sa.astype(np.int64)
    want = np.where((t == 0) | is_term[np.maximum(t - 1, 0)], 255, codes[np.maximum(t - 1, 0)])
    assert np.array_equal(bint, want.astype(np.uint8))
    # the one-block kernel (a block into an empty index) gives the same B_int
    bint1 = np.zeros(n, np.uint8)
    assert emu.emu_bint_plain(ptr(text), len(text), ptr(term), len(term), 0, ptr(sa), n, ptr(bint1)) == 0
    assert np.array_equal(bint1, want.astype(np.uint8))
    assert np.array_equal(gsa, gsa_want)
    r = gsa_want.astype(np.int64) + np.arange(n)
    plan_want = np.searchsorted(r, np.arange(nsb + 1, dtype=np.int64) << shift, side="left")
    assert np.array_equal(plan.astype(np.int64), plan_want)


# ---- queries and read-back over a finished dictionary ----------------------

def _occurrences(reads, off, pat: bytes) -> int:
    """Occurrences of pat inside the reads (overlapping, none across a read
    end); the empty pattern occurs at every row."""
    if not pat:
        return int(off[-1]) + len(off) - 1
    total = 0
    for j in range(len(off) - 1):
        s = reads[int(off[j]):int(off[j + 1])].tobytes()
        i = s.find(pat)
        while i >= 0:
            total += 1
            i = s.find(pat, i + 1)
    return total


@pytest.mark.timeout(600)
@pytest.mark.parametrize("k", [1, 2, 4])
def test_rank_queries_counts_and_read_back(emu, k):
    """rank(c, k) for the four codes and the terminator, FM-index counts of
    patterns (backward search with Lemma 1's C) and the read-back of row
    ranges, over the dictionary of the oracle's B (two superblocks)."""
    rng = np.random.default_rng(70 + k)
    g = readgen.genome(5_000, 9)
    reads, off = readgen.sampled_reads(g, 1_400, 90, 0.01, 10 + k)
    m = len(off) - 1
    B = oracle.bwt(reads, off)
    n = len(B)
    assert n > 1 << 16
    words, sup, C = dictionary(B, m, k)
    # rank queries: random rows plus the edges (row 0, the end, block and
    # superblock boundaries)
    edges = np.array([0, 1, 63, 64, 65, 64 * k, (1 << 16) - 1, 1 << 16, (1 << 16) + 1, n - 1, n], np.uint64)
    ks = np.concatenate([rng.integers(0, n + 1, size=3000).astype(np.uint64), np.repeat(edges, 5)])
    codes = np.concatenate([rng.integers(0, 5, size=3000), np.tile(np.arange(5), edges.size)]).astype(np.uint8)
    sym = np.frombuffer(b"ACGT$", np.uint8)
    cum = {c: np.concatenate([[0], np.cumsum(B == sym[c])]) for c in range(5)}
    want_rank = np.array([cum[int(c)][int(x)] for c, x in zip(codes, ks)], np.uint64)
    # patterns: substrings of the reads, random strings, a foreign byte, empty
    pats = []
    for _ in range(150):
        j = int(rng.integers(0, m))
        r = reads[int(off[j]):int(off[j + 1])]
        a = int(rng.integers(0, max(1, r.size - 1)))
        pats.append(r[a:a + int(rng.integers(1, 25))].tobytes())
    pats += [bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(L))) for L in (1, 2, 3, 6, 12)]
    pats += [b"ACGNT", b"", b"A" * 40]
    pbytes = np.frombuffer(b"".join(pats) or b"\0", np.uint8).copy()
    poffs = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.uint64)
    want_count = np.array([_occurrences(reads, off, p) for p in pats], np.uint64)
    # read-back of rows [r0, r1): a range from a part start to a ragged end
    r0, r1 = 64 * 37, n - 5
    rank_out = np.zeros(ks.size, np.uint64)
    count_out = np.zeros(len(pats), np.uint64)
    out = np.full((n + 63) // 64 * 64, 0xEE, np.uint8)
    assert emu.emu_queries(k, ctypes.c_void_p(words.ctypes.data), ctypes.c_void_p(sup.ctypes.data),
                           ctypes.c_void_p(C.ctypes.data), n, ctypes.c_void_p(codes.ctypes.data),
                           ctypes.c_void_p(ks.ctypes.data), ks.size, ctypes.c_void_p(rank_out.ctypes.data),
                           ctypes.c_void_p(pbytes.ctypes.data), pbytes.size, ctypes.c_void_p(poffs.ctypes.data),
                           len(pats), ctypes.c_void_p(count_out.ctypes.data), r0, r1,
                           ctypes.c_void_p(out.ctypes.data)) == 0
    assert np.array_equal(rank_out, want_rank)
    assert np.array_equal(count_out, want_count)
    assert want_count[:150].min() >= 1 and want_count[-3] == 0 and want_count[-2] == n
    assert np.array_equal(out[r0:r1], B[r0:r1])
    assert np.all(out[:r0] == 0xEE) and np.all(out[r1:] == 0xEE)


def dictionary_w(B: np.ndarray, m: int):
    """Blocks, superblock counters (16 per 4096 rows) and C[] of B in the
    4-bit layout of the 12-symbol alphabet (m terminators)."""
    from test_insert_w_emulation import codes_of, pack_dict_w
    n = len(B)
    nsb = (((n >> 6) + 1) + 63) // 64
    code = np.where(B == ord("$"), -1, codes_of(B))
    sup = np.zeros((nsb, 16), np.uint64)
    for s in range(1, nsb):
        head = code[: s * 4096]
        sup[s] = [np.count_nonzero(head == c) for c in range(16)]
    tot = np.array([np.count_nonzero(code == c) for c in range(16)], np.uint64)
    C = (np.uint64(m) + np.concatenate([[0], np.cumsum(tot)[:-1]])).astype(np.uint64)
    return pack_dict_w(B), sup.ravel(), C


@pytest.mark.timeout(600)
def test_rank_queries_counts_and_read_back_4bit(emu):
    """The same over the 4-bit dictionary of a 12-symbol alphabet: rank for
    every code (unused codes count zero) and the terminator, counts, and the
    read-back, over the oracle's B packed into the 4-bit layout."""
    from test_insert_w_emulation import ALPHA, codes_of, pack_dict_w
    rng = np.random.default_rng(91)
    sigma = len(ALPHA)
    g = readgen.genome_alpha(3_000, 5, np.full(sigma, 1.0 / sigma))
    reads, off = readgen.sampled_reads_alpha(g, 250, 60, 0.01, 6, ALPHA)
    m = len(off) - 1
    B = oracle.bwt(reads, off, ALPHA)
    n = len(B)
    assert n > 3 * 4096
    blocks, sup, C = dictionary_w(B, m)
    code = np.where(B == ord("$"), -1, codes_of(B))
    edges = np.array([0, 1, 63, 64, 4095, 4096, 4097, n - 1, n], np.uint64)
    ks = np.concatenate([rng.integers(0, n + 1, size=2000).astype(np.uint64), np.repeat(edges, 17)])
    codes = np.concatenate([rng.integers(0, 17, size=2000), np.tile(np.arange(17), edges.size)]).astype(np.uint8)
    cum = {c: np.concatenate([[0], np.cumsum(code == c)]) for c in range(16)}
    cum[16] = np.concatenate([[0], np.cumsum(B == ord("$"))])
    want_rank = np.array([cum[int(c)][int(x)] for c, x in zip(codes, ks)], np.uint64)
    pats = []
    for _ in range(80):
        j = int(rng.integers(0, m))
        r = reads[int(off[j]):int(off[j + 1])]
        a = int(rng.integers(0, max(1, r.size - 1)))
        pats.append(r[a:a + int(rng.integers(1, 15))].tobytes())
    pats += [b"ABCZ", b"", bytes(ALPHA[:3])]
    pbytes = np.frombuffer(b"".join(pats), np.uint8).copy()
    poffs = np.concatenate([[0], np.cumsum([len(p) for p in pats])]).astype(np.uint64)
    want_count = np.array([_occurrences(reads, off, p) for p in pats], np.uint64)
    r0, r1 = 64 * 11, n - 3
    rank_out = np.zeros(ks.size, np.uint64)
    count_out = np.zeros(len(pats), np.uint64)
    out = np.full((n + 63) // 64 * 64, 0xEE, np.uint8)
    alpha = np.frombuffer(ALPHA, np.uint8).copy()
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_queries_w(p(blocks), p(sup), p(C), n, p(alpha), sigma, p(codes), p(ks), ks.size, p(rank_out),
                             p(pbytes), pbytes.size, p(poffs), len(pats), p(count_out), r0, r1, p(out)) == 0
    assert np.array_equal(rank_out, want_rank)
    assert np.array_equal(count_out, want_count)
    assert want_count[:80].min() >= 1 and want_count[-3] == 0 and want_count[-2] == n
    assert np.array_equal(out[r0:r1], B[r0:r1])
    assert np.all(out[:r0] == 0xEE) and np.all(out[r1:] == 0xEE)


def append_text_w(reads: np.ndarray, off: np.ndarray) -> np.ndarray:
    """4-bit codes (index in the 12-symbol alphabet) of an append's positions,
    8 per word, MSB first, terminators as code 0, four zero words of padding."""
    from test_insert_w_emulation import codes_of
    m = len(off) - 1
    npos = int(off[-1]) + m
    codes = np.zeros(npos, np.uint32)
    pos = np.arange(int(off[-1])) + np.repeat(np.arange(m), np.diff(off.astype(np.int64)))
    codes[pos] = codes_of(reads).astype(np.uint32)
    nw = (npos + 7) // 8
    padded = np.zeros(nw * 8, np.uint32)
    padded[:npos] = codes
    sh = (28 - 4 * np.arange(8)).astype(np.uint32)
    words = np.bitwise_or.reduce(padded.reshape(nw, 8) << sh, axis=1).astype(np.uint32)
    return np.concatenate([words, np.zeros(4, np.uint32)])


def ragged_alpha(g, n, lo, hi, seed):
    """Reads of lengths lo..hi (some empty) sampled from genome g over the
    12-symbol alphabet."""
    from test_insert_w_emulation import ALPHA
    rng = np.random.default_rng(seed)
    full, _ = readgen.sampled_reads_alpha(g, n, hi, 0.02, seed, ALPHA)
    lens = rng.integers(lo, hi + 1, size=n)
    lens[::37] = 0
    rows = full.reshape(n, hi)
    reads = np.concatenate([rows[j, :lens[j]] for j in range(n)]).astype(np.uint8)
    return reads, readgen.offsets_from_lengths(lens)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("seg", [False, True])
@pytest.mark.parametrize("staged", [True, False])
def test_compute_ranks_4bit_matches_direct_counts(emu, seg, staged):
    """ComputeRanks over the 4-bit dictionary (both kernels, the superblock
    counters staged in shared memory or read from global memory) against the
    oracle's direct count of smaller old suffixes."""
    from test_insert_w_emulation import ALPHA
    sigma = len(ALPHA)
    g_ = readgen.genome_alpha(4_000, 17, np.full(sigma, 1.0 / sigma))
    hi = 1500 if seg else 90
    old = ragged_alpha(g_, 120 if seg else 300, 0, hi, 21)
    new = ragged_alpha(g_, 10 if seg else 120, 513 if seg else 0, hi, 22)
    B = oracle.bwt(old[0], old[1], ALPHA)
    m_ext = len(old[1]) - 1
    blocks, sup, C = dictionary_w(B, m_ext)
    text = append_text_w(*new)
    nreads = len(new[1]) - 1
    n_int = int(new[1][-1]) + nreads
    max_len = int(np.diff(new[1].astype(np.int64)).max())
    segs = max_len // SEG_ROWS + 1
    g = np.zeros(max(n_int, 1), np.uint32)
    err = ctypes.c_uint32(0)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    off = np.ascontiguousarray(new[1], np.uint64)
    assert emu.emu_compute_ranks_w(int(staged), int(seg), segs, SEG_ROWS, p(text), len(text), p(off), nreads,
                                   p(blocks), p(sup), p(C), len(B), m_ext, p(g), n_int, ctypes.byref(err)) == 0
    assert err.value == 0
    assert np.array_equal(g[:n_int], expected_g(old, new))
