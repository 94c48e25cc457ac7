"""Alphabets of 5 to 16 symbols (4-bit codes) through the C ABI against the
CPU oracle, bit-exact: B, each block's intermediates, rank and count
queries, persistence, prepends and the host tier.

The definition (Eq. 1) is the same for any alphabet; with more than 4
symbols the text and the rank dictionary hold 4-bit codes (64-byte
occurrence blocks of 64 rows, superblocks of 4096 rows) and the suffix keys
14 codes, so these tests also cross those block and superblock sizes.
"""
import os

import numpy as np
import pytest

import oracle
import paper_1410_0562_gb300 as sb
import readgen
from test_gpu_parity import check_full_size
from test_oracle import pack

pytestmark = pytest.mark.gpu

WIDE = [b"ACGNT", b"ABCDEFGH", b"ABCDEFGHIJKLMNOP", b"abcdefghijklm"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def random_reads(rng, alpha, m, max_len):
    sym = np.frombuffer(alpha, np.uint8)
    reads = []
    for _ in range(m):
        kind = rng.random()
        if kind < 0.08:
            reads.append(b"")
        elif kind < 0.2:  # one symbol repeated: long shared prefixes
            reads.append(bytes([alpha[rng.integers(0, len(alpha))]]) * int(rng.integers(1, 150)))
        elif kind < 0.3:  # a short tandem repeat
            unit = bytes(rng.choice(sym, size=int(rng.integers(1, 4))))
            reads.append((unit * 200)[: int(rng.integers(1, 250))])
        elif kind < 0.4 and reads:  # an exact duplicate
            reads.append(reads[int(rng.integers(0, len(reads)))])
        else:
            k = int(rng.integers(2, len(alpha) + 1))  # a slice of the alphabet: more repeats
            reads.append(bytes(rng.choice(sym[:k], size=int(rng.integers(1, max_len)))))
    return reads


def build(alpha, data, off, M=0, cuts=None, index_bits=0, capture=False, host_tier=0):
    m = len(off) - 1
    cuts = list(cuts) if cuts else [0, m]
    idx = sb.SetBWT(alpha, index_bits=index_bits, block_suffixes=M, host_tier=host_tier)
    if capture:
        sb.sbwt_set_capture(idx.handle, True)
    off = np.asarray(off, np.uint64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        idx.append(np.ascontiguousarray(data[int(off[a]):int(off[b])]), off[a:b + 1] - off[a])
    return idx


@pytest.mark.parametrize("seed", range(16))
def test_wide_random_sets(seed):
    rng = np.random.default_rng(3000 + seed)
    alpha = WIDE[seed % len(WIDE)]
    reads = random_reads(rng, alpha, int(rng.integers(1, 300)), 160)
    data, off = pack(reads)
    m = len(reads)
    expect = oracle.bwt(data, off, alpha)
    M = int(rng.choice([1, 50, 500, 5000, 1 << 20]))
    cuts = sorted(set([0, m] + [int(x) for x in rng.integers(0, m, size=int(rng.integers(0, 4)))]))
    idx = build(alpha, data, off, M=M, cuts=cuts, index_bits=int(rng.choice([0, 32, 64])))
    assert np.array_equal(idx.bwt(), expect)


def test_wide_block_intermediates():
    """SA_int, B_int, g and g_sa of the last block of a two-append build."""
    rng = np.random.default_rng(31)
    alpha = b"ACGNT"
    reads = random_reads(rng, alpha, 400, 120)
    data, off = pack(reads)
    j0 = 250
    idx = build(alpha, data, off, cuts=[0, j0, len(reads)], capture=True)
    sa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_SA)
    assert np.array_equal(sa, oracle.block_sa(data, off, j0, len(reads)))
    lut = np.zeros(256, np.uint8)
    lut[: len(alpha)] = np.frombuffer(alpha, np.uint8)
    lut[255] = ord("$")
    bint = lut[sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_BINT)]
    assert np.array_equal(bint, oracle.block_bint(data, off, j0, len(reads), sa))
    g = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_G)
    assert np.array_equal(g, oracle.block_g_direct(data, off, j0, len(reads)))
    gsa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_GSA)
    assert np.array_equal(gsa, g[sa])


@pytest.mark.parametrize("n_int", [4095, 4096, 4097, 8193, 65537])
def test_wide_superblock_boundaries(n_int):
    """Sizes around the 4-bit dictionary's 4096-row superblocks."""
    rng = np.random.default_rng(n_int)
    alpha = b"ABCDEFGHIJKLMNOP"
    lengths = []
    left = n_int
    while left > 0:
        L = min(int(rng.integers(0, 120)), left - 1)
        lengths.append(L)
        left -= L + 1
    off = readgen.offsets_from_lengths(lengths)
    data = rng.choice(np.frombuffer(alpha, np.uint8), size=int(off[-1]))
    expect = oracle.bwt(data, off, alpha)
    assert np.array_equal(build(alpha, data, off).bwt(), expect)
    h = len(lengths) // 2
    assert np.array_equal(build(alpha, data, off, cuts=[0, h, len(lengths)]).bwt(), expect)


def test_wide_rank_and_count_queries():
    rng = np.random.default_rng(77)
    alpha = b"abcdefghijklm"
    reads = random_reads(rng, alpha, 1500, 100)
    data, off = pack(reads)
    idx = build(alpha, data, off, M=20_000, cuts=[0, 700, 1500])
    B = oracle.bwt(data, off, alpha)
    n = len(B)
    ks = np.concatenate([[0, 1, 63, 64, 65, 4095, 4096, 4097, 8192, n - 1, n],
                         rng.integers(0, n + 1, size=200)]).astype(np.uint64)
    for c in b"$" + alpha:
        cum = np.concatenate([[0], np.cumsum(B == c)])
        assert np.array_equal(idx.rank_batch(np.full(len(ks), c, np.uint8), ks), cum[ks.astype(np.int64)])
    pats = [b"", b"a", b"m", b"z", b"abc", b"mmmm"]
    for L in (1, 2, 3, 5, 9, 20):
        for _ in range(5):
            r = reads[int(rng.integers(0, len(reads)))]
            if len(r) >= L:
                p0 = int(rng.integers(0, len(r) - L + 1))
                pats.append(r[p0:p0 + L])
            pats.append(bytes(rng.choice(np.frombuffer(alpha, np.uint8), size=L)))
    got = idx.count(pats)
    expect = [oracle.count(data, off, p) if all(c in alpha for c in p) else 0 for p in pats]
    assert list(got) == expect


def test_wide_save_load_prepend_and_host_tier(tmp_path):
    rng = np.random.default_rng(91)
    alpha = b"ACGNT"
    a = random_reads(rng, alpha, 300, 90)
    b = random_reads(rng, alpha, 200, 120)
    c = random_reads(rng, alpha, 150, 60)
    idx = sb.SetBWT(alpha, block_suffixes=7_000)
    idx.append(*pack(b))
    idx.prepend(*pack(a))  # a b
    path = os.path.join(str(tmp_path), "wide.sbwt")
    idx.save(path)
    loaded = sb.SetBWT.load(path)
    assert np.array_equal(loaded.bwt(), idx.bwt())
    loaded.append(*pack(c))  # a b c
    expect = oracle.bwt(*pack(a + b + c), alpha)
    assert np.array_equal(loaded.bwt(), expect)
    # the same reads with the dictionaries in pinned host memory
    h = sb.SetBWT(alpha, block_suffixes=7_000, host_tier=3)
    h.append(*pack(a + b))
    h.append(*pack(c))
    assert np.array_equal(h.bwt(), expect)


def test_wide_larger_genome_reads():
    """20k reads x 100 bp over A,C,G,N,T from a 400 kbp genome (5x
    coverage; the CTA-local sorts and three doubling rounds of 14-code
    keys), then 3,000 x 80 bp reads from a 300-symbol genome (~800x
    coverage: buckets and groups far over the CTA-local capacity, so the
    device-wide path runs)."""
    rng = np.random.default_rng(2024)
    genome = rng.choice(np.frombuffer(b"ACGNT", np.uint8), size=400_000, p=[0.24, 0.24, 0.24, 0.04, 0.24])
    starts = rng.integers(0, len(genome) - 100, size=20_000)
    reads = [bytes(genome[s:s + 100]) for s in starts]
    data, off = pack(reads)
    expect = oracle.bwt(data, off, b"ACGNT")
    assert np.array_equal(build(b"ACGNT", data, off).bwt(), expect)
    assert np.array_equal(build(b"ACGNT", data, off, M=1 << 16, cuts=[0, 9_000, 20_000]).bwt(), expect)
    small = rng.choice(np.frombuffer(b"ACGNT", np.uint8), size=300)
    starts = rng.integers(0, len(small) - 80, size=3_000)
    reads = [bytes(small[s:s + 80]) for s in starts]
    data, off = pack(reads)
    expect = oracle.bwt(data, off, b"ACGNT")
    assert np.array_equal(build(b"ACGNT", data, off).bwt(), expect)


def test_wide_workload_full_size():
    """The wide workload (1M x 100 bp over A,C,G,N,T, blocks of 2^24) in the
    launch configuration the benchmark times: multiset, terminator rows,
    sampled rows counted by the oracle and LF inversion of the whole B."""
    w = readgen.wide()
    idx = build(w.alphabet, w.reads, w.offsets, M=w.block_suffixes, index_bits=w.index_bits)
    assert idx.size() == (oracle.num_suffixes(w.offsets), w.m)
    check_full_size(w, idx.bwt(), samples=2)
