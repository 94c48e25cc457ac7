"""Pins the CPU oracle to things other than itself (no GPU needed).

* brute-force rotation sorting on tiny random sets (tests/brute.py);
* textbook and hand-derived BWTs (tests/golden/bwt_examples.txt);
* invariants of any set BWT: B is a permutation of T with exactly m '$',
  rows 0..m-1 hold the last symbol of each read, LF inversion recovers
  every read;
* the block-partition identity of Algorithm 1: any partition gives the
  one-shot BWT of Eq. 1;
* Lemma 1 / Algorithm 2 ranks equal the directly counted ranks;
* rank equals a numpy count.
"""
import os

import numpy as np
import pytest

import brute
import oracle
import readgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bwt_examples.txt")


def load_golden():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            alpha, reads, expect, _src = [x.strip() for x in line.split(" | ")]
            rs = [b"" if r == "-" else r.encode() for r in reads.split(",")]
            cases.append((alpha.encode(), rs, expect.encode()))
    return cases


def pack(reads):
    off = readgen.offsets_from_lengths([len(r) for r in reads])
    data = np.frombuffer(b"".join(reads), dtype=np.uint8) if reads and sum(map(len, reads)) else np.zeros(0, np.uint8)
    return data, off


def random_set(rng, m, max_len, alphabet=b"ACGT", p_empty=0.15):
    reads = []
    for _ in range(m):
        L = 0 if rng.random() < p_empty else int(rng.integers(1, max_len + 1))
        # a small alphabet slice makes long shared prefixes likely
        k = int(rng.integers(1, len(alphabet) + 1))
        reads.append(bytes(rng.choice(np.frombuffer(alphabet[:k], np.uint8), size=L)))
    return reads


@pytest.mark.parametrize("alpha,reads,expect", load_golden())
def test_golden_bwt(alpha, reads, expect):
    data, off = pack(reads)
    assert bytes(oracle.bwt(data, off, alpha)) == expect
    assert brute.bwt(reads) == expect


@pytest.mark.parametrize("seed", range(60))
def test_oracle_vs_brute_force(seed):
    rng = np.random.default_rng(seed)
    reads = random_set(rng, int(rng.integers(0, 10)), 9)
    data, off = pack(reads)
    assert bytes(oracle.bwt(data, off)) == brute.bwt(reads)


@pytest.mark.parametrize("seed", range(12))
def test_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    reads = random_set(rng, int(rng.integers(1, 40)), 30)
    data, off = pack(reads)
    B = oracle.bwt(data, off)
    m = len(reads)
    # permutation of T: same multiset of symbols, exactly m terminators
    T = b"".join(r + b"$" for r in reads)
    assert sorted(bytes(B)) == sorted(T)
    assert int(np.count_nonzero(B == ord("$"))) == m
    # rows 0..m-1 are $_0..$_{m-1}: B holds each read's last symbol ('$' if empty)
    for r, s in enumerate(reads):
        assert B[r] == (s[-1] if s else ord("$"))
    # LF inversion recovers every read
    rec, roff = oracle.lf_invert(B, m)
    assert brute.to_set(rec, roff) == reads


@pytest.mark.parametrize("seed", range(6))
def test_sampled_lf_invert_matches_full(seed):
    rng = np.random.default_rng(700 + seed)
    reads = random_set(rng, int(rng.integers(1, 120)), 150)
    data, off = pack(reads)
    B = oracle.bwt(data, off)
    a = oracle.lf_invert(B, len(reads))
    b = oracle.lf_invert_sampled(B, len(reads))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert brute.to_set(*b) == reads
    bad = B.copy()
    bad[len(reads)] = ord("$") if bad[len(reads)] != ord("$") else ord("A")
    with pytest.raises(oracle.OracleError):
        oracle.lf_invert_sampled(bad, len(reads))


def test_lf_invert_rejects_broken_bwt():
    data, off = pack([b"ACGTTGCA", b"GATTACA"])
    B = oracle.bwt(data, off).copy()
    bad = B.copy()
    i = 2  # swap row 2 with the first later row holding a different symbol
    j = next(k for k in range(3, len(B)) if B[k] != B[i])
    bad[i], bad[j] = bad[j], bad[i]
    rec = None
    try:
        rec, roff = oracle.lf_invert(bad, 2)
    except oracle.OracleError:
        pass
    if rec is not None:
        assert brute.to_set(rec, roff) != [b"ACGTTGCA", b"GATTACA"]
    with pytest.raises(oracle.OracleError):
        oracle.lf_invert(B, 3)  # wrong number of terminators


@pytest.mark.parametrize("seed", range(10))
def test_block_intermediates_vs_brute(seed):
    rng = np.random.default_rng(200 + seed)
    reads = random_set(rng, int(rng.integers(2, 9)), 7)
    data, off = pack(reads)
    m = len(reads)
    j0 = int(rng.integers(0, m))
    j1 = int(rng.integers(j0 + 1, m + 1))
    block = reads[j0:j1]
    # SA_int: brute-force rotation order of the block alone; block-local
    # positions are the positions of the block's own text
    sa = oracle.block_sa(data, off, j0, j1)
    assert list(sa) == brute.sorted_rotations(block)
    # B_int is the block's own set BWT
    bint = oracle.block_bint(data, off, j0, j1, sa)
    assert bytes(bint) == brute.bwt(block)
    # g: old suffixes below each block suffix, from the brute-force union order
    g = oracle.block_g_direct(data, off, j0, j1)
    assert list(g) == brute.g_values(reads[:j0], block)


@pytest.mark.parametrize("seed", range(10))
def test_lemma1_ranks_equal_direct_ranks(seed):
    rng = np.random.default_rng(300 + seed)
    reads = random_set(rng, int(rng.integers(2, 60)), 25)
    data, off = pack(reads)
    m = len(reads)
    j0 = int(rng.integers(1, m))
    j1 = int(rng.integers(j0 + 1, m + 1))
    d_old, o_old = pack(reads[:j0])
    B_ext = oracle.bwt(d_old, o_old)
    g1 = oracle.block_g_lemma1(B_ext, data, off, j0, j1)
    g2 = oracle.block_g_direct(data, off, j0, j1)
    assert np.array_equal(g1, g2)


WIDE_ALPHABETS = [b"ACGNT", b"ABCDEFGH", b"ABCDEFGHIJKLMNOP", bytes(range(0x61, 0x61 + 13))]


@pytest.mark.parametrize("seed", range(24))
def test_wide_alphabet_vs_brute_force(seed):
    """Alphabets of 5 to 16 symbols: the same definition (Eq. 1), symbols
    ordered by byte value."""
    rng = np.random.default_rng(900 + seed)
    alpha = WIDE_ALPHABETS[seed % len(WIDE_ALPHABETS)]
    reads = random_set(rng, int(rng.integers(0, 10)), 9, alphabet=alpha)
    data, off = pack(reads)
    assert bytes(oracle.bwt(data, off, alpha)) == brute.bwt(reads)


@pytest.mark.parametrize("seed", range(6))
def test_wide_alphabet_partition_lemma1_and_inversion(seed):
    rng = np.random.default_rng(950 + seed)
    alpha = WIDE_ALPHABETS[seed % len(WIDE_ALPHABETS)]
    reads = random_set(rng, int(rng.integers(2, 50)), 30, alphabet=alpha)
    data, off = pack(reads)
    m = len(reads)
    one_shot = oracle.bwt(data, off, alpha)
    cuts = sorted(set(int(x) for x in rng.integers(1, m, size=3)))
    bounds = [0] + cuts + [m]
    assert np.array_equal(oracle.setbwte(data, off, bounds, alphabet=alpha), one_shot)
    assert np.array_equal(oracle.setbwte(data, off, bounds, alphabet=alpha, reverse=True), one_shot)
    j0 = int(rng.integers(1, m))
    d_old, o_old = pack(reads[:j0])
    B_ext = oracle.bwt(d_old, o_old, alpha)
    assert np.array_equal(oracle.block_g_lemma1(B_ext, data, off, j0, m, alphabet=alpha),
                          oracle.block_g_direct(data, off, j0, m))
    rec, roff = oracle.lf_invert(one_shot, m, alphabet=alpha)
    assert np.array_equal(rec, data) and np.array_equal(roff, off)


def test_alphabet_size_limit():
    with pytest.raises(oracle.OracleError):
        oracle.bwt(*pack([b"AB"]), alphabet=bytes(range(0x41, 0x41 + 17)))


def test_worked_example_intermediates():
    """AC then A: Algorithm 1 step by step (derivation in tests/golden)."""
    data, off = pack([b"AC", b"A"])
    B_ext = oracle.bwt(*pack([b"AC"]))
    assert bytes(B_ext) == b"C$A"
    g = oracle.block_g_lemma1(B_ext, data, off, 1, 2)
    assert list(g) == [1, 1]
    sa = oracle.block_sa(data, off, 1, 2)
    assert list(sa) == [1, 0]
    bint = oracle.block_bint(data, off, 1, 2, sa)
    assert bytes(bint) == b"A$"
    gsa = g[sa.astype(np.int64)]
    assert list(gsa) == [1, 1]
    assert bytes(oracle.insert(B_ext, bint, gsa)) == b"CA$$A"
    # the literal start value i := n_ext would give g_sa = [3, 2], which is
    # not non-decreasing, so Insert must refuse it
    with pytest.raises(oracle.OracleError):
        oracle.insert(B_ext, bint, np.array([3, 2], np.uint64))


@pytest.mark.parametrize("seed", range(8))
def test_block_partition_identity(seed):
    rng = np.random.default_rng(400 + seed)
    reads = random_set(rng, int(rng.integers(1, 80)), 40)
    data, off = pack(reads)
    m = len(reads)
    one_shot = oracle.bwt(data, off)
    cuts = sorted(set(int(x) for x in rng.integers(1, m + 1, size=int(rng.integers(0, 6))))) if m > 1 else []
    bounds = [0] + [c for c in cuts if 0 < c < m] + [m]
    assert np.array_equal(oracle.setbwte(data, off, bounds), one_shot)
    assert np.array_equal(oracle.setbwte(data, off, list(range(m + 1))), one_shot)  # one read per block
    # the reverse order (Section 2): the same blocks from last to first
    assert np.array_equal(oracle.setbwte(data, off, bounds, reverse=True), one_shot)
    assert np.array_equal(oracle.setbwte(data, off, list(range(m + 1)), reverse=True), one_shot)


def test_partition_identity_tiny_workload():
    """1,000 x 100 bp i.i.d. reads appended as 2 x 500 (and as 7 ragged blocks)."""
    w = readgen.tiny()
    one_shot = oracle.bwt(w.reads, w.offsets)
    assert np.array_equal(oracle.setbwte(w.reads, w.offsets, list(w.appends)), one_shot)
    assert np.array_equal(oracle.setbwte(w.reads, w.offsets, [0, 1, 13, 200, 499, 500, 877, 1000]), one_shot)
    assert np.array_equal(oracle.setbwte(w.reads, w.offsets, [0, 1, 13, 200, 499, 500, 877, 1000], reverse=True),
                          one_shot)
    rec, roff = oracle.lf_invert(one_shot, w.m)
    assert np.array_equal(rec, w.reads) and np.array_equal(roff, w.offsets)


def test_rank_is_a_count():
    rng = np.random.default_rng(7)
    B = rng.choice(np.frombuffer(b"$ACGT", np.uint8), size=1000)
    for c in b"$ACGT":
        for k in [0, 1, 2, 63, 64, 65, 500, 999, 1000]:
            assert oracle.rank(B, c, k) == int(np.count_nonzero(B[:k] == c))


def test_row_of_suffix_vs_brute():
    rng = np.random.default_rng(11)
    reads = random_set(rng, 7, 8)
    data, off = pack(reads)
    rows = brute.suffix_rows(reads)
    B = brute.bwt(reads)
    for (r, p), row in rows.items():
        assert oracle.row_of_suffix(data, off, r, p) == row
        assert oracle.bwt_symbol_of_suffix(data, off, r, p) == B[row]


def test_rejects_bad_input():
    data, off = pack([b"ACGN"])
    with pytest.raises(oracle.OracleError):
        oracle.bwt(data, off)
    with pytest.raises(oracle.OracleError):
        oracle.bwt(*pack([b"AC"]), alphabet=b"CA")  # not increasing
    with pytest.raises(oracle.OracleError):
        oracle.bwt(np.frombuffer(b"ACGT", np.uint8), np.array([0, 3, 2, 4], np.uint64))


def test_empty_set():
    assert len(oracle.bwt(np.zeros(0, np.uint8), np.zeros(1, np.uint64))) == 0
    assert bytes(oracle.bwt(*pack([b"", b"", b""]))) == b"$$$"


@pytest.mark.parametrize("seed", range(5))
def test_count_is_overlapping_substring_count(seed):
    rng = np.random.default_rng(900 + seed)
    reads = random_set(rng, 30, 40, alphabet=b"AC")
    data, off = pack(reads)
    for L in (1, 2, 3, 5):
        for _ in range(5):
            pat = bytes(rng.choice(np.frombuffer(b"AC", np.uint8), size=L))
            expect = sum(1 for r in reads for p in range(len(r) - L + 1) if r[p:p + L] == pat)
            assert oracle.count(data, off, pat) == expect
