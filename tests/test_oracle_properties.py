"""Property-based pins of the oracle (hypothesis generates the read sets):
the brute-force rotation sort, the block-partition identity of Algorithm 1
in both block orders, Lemma-1 ranks against direct counts, and LF
inversion, over alphabets of 1 to 16 symbols.  CPU only; skipped where
hypothesis is not installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import brute  # noqa: E402
import oracle  # noqa: E402
from test_oracle import pack  # noqa: E402

ALPHABETS = [b"A", b"AC", b"ACG", b"ACGT", b"ACGNT", b"ABCDEFGH", b"ABCDEFGHIJKLMNOP"]


@st.composite
def read_sets(draw, max_reads=8, max_len=8):
    alpha = draw(st.sampled_from(ALPHABETS))
    sym = st.sampled_from(list(alpha))
    reads = draw(st.lists(st.lists(sym, max_size=max_len).map(bytes), max_size=max_reads))
    return alpha, reads


@settings(max_examples=150, deadline=None)
@given(read_sets())
def test_bwt_equals_sorted_rotations(case):
    alpha, reads = case
    data, off = pack(reads)
    assert bytes(oracle.bwt(data, off, alpha)) == brute.bwt(reads)


@settings(max_examples=100, deadline=None)
@given(read_sets(max_reads=12, max_len=12), st.data())
def test_any_partition_any_order_gives_the_same_bwt(case, data_st):
    alpha, reads = case
    m = len(reads)
    if m == 0:  # a partition needs at least one block
        return
    data, off = pack(reads)
    expect = oracle.bwt(data, off, alpha)
    cuts = data_st.draw(st.lists(st.integers(0, m), max_size=4))
    bounds = sorted(set([0, m] + cuts))
    assert np.array_equal(oracle.setbwte(data, off, bounds, alphabet=alpha), expect)
    assert np.array_equal(oracle.setbwte(data, off, bounds, alphabet=alpha, reverse=True), expect)


@settings(max_examples=100, deadline=None)
@given(read_sets(max_reads=12, max_len=10), st.data())
def test_lemma1_ranks_and_inversion(case, data_st):
    alpha, reads = case
    m = len(reads)
    if m < 2:
        return
    data, off = pack(reads)
    j0 = data_st.draw(st.integers(1, m - 1))
    d_old, o_old = pack(reads[:j0])
    B_ext = oracle.bwt(d_old, o_old, alpha)
    assert np.array_equal(oracle.block_g_lemma1(B_ext, data, off, j0, m, alphabet=alpha),
                          oracle.block_g_direct(data, off, j0, m))
    B = oracle.bwt(data, off, alpha)
    rec, roff = oracle.lf_invert(B, m, alphabet=alpha)
    assert np.array_equal(rec, data) and np.array_equal(roff, off)
