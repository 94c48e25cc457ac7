"""sbwt_save / sbwt_load: a saved and reloaded index answers like the one
that wrote it, and later appends continue it exactly (checked against the
oracle's BWT of all reads)."""
import numpy as np
import pytest

import oracle
import paper_1410_0562_gb300 as sb
import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def concat(parts):
    reads = np.concatenate([r for r, _ in parts])
    lengths = np.concatenate([np.diff(o.astype(np.int64)) for _, o in parts])
    return reads, readgen.offsets_from_lengths(lengths)


@pytest.mark.parametrize("index_bits,host_tier", [(32, 0), (64, 0), (32, 3)])
def test_round_trip_then_append(tmp_path, index_bits, host_tier):
    a = readgen.ragged_reads(700, 0, 160, seed=71, p_empty=0.02, p_repeat=0.05)
    b = readgen.ragged_reads(500, 1, 120, seed=72)
    idx = sb.SetBWT(b"ACGT", index_bits=index_bits, block_suffixes=30_000)
    idx.append(*a)
    path = tmp_path / "idx.sbwt"
    idx.save(path)
    back = sb.SetBWT.load(path, block_suffixes=30_000, host_tier=host_tier)
    assert back.size() == idx.size()
    assert np.array_equal(back.bwt(), idx.bwt())
    n, _ = idx.size()
    ks = np.arange(0, n + 1, 37, dtype=np.uint64)
    for c in b"ACGT$":
        cs = np.full(len(ks), c, np.uint8)
        assert np.array_equal(back.rank_batch(cs, ks), idx.rank_batch(cs, ks))
    pats = [b"A", b"ACG", b"TTT", b"GATTACA", b""]
    assert np.array_equal(back.count(pats), idx.count(pats))
    if host_tier == 3:
        hbm, host = sb.sbwt_memory(back.handle)
        assert host > 0
    # appends continue the read ids of the saved index
    idx.append(*b)
    back.append(*b)
    expect = oracle.bwt(*concat([a, b]))
    assert np.array_equal(idx.bwt(), expect)
    assert np.array_equal(back.bwt(), expect)


def test_empty_index_round_trip(tmp_path):
    path = tmp_path / "empty.sbwt"
    sb.SetBWT(b"ACG").save(path)
    back = sb.SetBWT.load(path)
    assert back.size() == (0, 0)
    r = readgen.uniform_reads(50, 30, seed=5, alphabet=b"ACG")
    back.append(*r)
    assert np.array_equal(back.bwt(), oracle.bwt(*r, alphabet=b"ACG"))
