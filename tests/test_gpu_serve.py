"""The served form: continuous batching of append requests.

Requests submitted while others run are coalesced into later batches; each
request's reads must land exactly as if the requests had been appended one by
one in arrival order, and the index must equal the oracle's BWT of the
concatenation.  A request with a byte outside the alphabet fails alone.
"""
import threading

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


def concat(reqs):
    reads = np.concatenate([r for r, _ in reqs]) if reqs else np.zeros(0, np.uint8)
    lengths = np.concatenate([np.diff(o.astype(np.int64)) for _, o in reqs])
    return reads, readgen.offsets_from_lengths(lengths)


def test_serving_equals_sequential_appends():
    rng = np.random.default_rng(5)
    reqs = [readgen.ragged_reads(int(rng.integers(1, 300)), 0, 150, seed=100 + i, p_empty=0.02)
            for i in range(48)]
    bad_at = 17
    bad_reads = reqs[bad_at][0].copy()
    bad_reads[len(bad_reads) // 2] = ord("N")
    reqs[bad_at] = (bad_reads, reqs[bad_at][1])

    idx = sb.SetBWT(b"ACGT", block_suffixes=40_000)
    sb.sbwt_serve_start(idx.handle, 0)
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for i in range(lo, hi):
            tickets[i] = sb.sbwt_submit(idx.handle, *reqs[i])

    # the first half from this thread, the rest from another one, while the
    # first batches already run
    submit(0, 24)
    t = threading.Thread(target=submit, args=(24, 48))
    t.start()
    with pytest.raises(sb.SbwtError) as e:
        idx.append(*reqs[0])  # only submit/wait while serving
    assert e.value.code == sb.SBWT_EBUSY
    t.join()
    results = {i: sb.sbwt_wait(idx.handle, tickets[i]) for i in range(len(reqs))}
    sb.sbwt_serve_stop(idx.handle)

    assert results[bad_at][0] == sb.SBWT_EINVAL
    order = sorted((i for i in range(len(reqs)) if i != bad_at), key=lambda i: tickets[i])
    first = 0
    for i in order:
        status, first_id, latency = results[i]
        assert status == sb.SBWT_OK and latency > 0
        assert first_id == first
        first += len(reqs[i][1]) - 1
    B = idx.bwt()
    # alone: the same requests appended one by one, in arrival order
    alone = sb.SetBWT(b"ACGT", block_suffixes=40_000)
    for i in order:
        alone.append(*reqs[i])
    assert np.array_equal(B, alone.bwt())
    reads, offsets = concat([reqs[i] for i in order])
    assert np.array_equal(B, oracle.bwt(reads, offsets))


def test_serving_with_batch_cap_and_graph_replay():
    reqs = [readgen.uniform_reads(200, 100, seed=300 + i) for i in range(20)]
    idx = sb.SetBWT(b"ACGT")
    sb.sbwt_set_graph_replay(idx.handle, True)
    sb.sbwt_serve_start(idx.handle, 3 * 200 * 100)  # at most three requests per batch
    tickets = [sb.sbwt_submit(idx.handle, *r) for r in reqs]
    res = [sb.sbwt_wait(idx.handle, tk) for tk in tickets]
    sb.sbwt_serve_stop(idx.handle)
    assert all(r[0] == sb.SBWT_OK for r in res)
    assert [r[1] for r in res] == [200 * i for i in range(20)]
    reads, offsets = concat(reqs)
    assert np.array_equal(idx.bwt(), oracle.bwt(reads, offsets))
