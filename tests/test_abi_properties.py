"""Host-side argument checks of the C ABI on generated inputs, without a GPU:
an append's offsets (m+1 entries, starting at 0, never decreasing) and rank
queries (c in the alphabet or '$', 0 <= k <= n) are checked before any
device work, so on a machine without a GPU a bad call gives SBWT_EINVAL and
a good one reaches the device step (SBWT_EDEVICE) -- never a result
computed on the host.  Skipped where hypothesis is not installed or a GPU is
present."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import paper_1410_0562_gb300 as sb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _no_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: valid calls would run")
    sb.build()


def _offsets_valid(off) -> bool:
    return off[0] == 0 and all(b >= a for a, b in zip(off, off[1:]))


@settings(max_examples=200, deadline=None)
@given(st.lists(st.integers(0, 40), min_size=1, max_size=12),
       st.sampled_from([b"ACGT", b"AC", b"ACGNT", b"ABCDEFGHIJKLMNOP"]))
def test_append_offsets_checked_before_the_device(off, alphabet):
    h = sb.sbwt_create(alphabet)
    try:
        reads = np.full(max(off) + 1, alphabet[0], np.uint8)
        offsets = np.array(off, np.uint64)
        m = len(off) - 1
        if not _offsets_valid(off):
            expect = sb.SBWT_EINVAL
        elif m == 0:
            expect = sb.SBWT_OK
        else:
            expect = sb.SBWT_EDEVICE
        for call in (sb.sbwt_append, sb.sbwt_prepend):
            try:
                call(h, reads, offsets)
                rc = sb.SBWT_OK
            except sb.SbwtError as e:
                rc = e.code
            assert rc == expect
        assert sb.sbwt_size(h) == (0, 0)
    finally:
        sb.sbwt_destroy(h)


@settings(max_examples=200, deadline=None)
@given(st.lists(st.tuples(st.sampled_from(list(b"$ACGTN")), st.integers(0, 2)), max_size=6))
def test_rank_queries_checked_before_the_device(queries):
    h = sb.sbwt_create(b"ACGT")  # empty: n = 0
    try:
        cs = np.array([c for c, _ in queries], np.uint8)
        ks = np.array([k for _, k in queries], np.uint64)
        bad = any(c == ord("N") or k > 0 for c, k in queries)
        try:
            sb.sbwt_rank_batch(h, cs, ks)
            rc = sb.SBWT_OK
        except sb.SbwtError as e:
            rc = e.code
        if bad:
            assert rc == sb.SBWT_EINVAL
        else:
            assert rc == (sb.SBWT_EDEVICE if queries else sb.SBWT_OK)
    finally:
        sb.sbwt_destroy(h)
