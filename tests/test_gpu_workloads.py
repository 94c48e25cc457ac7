"""Bit-exact parity of the CUDA path with the oracle's whole B (Eq. 1) on the
full-size workloads, element by element.

* short reads: 1M x 100 bp from a 10 Mbp genome, blocks of 2^24 suffixes,
  32-bit indices -- the configuration the benchmark times;
* batched: 2M reads of U[50, 250] bp from a 50 Mbp genome, 64-bit indices;
* long reads: 20k log-normal reads (mean 10 kbp) with 10% errors from a
  100 Mbp genome, 64-bit indices;
* served, at 1/20 of its size in every dimension: a resident index of 1M x
  100 bp reads, then 48 requests of 500 to 50k reads of U[100, 150] bp
  submitted to the continuous-batching server while it runs, so batches
  coalesce several requests; B must equal the oracle's B of every read in
  arrival order.

The oracle (single-threaded, minutes per workload) runs in background
processes from the start of the session (``oracle_jobs``).  Exact integer
work: every comparison is equality, there is no tolerance.
"""
import threading
import time

import numpy as np
import pytest

import oracle_jobs
import paper_1410_0562_gb300 as sb
import readgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def build_device(w, M, index_bits, replay=False):
    """B through sbwt_append_device, as the benchmark runs it."""
    import torch
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(w.alphabet, index_bits=index_bits, block_suffixes=M)
    if replay:
        sb.sbwt_set_graph_replay(idx.handle, True)
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    B = idx.bwt()
    assert idx.size() == (len(B), w.m)
    idx.close()
    return B


def assert_same(B, expect):
    assert len(B) == len(expect)
    if not np.array_equal(B, expect):
        bad = np.nonzero(B != expect)[0]
        raise AssertionError(f"{len(bad)} rows differ, first at {bad[:8].tolist()}")


@pytest.mark.oracle_full("short")
def test_short_reads_full_size_equals_oracle():
    w = readgen.short()
    B = build_device(w, w.block_suffixes, w.index_bits)
    assert_same(B, oracle_jobs.result("short"))


@pytest.mark.oracle_full("batched")
def test_batched_workload_full_size_equals_oracle():
    w = readgen.batched()
    B = build_device(w, 1 << 25, 64)
    assert_same(B, oracle_jobs.result("batched"))


@pytest.mark.oracle_full("long")
def test_long_reads_full_size_equals_oracle():
    w = readgen.long()
    B = build_device(w, 1 << 25, 64)
    assert_same(B, oracle_jobs.result("long"))


@pytest.mark.oracle_full("serving_20")
def test_served_workload_one_twentieth_equals_oracle():
    resident, requests = readgen.serving_scaled(20)
    idx = sb.SetBWT(b"ACGT", hbm_budget=8 << 30, index_bits=64, block_suffixes=1 << 25)
    idx.append(resident.reads, resident.offsets)
    sb.sbwt_serve_start(idx.handle, 0)
    tickets = [None] * len(requests)
    gaps = np.random.default_rng(20).exponential(0.004, size=len(requests))

    def submit():
        for i, (r, o) in enumerate(requests):
            time.sleep(gaps[i])
            tickets[i] = sb.sbwt_submit(idx.handle, r, o)

    th = threading.Thread(target=submit)
    th.start()
    th.join()
    first_ids = []
    for t in tickets:
        rc, first, _ = sb.sbwt_wait(idx.handle, t)
        assert rc == sb.SBWT_OK
        first_ids.append(first)
    sb.sbwt_serve_stop(idx.handle)
    # read ids follow arrival order
    sizes = [len(o) - 1 for _, o in requests]
    assert first_ids == list(resident.m + np.concatenate([[0], np.cumsum(sizes)[:-1]]))
    B = idx.bwt()
    idx.close()
    assert_same(B, oracle_jobs.result("serving_20"))


@pytest.mark.oracle_full("short")
def test_short_reads_host_tier_equals_oracle():
    """The short-read workload with its one dictionary in pinned host memory
    (occurrence sampling 256), rewritten in place by every block's Insert,
    from the top down in chunks staged in HBM (a 101M-row dictionary spans
    four chunks): B equals the oracle's, and the host holds at most 6 bits per
    row (the paper's bound of 3 n log sigma bits for DNA)."""
    import torch
    w = readgen.short()
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(w.alphabet, index_bits=w.index_bits, block_suffixes=w.block_suffixes, host_tier=3,
                    occ_sampling=256)
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    n, _ = idx.size()
    hbm, host = sb.sbwt_memory(idx.handle)
    assert 8.0 * host / n <= 6.0
    B = idx.bwt()
    idx.close()
    assert_same(B, oracle_jobs.result("short"))
