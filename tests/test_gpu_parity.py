"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is exact integer work, so every comparison is bit-exact:
the BWT, each block's intermediates (SA_int, B_int, g, g_sa), and rank
queries.  Inputs are seeded and synthetic (readgen) or hand-made edge cases.
"""
import numpy as np
import pytest

import oracle
import paper_1410_0562_gb300 as sb
import readgen
from test_oracle import load_golden, pack

pytestmark = pytest.mark.gpu

CODE_BYTES = {255: ord("$")}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def gpu_bwt(reads, offsets, alphabet=b"ACGT", M=0, cuts=None, index_bits=0, capture=False, occ_sampling=0):
    """Build through the C ABI, appending reads [cuts[k], cuts[k+1]) per call."""
    m = len(offsets) - 1
    cuts = list(cuts) if cuts else [0, m]
    idx = sb.SetBWT(alphabet, index_bits=index_bits, block_suffixes=M, occ_sampling=occ_sampling)
    if capture:
        sb.sbwt_set_capture(idx.handle, True)
    offsets = np.asarray(offsets, np.uint64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        o = offsets[a:b + 1] - offsets[a]
        idx.append(np.ascontiguousarray(reads[int(offsets[a]):int(offsets[b])]), o)
    return idx


def bint_bytes(bint_codes, alphabet=b"ACGT"):
    lut = np.zeros(256, np.uint8)
    for i, c in enumerate(alphabet):
        lut[i] = c
    lut[255] = ord("$")
    return lut[bint_codes]


@pytest.mark.parametrize("alpha,reads,expect", load_golden())
def test_golden_examples(alpha, reads, expect):
    data, off = pack(reads)
    assert bytes(gpu_bwt(data, off, alpha).bwt()) == expect
    # one read per append gives the same B (Algorithm 1, forward order)
    assert bytes(gpu_bwt(data, off, alpha, cuts=range(len(reads) + 1)).bwt()) == expect


def test_tiny_workload_and_intermediates():
    """1,000 x 100 bp i.i.d. reads appended as 2 x 500: B and every
    intermediate of the second block against the oracle."""
    w = readgen.tiny()
    idx = gpu_bwt(w.reads, w.offsets, M=w.block_suffixes, cuts=w.appends, capture=True)
    B = idx.bwt()
    expect = oracle.bwt(w.reads, w.offsets)
    assert np.array_equal(B, expect)
    j0, j1 = 500, 1000
    sa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_SA)
    assert np.array_equal(sa.astype(np.uint64), oracle.block_sa(w.reads, w.offsets, j0, j1))
    bint = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_BINT)
    assert np.array_equal(bint_bytes(bint), oracle.block_bint(w.reads, w.offsets, j0, j1, sa))
    g = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_G)
    assert np.array_equal(g, oracle.block_g_direct(w.reads, w.offsets, j0, j1))
    gsa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_GSA)
    assert np.array_equal(gsa, g[sa.astype(np.int64)])
    assert np.all(np.diff(gsa.astype(np.int64)) >= 0)
    assert idx.size() == (len(expect), w.m)


def test_first_block_intermediates():
    """The first block ranks against an empty index: g = 0 everywhere."""
    w = readgen.tiny()
    idx = gpu_bwt(w.reads, w.offsets, cuts=[0, 500], capture=True)
    sa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_SA)
    assert np.array_equal(sa.astype(np.uint64), oracle.block_sa(w.reads, w.offsets, 0, 500))
    assert not np.any(sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_G))


@pytest.mark.parametrize("M", [1, 7, 64, 1000, 4096, 50_500, 1 << 24])
def test_block_partition_invariance(M):
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    assert np.array_equal(gpu_bwt(w.reads, w.offsets, M=M, cuts=w.appends).bwt(), expect)


@pytest.mark.parametrize("seed", range(24))
def test_random_edge_sets(seed):
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(1, 300))
    reads = []
    for _ in range(m):
        kind = rng.random()
        if kind < 0.1:
            reads.append(b"")
        elif kind < 0.25:  # a run of one base: long common prefixes
            reads.append(bytes([b"ACGT"[rng.integers(0, 4)]]) * int(rng.integers(1, 200)))
        elif kind < 0.35:  # a short tandem repeat
            unit = bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(rng.integers(1, 4))))
            reads.append((unit * 200)[: int(rng.integers(1, 300))])
        elif kind < 0.45 and reads:  # an exact duplicate
            reads.append(reads[int(rng.integers(0, len(reads)))])
        else:
            reads.append(bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(rng.integers(1, 150)))))
    data, off = pack(reads)
    expect = oracle.bwt(data, off)
    M = int(rng.choice([1, 50, 500, 5000, 1 << 20]))
    cuts = sorted(set([0, m] + [int(x) for x in rng.integers(0, m, size=int(rng.integers(0, 4)))]))
    idx = gpu_bwt(data, off, M=M, cuts=cuts, index_bits=int(rng.choice([0, 32, 64])))
    assert np.array_equal(idx.bwt(), expect)


@pytest.mark.parametrize("alphabet", [b"A", b"AC", b"ACG", b"abn", b"imps"])
def test_small_alphabets(alphabet):
    rng = np.random.default_rng(len(alphabet))
    reads = [bytes(rng.choice(np.frombuffer(alphabet, np.uint8), size=int(rng.integers(0, 80))))
             for _ in range(200)]
    data, off = pack(reads)
    expect = oracle.bwt(data, off, alphabet)
    assert np.array_equal(gpu_bwt(data, off, alphabet, M=777, cuts=[0, 60, 200]).bwt(), expect)


def test_long_reads_many_doubling_rounds():
    """Reads up to 3 kbp sharing long prefixes need several doubling rounds."""
    rng = np.random.default_rng(5)
    base = bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=3000))
    reads = [base[int(rng.integers(0, 50)):][: int(rng.integers(500, 2950))] for _ in range(40)]
    reads += [b"A" * 2500, b"A" * 2499, b"AC" * 1200, b"A" * 2500]
    data, off = pack(reads)
    expect = oracle.bwt(data, off)
    assert np.array_equal(gpu_bwt(data, off, M=30_000, cuts=[0, 20, 44]).bwt(), expect)


@pytest.mark.parametrize("n_int", [4095, 4096, 4097, 8193, 65535, 65536, 65537])
def test_ragged_tile_and_superblock_sizes(n_int):
    """Blocks whose suffix count straddles a radix tile (4096) and B sizes
    that straddle a superblock (65536 rows)."""
    rng = np.random.default_rng(n_int)
    lengths = []
    left = n_int
    while left > 0:
        L = min(int(rng.integers(0, 120)), left - 1)
        lengths.append(L)
        left -= L + 1
    off = readgen.offsets_from_lengths(lengths)
    data = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(off[-1]))
    assert oracle.num_suffixes(off) == n_int
    expect = oracle.bwt(data, off)
    idx = gpu_bwt(data, off, capture=True)
    assert np.array_equal(idx.bwt(), expect)
    sa = sb.sbwt_get_stage(idx.handle, sb.SBWT_STAGE_SA)
    assert len(sa) == n_int
    # and appended in two halves
    h = len(lengths) // 2
    assert np.array_equal(gpu_bwt(data, off, cuts=[0, h, len(lengths)]).bwt(), expect)


def test_rank_queries_match_counts():
    w = readgen.tiny()
    idx = gpu_bwt(w.reads, w.offsets, cuts=w.appends)
    B = oracle.bwt(w.reads, w.offsets)
    n = len(B)
    rng = np.random.default_rng(3)
    ks = np.concatenate([[0, 1, 63, 64, 65, 65535, 65536, 65537, n - 1, n], rng.integers(0, n + 1, size=200)])
    for c in b"$ACGT":
        cum = np.concatenate([[0], np.cumsum(B == c)])
        got = idx.rank_batch(np.full(len(ks), c, np.uint8), ks.astype(np.uint64))
        assert np.array_equal(got, cum[ks])
    assert idx.rank("G", n) == int(np.count_nonzero(B == ord("G")))
    with pytest.raises(sb.SbwtError):
        idx.rank("A", n + 1)


def test_bad_input_leaves_index_unchanged():
    w = readgen.tiny()
    idx = gpu_bwt(w.reads, w.offsets, cuts=[0, 500])
    before = idx.bwt().copy()
    bad = w.reads[int(w.offsets[500]):].copy()
    bad[1234] = ord("N")
    with pytest.raises(sb.SbwtError) as e:
        idx.append(bad, w.offsets[500:] - w.offsets[500])
    assert e.value.code == sb.SBWT_EINVAL
    assert np.array_equal(idx.bwt(), before)
    assert idx.size() == (len(before), 500)
    idx.append(w.reads[int(w.offsets[500]):], w.offsets[500:] - w.offsets[500])
    assert np.array_equal(idx.bwt(), oracle.bwt(w.reads, w.offsets))


def test_budget_too_small_is_enomem_and_harmless():
    w = readgen.tiny()
    idx = sb.SetBWT(b"ACGT", hbm_budget=1 << 16)
    with pytest.raises(sb.SbwtError) as e:
        idx.append(w.reads, w.offsets)
    assert e.value.code == sb.SBWT_ENOMEM
    assert idx.size() == (0, 0)


def test_index_bits_64_matches_32():
    w = readgen.tiny()
    a = gpu_bwt(w.reads, w.offsets, cuts=w.appends, index_bits=32, capture=True)
    b = gpu_bwt(w.reads, w.offsets, cuts=w.appends, index_bits=64, capture=True)
    assert np.array_equal(a.bwt(), b.bwt())
    assert np.array_equal(sb.sbwt_get_stage(a.handle, sb.SBWT_STAGE_GSA), sb.sbwt_get_stage(b.handle, sb.SBWT_STAGE_GSA))


def test_device_append_matches_host_append():
    import torch
    w = readgen.tiny()
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(b"ACGT")
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    assert np.array_equal(idx.bwt(), oracle.bwt(w.reads, w.offsets))
    idx.reset()
    assert idx.size() == (0, 0)
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    assert np.array_equal(idx.bwt(), oracle.bwt(w.reads, w.offsets))


def test_repeated_appends_reuse_buffers():
    """Many small appends into one index equal the one-shot BWT."""
    w = readgen.tiny()
    cuts = list(range(0, 1001, 37)) + [1000]
    cuts = sorted(set(cuts))
    assert np.array_equal(gpu_bwt(w.reads, w.offsets, cuts=cuts).bwt(), oracle.bwt(w.reads, w.offsets))


def check_full_size(w, B, samples=3, seed=17):
    """Properties that pin B at any size: the symbol multiset, the terminator
    rows, rows of sampled suffixes counted one by one by the oracle, and LF
    inversion of the whole B back to every read."""
    n = oracle.num_suffixes(w.offsets)
    assert len(B) == n
    counts = np.bincount(B, minlength=256)
    expect_counts = np.bincount(w.reads, minlength=256)
    expect_counts[ord("$")] += w.m
    assert np.array_equal(counts, expect_counts)
    lens = np.diff(w.offsets.astype(np.int64))
    last = np.where(lens > 0, w.reads[np.maximum(w.offsets[1:].astype(np.int64) - 1, 0)], ord("$"))
    assert np.array_equal(B[: w.m], last.astype(np.uint8))
    rng = np.random.default_rng(seed)
    for _ in range(samples):
        r = int(rng.integers(0, w.m))
        p = int(rng.integers(0, int(lens[r]) + 1))
        row = oracle.row_of_suffix(w.reads, w.offsets, r, p)
        assert B[row] == oracle.bwt_symbol_of_suffix(w.reads, w.offsets, r, p)
    rec, roff = oracle.lf_invert_sampled(B, w.m, alphabet=w.alphabet)
    assert np.array_equal(roff, w.offsets) and np.array_equal(rec, w.reads)


def test_full_size_repetitive_reads():
    """Reads from a 2 kbp genome at ~15,000x coverage: the buckets and most
    groups overflow the CTA-local sorts, so the device-wide path (one
    cooperative radix sort per round) does the work at full size."""
    w = readgen.repetitive()
    idx = gpu_bwt(w.reads, w.offsets, M=w.block_suffixes, index_bits=w.index_bits)
    assert idx.size() == (oracle.num_suffixes(w.offsets), w.m)
    check_full_size(w, idx.bwt(), samples=2)


def test_graph_replay_serves_different_appends_into_a_growing_index():
    """The batched form: every append is one graph launch; the graph
    instantiated for a pipeline shape is updated in place for the later
    appends of that shape, which carry other reads (other host buffers) into
    a larger index."""
    w = readgen.tiny()
    cuts = [0, 150, 300, 450, 600, 750, 900, 1000]
    idx = sb.SetBWT(b"ACGT", block_suffixes=20_000)  # one block per append
    sb.sbwt_set_graph_replay(idx.handle, True)
    for a, b in zip(cuts[:-1], cuts[1:]):
        reads = w.reads[int(w.offsets[a]):int(w.offsets[b])].copy()  # a fresh host buffer each time
        idx.append(reads, w.offsets[a:b + 1] - w.offsets[a])
        assert np.array_equal(idx.bwt(), oracle.bwt(w.reads[: int(w.offsets[b])], w.offsets[: b + 1]))
    counts = {s["name"]: s["launches"] for s in sb.sbwt_get_kernel_stats(idx.handle)}
    assert counts["host:graph_launch"] == len(cuts) - 1
    assert counts["host:graph_instantiate"] == 1
    assert counts["host:graph_update"] == len(cuts) - 2


def test_graph_replay_matches_eager():
    """The batched form: repeated identical appends run as graph launches;
    every one gives the oracle's B."""
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    idx = sb.SetBWT(b"ACGT", block_suffixes=20_000)  # several blocks per append
    sb.sbwt_set_graph_replay(idx.handle, True)
    for _ in range(6):  # eager, eager, capture, capture, replay, replay
        idx.reset()
        idx.append(w.reads, w.offsets)
        assert np.array_equal(idx.bwt(), expect)
    # incremental appends under replay: same results as one shot
    for _ in range(3):
        idx.reset()
        idx.append(w.reads[: int(w.offsets[500])], w.offsets[:501])
        idx.append(w.reads[int(w.offsets[500]):], w.offsets[500:] - w.offsets[500])
        assert np.array_equal(idx.bwt(), expect)
    stats = {s["name"]: s["launches"] for s in sb.sbwt_get_kernel_stats(idx.handle)}
    assert stats.get("compute_ranks", 0) > 0 and stats.get("insert_merge", 0) > 0
    sb.sbwt_set_graph_replay(idx.handle, False)
    idx.reset()
    idx.append(w.reads, w.offsets)
    assert np.array_equal(idx.bwt(), expect)


def test_graph_replay_device_input_with_profiling():
    import torch
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(b"ACGT", block_suffixes=30_000)
    sb.sbwt_set_graph_replay(idx.handle, True)
    sb.sbwt_set_profiling(idx.handle, True)
    for _ in range(5):
        idx.reset()
        idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
        assert np.array_equal(idx.bwt(), expect)
    stats = {s["name"]: s for s in sb.sbwt_get_kernel_stats(idx.handle)}
    # every append ran the insert kernel of each of its 4 blocks, timed
    assert stats["insert_merge"]["launches"] == 5 * 4
    assert stats["insert_merge"]["ms"] > 0 and stats["insert_merge"]["bytes"] > 0


def test_autotune_block_suffixes():
    import torch
    w = readgen.tiny()
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(b"ACGT")
    best, times = sb.sbwt_autotune_block_suffixes(idx.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m,
                                                  [2048, 30_000, 1 << 20])
    assert best in (2048, 30_000, 1 << 20) and times[best] == min(t for t in times.values() if t >= 0)
    assert idx.size() == (0, 0)
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    assert np.array_equal(idx.bwt(), oracle.bwt(w.reads, w.offsets))
    with pytest.raises(sb.SbwtError):
        sb.sbwt_autotune_block_suffixes(idx.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m, [0])


@pytest.mark.parametrize("sampling", [64, 128, 256])
def test_host_tier_forced(sampling):
    """The dictionary in mapped pinned host memory, rewritten in place by
    every block's Insert: same B, same ranks; a byte outside the alphabet is
    refused before the rewrite, leaving the index as it was."""
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    idx = gpu_bwt(w.reads, w.offsets, M=20_000, cuts=w.appends)
    ref_ranks = idx.rank_batch(np.full(50, ord("C"), np.uint8), np.arange(0, 101_000, 2020, dtype=np.uint64))
    h = sb.SetBWT(b"ACGT", block_suffixes=20_000, host_tier=3, occ_sampling=sampling)
    bad = w.reads[: int(w.offsets[300])].copy()
    bad[777] = ord("N")
    with pytest.raises(sb.SbwtError) as e:
        h.append(bad, w.offsets[:301])
    assert e.value.code == sb.SBWT_EINVAL and h.size() == (0, 0)
    h.append(w.reads[: int(w.offsets[500])], w.offsets[:501])
    h.append(w.reads[int(w.offsets[500]):], w.offsets[500:] - w.offsets[500])
    assert np.array_equal(h.bwt(), expect)
    hbm, host = sb.sbwt_memory(h.handle)
    assert host > 0
    assert np.array_equal(h.rank_batch(np.full(50, ord("C"), np.uint8), np.arange(0, 101_000, 2020, dtype=np.uint64)),
                          ref_ranks)
    before = h.bwt().copy()
    with pytest.raises(sb.SbwtError) as e:
        h.append(bad, w.offsets[:301])
    assert e.value.code == sb.SBWT_EINVAL
    assert np.array_equal(h.bwt(), before)
    n, _ = h.size()
    assert 8.0 * sb.sbwt_memory(h.handle)[1] / n <= 6.0


def test_bandwidth_probe():
    idx = sb.SetBWT(b"ACGT")  # kept alive for the call
    bw = sb.sbwt_measure_bandwidth(idx.handle)
    idx.close()
    assert bw["h2d_GBps"] > 1 and bw["d2h_GBps"] > 1
    assert 0.1 < bw["host_random_32B_GBps"] < bw["hbm_random_32B_GBps"]


def test_host_tier_under_budget():
    """A budget between what the index needs with its dictionaries in HBM
    and what it needs in the host tier moves them to the host tier instead
    of failing; B is unchanged.  With the host tier forbidden the same
    budget is SBWT_ENOMEM."""
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    probe = sb.SetBWT(b"ACGT", host_tier=3)
    probe.append(w.reads, w.offsets)
    hbm_tiered, host_tiered = sb.sbwt_memory(probe.handle)
    full = sb.SetBWT(b"ACGT")
    full.append(w.reads, w.offsets)
    hbm_full, host_full = sb.sbwt_memory(full.handle)
    assert host_tiered > 0 and host_full == 0 and hbm_tiered < hbm_full
    budget = (hbm_tiered + hbm_full) // 2
    idx = sb.SetBWT(b"ACGT", hbm_budget=budget)
    idx.append(w.reads, w.offsets)
    assert np.array_equal(idx.bwt(), expect)
    hbm, host = sb.sbwt_memory(idx.handle)
    assert hbm <= budget and host > 0
    forbidden = sb.SetBWT(b"ACGT", hbm_budget=budget, host_tier=2)
    with pytest.raises(sb.SbwtError) as e:
        forbidden.append(w.reads, w.offsets)
    assert e.value.code == sb.SBWT_ENOMEM


def test_count_queries_match_oracle():
    w = readgen.tiny()
    idx = gpu_bwt(w.reads, w.offsets, M=20_000, cuts=w.appends)
    rng = np.random.default_rng(21)
    pats = [b"", b"A", b"ACGT", b"TTTT", b"N", b"ACN"]
    for L in (1, 2, 3, 5, 8, 12, 20, 100, 101):
        for _ in range(6):
            r = int(rng.integers(0, w.m))
            p0 = int(rng.integers(0, max(1, 101 - L)))
            pats.append(bytes(w.reads[int(w.offsets[r]) + p0:int(w.offsets[r]) + p0 + L]))  # present
            pats.append(bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=L)))        # random
    got = idx.count(pats)
    expect = [oracle.count(w.reads, w.offsets, p) if all(c in b"ACGT" for c in p) else 0 for p in pats]
    assert list(got) == expect
    assert got[0] == oracle.num_suffixes(w.offsets)


@pytest.mark.parametrize("M", [0, 7_000])
def test_prepend_places_reads_first(M):
    """sbwt_prepend: the reads go before the index's reads (Section 2's
    reverse order); every mix of appends and prepends equals one append of
    the reads in their final order (checked by the oracle).  M = 7000 makes
    the prepended sets span several blocks, run last to first."""
    a = readgen.ragged_reads(300, 0, 90, seed=81, p_empty=0.03)
    b = readgen.ragged_reads(250, 1, 120, seed=82, p_repeat=0.05)
    c = readgen.uniform_reads(200, 60, seed=83)
    d = readgen.ragged_reads(150, 0, 40, seed=84)
    idx = sb.SetBWT(b"ACGT", block_suffixes=M)
    idx.append(*b)
    idx.prepend(*a)   # a b
    idx.append(*c)    # a b c
    idx.prepend(*d)   # d a b c
    parts = [d, a, b, c]
    reads = np.concatenate([r for r, _ in parts])
    lens = np.concatenate([np.diff(o.astype(np.int64)) for _, o in parts])
    offsets = readgen.offsets_from_lengths(lens)
    assert idx.size() == (oracle.num_suffixes(offsets), len(offsets) - 1)
    assert np.array_equal(idx.bwt(), oracle.bwt(reads, offsets))
    # into an empty index, a prepend is an append
    e = sb.SetBWT(b"ACGT", block_suffixes=M).prepend(*a)
    assert np.array_equal(e.bwt(), oracle.bwt(*a))


@pytest.mark.parametrize("sampling", [64, 128, 256])
def test_occurrence_sampling(sampling):
    """Every occurrence sampling gives the oracle's B, ranks and counts: the
    tiny workload in two appends and in many small blocks, a ragged set over
    superblock-straddling sizes with empty reads and repeats, and rank
    queries at the block and superblock edges."""
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    for M, cuts in ((w.block_suffixes, w.appends), (777, [0, 100, 640, 1000])):
        idx = gpu_bwt(w.reads, w.offsets, M=M, cuts=cuts, occ_sampling=sampling)
        assert np.array_equal(idx.bwt(), expect)
    reads, off = readgen.ragged_reads(1300, 0, 200, seed=sampling, p_empty=0.03, p_repeat=0.05)
    B = oracle.bwt(reads, off)
    idx = gpu_bwt(reads, off, M=40_000, cuts=[0, 300, 1300], occ_sampling=sampling, index_bits=64)
    assert np.array_equal(idx.bwt(), B)
    n = len(B)
    ks = np.unique(np.concatenate([[0, 1, 63, 64, 65, 127, 128, 129, 255, 256, 257, 65535, 65536, 65537, n - 1, n],
                                   np.random.default_rng(1).integers(0, n + 1, size=300)]))
    ks = ks[ks <= n]
    for c in b"$ACGT":
        cum = np.concatenate([[0], np.cumsum(B == c)])
        assert np.array_equal(idx.rank_batch(np.full(len(ks), c, np.uint8), ks.astype(np.uint64)), cum[ks])
    pats = [b"A", b"CG", b"TTA", b"ACGTA", b"GGGG"]
    assert list(idx.count(pats)) == [oracle.count(reads, off, p) for p in pats]


def test_autotune_picks_block_size_and_sampling():
    """The joint autotuner times every (sampling, M) pair on the given reads,
    keeps the fastest in the index, and the index it leaves builds the
    oracle's B."""
    import torch
    w = readgen.tiny()
    d_reads = torch.from_numpy(w.reads).cuda()
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    idx = sb.SetBWT(b"ACGT")
    best_m, best_s, times = sb.sbwt_autotune(idx.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m,
                                             [20_000, 1 << 20], [64, 128, 256])
    assert best_m in (20_000, 1 << 20) and best_s in (64, 128, 256)
    assert len(times) == 6 and all(t > 0 for t in times.values())
    assert times[(best_s, best_m)] == min(times.values())
    assert idx.size() == (0, 0)
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
    assert np.array_equal(idx.bwt(), oracle.bwt(w.reads, w.offsets))


def test_block_overlap_off_gives_the_same_b():
    """The plain per-block loop (every step of every block in turn on one
    stream) and the overlapped pipeline give the oracle's B."""
    w = readgen.tiny()
    expect = oracle.bwt(w.reads, w.offsets)
    for overlap in (False, True, False):
        idx = sb.SetBWT(b"ACGT", block_suffixes=9_000)
        sb.sbwt_set_block_overlap(idx.handle, overlap)
        idx.append(w.reads, w.offsets)
        assert np.array_equal(idx.bwt(), expect)


def test_tile_shapes_give_the_same_b():
    """Every Insert CTA size and ComputeRanks segment length gives the
    oracle's B (long reads take the segmented kernel), and the shape
    autotuner keeps one of its candidates."""
    import torch
    rng = np.random.default_rng(41)
    g_ = readgen.genome(200_000, seed=41)
    lens = rng.integers(300, 4000, size=120)
    reads, off = readgen.sampled_reads(g_, 120, lens, 0.05, seed=42)
    expect = oracle.bwt(reads, off)
    for shape in ((0, 256), (256, 256), (512, 256), (0, 512), (512, 1024)):
        idx = sb.SetBWT(b"ACGT", block_suffixes=60_000)
        sb.sbwt_set_tile_shapes(idx.handle, *shape)
        assert sb.sbwt_get_tile_shapes(idx.handle) == shape
        idx.append(reads[: int(off[40])], off[:41])
        idx.append(reads[int(off[40]):], off[40:] - off[40])
        assert np.array_equal(idx.bwt(), expect), shape
    with pytest.raises(sb.SbwtError):
        sb.sbwt_set_tile_shapes(idx.handle, 384, 256)
    d_reads = torch.from_numpy(reads).cuda()
    d_off = torch.from_numpy(off.astype(np.int64)).cuda()
    best, times = sb.sbwt_autotune_tile_shapes(idx.handle, d_reads.data_ptr(), d_off.data_ptr(), len(off) - 1)
    assert best in times and times[best] == min(times.values())
