"""The seeded input generators (readgen) produce the shapes the workloads
state: lengths, alphabets, determinism, reads drawn from their genome with
the stated substitution rate.  No GPU needed."""
import numpy as np

import readgen


def test_short_reads_are_genome_windows_with_substitutions():
    g = readgen.genome(200_000, 7)
    reads, off = readgen.sampled_reads(g, 2_000, 100, 0.01, 8)
    assert len(off) == 2_001 and int(off[-1]) == 200_000
    assert set(np.unique(reads).tolist()) <= set(b"ACGT")
    again, off2 = readgen.sampled_reads(g, 2_000, 100, 0.01, 8)
    assert np.array_equal(reads, again) and np.array_equal(off, off2)
    # every read matches a window of the genome or its reverse complement at
    # ~99% of its positions
    lut = np.zeros(256, np.uint8)
    lut[list(b"ACGT")] = [0, 1, 2, 3]
    codes = lut[reads].reshape(2_000, 100)
    gs = g.tobytes()
    for r in codes[:20]:
        fwd, rev = r.tobytes(), (3 - r[::-1]).astype(np.uint8).tobytes()
        best = 0
        for s in range(len(g) - 100 + 1):
            w = gs[s:s + 100]
            best = max(best, sum(a == b for a, b in zip(w, fwd)), sum(a == b for a, b in zip(w, rev)))
            if best >= 95:
                break
        assert best >= 95


def test_wide_workload_shape():
    w = readgen.wide(n_reads=5_000, genome_size=50_000)
    assert w.alphabet == b"ACGNT" and w.m == 5_000 and w.bases == 500_000
    assert set(np.unique(w.reads).tolist()) <= set(b"ACGNT")
    share_n = float(np.mean(w.reads == ord("N")))
    assert 0.02 < share_n < 0.07  # 4% N in the genome, plus substitutions
    w2 = readgen.wide(n_reads=5_000, genome_size=50_000)
    assert np.array_equal(w.reads, w2.reads)


def test_tiny_and_repetitive_shapes():
    t = readgen.tiny()
    assert t.m == 1_000 and t.bases == 100_000 and t.appends == (0, 500, 1_000)
    r = readgen.repetitive(n_reads=2_000, genome_size=300)
    assert r.m == 2_000 and r.bases == 200_000 and r.index_bits == 64


def _window_match(g, seq):
    """True when seq is a window of g or of its reverse complement."""
    gs, L = g.tobytes(), len(seq)
    lut = np.zeros(256, np.uint8)
    lut[list(b"ACGT")] = [0, 1, 2, 3]
    codes = lut[seq]
    rev = (3 - codes[::-1]).astype(np.uint8).tobytes()
    return gs.find(codes.tobytes()) >= 0 or gs.find(rev) >= 0 if L else True


def test_long_reads_lengths_and_error_model():
    g = readgen.genome(400_000, 11)
    reads, off = readgen.long_reads(g, 400, 10_000.0, 0.5, (1_000, 50_000), 0.0, 0.0, 0.0, 12)
    lengths = np.diff(off)
    assert lengths.min() >= 1_000 and lengths.max() <= 50_000
    assert 9_000 < lengths.mean() < 11_000  # log-normal with mean 10 kbp, sigma 0.5
    # without errors every read is a window of the genome or its reverse complement
    for j in range(0, 400, 40):
        assert _window_match(g, reads[off[j]:off[j + 1]])
    # substitutions only: the same windows, ~p_sub of the positions changed
    sub, off2 = readgen.long_reads(g, 40, 10_000.0, 0.5, (1_000, 50_000), 0.0, 0.0, 0.06, 12)
    assert np.array_equal(off2, off[:41])
    assert set(np.unique(sub).tolist()) <= set(b"ACGT")
    clean, _ = readgen.long_reads(g, 40, 10_000.0, 0.5, (1_000, 50_000), 0.0, 0.0, 0.0, 12)
    assert 0.05 < float(np.mean(sub != clean)) < 0.07  # same draws, 6% of positions substituted
    # indels change the emitted sequence but keep the drawn lengths
    ind, off3 = readgen.long_reads(g, 40, 10_000.0, 0.5, (1_000, 50_000), 0.02, 0.02, 0.06, 12)
    assert np.array_equal(off3, off[:41]) and not np.array_equal(ind, sub)


def test_batched_and_serving_shapes():
    b = readgen.batched(n_reads=20_000, genome_size=1_000_000)
    lengths = np.diff(b.offsets)
    assert lengths.min() >= 50 and lengths.max() <= 250 and 140 < lengths.mean() < 160
    assert b.index_bits == 64 and b.block_suffixes == 0  # block size is autotuned
    resident, requests = readgen.serving(n_resident=5_000, genome_size=200_000, n_requests=6,
                                         max_request=40_000)
    assert resident.m == 5_000 and resident.bases == 500_000 and resident.index_bits == 64
    assert len(requests) == 6
    for reads, off in requests:
        m = len(off) - 1
        assert 10_000 <= m <= 40_000
        ln = np.diff(off)
        assert ln.min() >= 100 and ln.max() <= 150 and int(off[-1]) == len(reads)
