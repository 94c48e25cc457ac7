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
