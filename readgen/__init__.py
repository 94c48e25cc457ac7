"""Seeded synthetic read sets shaped like the workloads of arXiv 1410.0562.

This module holds no part of the BWT method: it only draws reads.  Both the
oracle (in the tests and the CPU baseline) and the GPU library consume what it
returns, and neither is imported here.

The paper measures on two real sequencing sets that are not available here
(NA12878, 1.2 G x 101 bp Illumina reads; Venter, 32 M x 875 bp Sanger reads;
Section 7).  The generators below stand in for them with the same shapes:
short reads at ~10x coverage of a genome, ragged mid-length reads, long
reads with indels, and request streams for the served form.  All randomness
comes from numpy's PCG64 generator seeded with each workload function's
default seeds; the same seed gives the same reads on any machine with the
same numpy version.

A read set is returned as ``(reads, offsets)``: ``reads`` is a uint8 array of
ASCII bases (the concatenation of all reads) and ``offsets`` a uint64 array of
``m + 1`` non-decreasing entries, read ``j`` being
``reads[offsets[j]:offsets[j+1]]``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DNA = b"ACGT"
_LUT = np.frombuffer(DNA, dtype=np.uint8)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def offsets_from_lengths(lengths) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.uint64)
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    return off


def genome(size: int, seed: int) -> np.ndarray:
    """An i.i.d. uniform genome over {0,1,2,3} (codes of A,C,G,T)."""
    return _rng(seed).integers(0, 4, size=size, dtype=np.uint8)


def uniform_reads(n_reads: int, length: int, seed: int, alphabet: bytes = DNA):
    """n_reads reads of equal length, every base i.i.d. uniform over the alphabet."""
    rng = _rng(seed)
    lut = np.frombuffer(alphabet, dtype=np.uint8)
    codes = rng.integers(0, len(lut), size=n_reads * length, dtype=np.uint8)
    return lut[codes], offsets_from_lengths(np.full(n_reads, length))


def ragged_reads(n_reads: int, min_len: int, max_len: int, seed: int, alphabet: bytes = DNA,
                 p_empty: float = 0.0, p_repeat: float = 0.0):
    """Reads of uniform random length in [min_len, max_len], i.i.d. bases.

    ``p_empty`` makes that fraction of reads empty; ``p_repeat`` makes that
    fraction of reads a single repeated base (long common prefixes).
    """
    rng = _rng(seed)
    lut = np.frombuffer(alphabet, dtype=np.uint8)
    lengths = rng.integers(min_len, max_len + 1, size=n_reads)
    if p_empty > 0:
        lengths[rng.random(n_reads) < p_empty] = 0
    off = offsets_from_lengths(lengths)
    codes = rng.integers(0, len(lut), size=int(off[-1]), dtype=np.uint8)
    if p_repeat > 0:
        rep = np.nonzero(rng.random(n_reads) < p_repeat)[0]
        for j in rep:
            codes[off[j]:off[j + 1]] = codes[off[j]] if off[j + 1] > off[j] else 0
    return lut[codes], off


def _revcomp(codes: np.ndarray) -> np.ndarray:
    return (3 - codes)[..., ::-1]


def sampled_reads(g: np.ndarray, n_reads: int, lengths, sub_rate: float, seed: int):
    """Reads sampled from genome g at uniform offsets and strands, with
    uniform substitutions (the new base is one of the other three).

    ``lengths`` is an int (all reads that long) or an array of n_reads lengths.
    """
    rng = _rng(seed)
    G = len(g)
    if np.isscalar(lengths):
        lengths = np.full(n_reads, int(lengths), dtype=np.int64)
    lengths = np.asarray(lengths, dtype=np.int64)
    off = offsets_from_lengths(lengths)
    out = np.empty(int(off[-1]), dtype=np.uint8)
    starts = rng.integers(0, G - lengths + 1)
    minus = rng.random(n_reads) < 0.5
    # group by length so each group is one vectorised gather, in chunks of
    # reads to bound the temporary arrays
    chunk = 1 << 19
    for L in np.unique(lengths):
        if L == 0:
            continue
        all_idx = np.nonzero(lengths == L)[0]
        for c0 in range(0, len(all_idx), chunk):
            idx = all_idx[c0:c0 + chunk]
            win = np.lib.stride_tricks.sliding_window_view(g, int(L))[starts[idx]].copy()
            mi = minus[idx]
            win[mi] = _revcomp(win[mi])
            sub = rng.random(win.shape) < sub_rate
            shift = rng.integers(1, 4, size=win.shape, dtype=np.uint8)
            win = np.where(sub, (win + shift) & 3, win).astype(np.uint8)
            pos = off[idx][:, None].astype(np.int64) + np.arange(int(L))[None, :]
            out[pos.ravel()] = win.ravel()
    return _LUT[out], off


def long_reads(g: np.ndarray, n_reads: int, mean_len: float, sigma: float, clip: tuple, p_del: float,
               p_ins: float, p_sub: float, seed: int):
    """Long reads with indels: log-normal lengths with the given mean and
    sigma, clipped to ``clip``; each emitted step is a deletion (skip a genome
    base) with probability p_del, an insertion (emit a random base) with
    p_ins, a substitution with p_sub, else a copy; a read stops after its
    drawn number of emitted bases.  Strands are 50/50.
    """
    rng = _rng(seed)
    mu = np.log(mean_len) - sigma * sigma / 2
    lengths = np.clip(np.round(rng.lognormal(mu, sigma, size=n_reads)), clip[0], clip[1]).astype(np.int64)
    off = offsets_from_lengths(lengths)
    out = np.empty(int(off[-1]), dtype=np.uint8)
    G = len(g)
    for j in range(n_reads):
        L = int(lengths[j])
        steps = int(L * 1.25) + 64
        u = rng.random(steps)
        rand_base = rng.integers(0, 4, size=steps, dtype=np.uint8)
        shift = rng.integers(1, 4, size=steps, dtype=np.uint8)
        is_del = u < p_del
        is_ins = (u >= p_del) & (u < p_del + p_ins)
        is_sub = (u >= p_del + p_ins) & (u < p_del + p_ins + p_sub)
        emit = ~is_del
        consume = ~is_ins  # copies, substitutions and deletions advance the genome
        gpos = np.cumsum(consume) - consume  # genome offset consumed before each step
        span = int(gpos[-1]) + 2
        start = int(rng.integers(0, max(G - span, 1)))
        src = g[(start + np.minimum(gpos, G - 1 - start))]
        base = np.where(is_ins, rand_base, np.where(is_sub, (src + shift) & 3, src)).astype(np.uint8)
        seq = base[emit][:L]
        if len(seq) < L:  # never expected with the 25% slack, but stay exact
            seq = np.concatenate([seq, rng.integers(0, 4, size=L - len(seq), dtype=np.uint8)])
        if rng.random() < 0.5:
            seq = _revcomp(seq)
        out[off[j]:off[j + 1]] = seq
    return _LUT[out], off


@dataclass(frozen=True)
class Workload:
    name: str
    reads: np.ndarray
    offsets: np.ndarray
    block_suffixes: int
    index_bits: int
    appends: tuple  # read-count boundaries of the sbwt_append calls
    alphabet: bytes = DNA

    @property
    def m(self) -> int:
        return len(self.offsets) - 1

    @property
    def bases(self) -> int:
        return int(self.offsets[-1])


def tiny(seed: int = 0x05621410 + 1) -> Workload:
    """1,000 reads x 100 bp, i.i.d. uniform bases, appended as 2 x 500 reads."""
    reads, off = uniform_reads(1000, 100, seed)
    return Workload("tiny-1000x100-iid", reads, off, 1 << 24, 32, (0, 500, 1000))


def short(n_reads: int = 1_000_000, genome_size: int = 10_000_000, seed_genome: int = 0x14100562 + 2,
          seed_reads: int = 0x05621410 + 2) -> Workload:
    """1M x 100 bp reads from a 10 Mbp i.i.d. genome, uniform offsets and
    strands, 1% substitutions; blocks of 16,777,216 suffixes; 32-bit indices."""
    g = genome(genome_size, seed_genome)
    reads, off = sampled_reads(g, n_reads, 100, 0.01, seed_reads)
    return Workload(f"short-{n_reads}x100-g{genome_size}", reads, off, 1 << 24, 32, (0, n_reads))


def batched(n_reads: int = 2_000_000, genome_size: int = 50_000_000, seed_genome: int = 0x14100562 + 3,
            seed_reads: int = 0x05621410 + 3) -> Workload:
    """2M reads of length uniform in [50, 250] from a 50 Mbp i.i.d. genome, 1% substitutions; 64-bit indices."""
    g = genome(genome_size, seed_genome)
    lengths = _rng(seed_reads ^ 0x5A5A).integers(50, 251, size=n_reads)
    reads, off = sampled_reads(g, n_reads, lengths, 0.01, seed_reads)
    return Workload(f"batched-{n_reads}xU[50,250]-g{genome_size}", reads, off, 0, 64, (0, n_reads))


def long(n_reads: int = 20_000, genome_size: int = 100_000_000, seed_genome: int = 0x14100562 + 4,
         seed_reads: int = 0x05621410 + 4) -> Workload:
    """20k log-normal reads (mean 10 kbp, sigma 0.5, clipped to [1k, 50k]) with
    6% substitutions, 2% insertions, 2% deletions; 64-bit indices."""
    g = genome(genome_size, seed_genome)
    reads, off = long_reads(g, n_reads, 10_000.0, 0.5, (1_000, 50_000), 0.02, 0.02, 0.06, seed_reads)
    return Workload(f"long-{n_reads}xlognormal10k-g{genome_size}", reads, off, 0, 64, (0, n_reads))


def repetitive(n_reads: int = 300_000, genome_size: int = 2_000, seed_genome: int = 0x14100562 + 6,
               seed_reads: int = 0x05621410 + 6) -> Workload:
    """300k x 100 bp reads from a 2 kbp i.i.d. genome (~15,000x coverage),
    1% substitutions: every bucket of a few leading symbols and most groups
    of equal 29-symbol prefixes hold thousands of suffixes.  One block of
    2^25 suffixes; 64-bit indices."""
    g = genome(genome_size, seed_genome)
    reads, off = sampled_reads(g, n_reads, 100, 0.01, seed_reads)
    return Workload(f"repetitive-{n_reads}x100-g{genome_size}", reads, off, 1 << 25, 64, (0, n_reads))


def genome_alpha(size: int, seed: int, probs) -> np.ndarray:
    """An i.i.d. genome of codes 0..len(probs)-1 drawn with the given probabilities."""
    return _rng(seed).choice(len(probs), size=size, p=np.asarray(probs, dtype=np.float64)).astype(np.uint8)


def sampled_reads_alpha(g: np.ndarray, n_reads: int, length: int, sub_rate: float, seed: int, alphabet: bytes):
    """Reads of one length sampled from genome g (codes into ``alphabet``) at
    uniform offsets, forward strand, with uniform substitutions (the new
    symbol is one of the other len(alphabet) - 1)."""
    rng = _rng(seed)
    sigma = len(alphabet)
    starts = rng.integers(0, len(g) - length + 1, size=n_reads)
    out = np.empty((n_reads, length), dtype=np.uint8)
    chunk = 1 << 18
    for c0 in range(0, n_reads, chunk):
        s = starts[c0:c0 + chunk]
        win = np.lib.stride_tricks.sliding_window_view(g, length)[s]
        sub = rng.random(win.shape) < sub_rate
        shift = rng.integers(1, sigma, size=win.shape, dtype=np.uint8)
        out[c0:c0 + chunk] = np.where(sub, (win + shift) % sigma, win)
    lut = np.frombuffer(alphabet, dtype=np.uint8)
    return lut[out.ravel()], offsets_from_lengths(np.full(n_reads, length))


def wide(n_reads: int = 1_000_000, genome_size: int = 10_000_000, seed_genome: int = 0x14100562 + 7,
         seed_reads: int = 0x05621410 + 7) -> Workload:
    """The short-read shape over a five-symbol alphabet (A, C, G, N, T; N at
    4%): 1M x 100 bp reads from a 10 Mbp i.i.d. genome, forward strand, 1%
    substitutions; blocks of 16,777,216 suffixes; 32-bit indices.  Exercises
    the 4-bit-code path."""
    alphabet = b"ACGNT"
    g = genome_alpha(genome_size, seed_genome, [0.24, 0.24, 0.24, 0.04, 0.24])
    reads, off = sampled_reads_alpha(g, n_reads, 100, 0.01, seed_reads, alphabet)
    return Workload(f"wide-ACGNT-{n_reads}x100-g{genome_size}", reads, off, 1 << 24, 32, (0, n_reads), alphabet)


def serving(n_resident: int = 20_000_000, genome_size: int = 200_000_000, n_requests: int = 48,
            seed_genome: int = 0x14100562 + 5, seed_reads: int = 0x05621410 + 5, max_request: int = 1_000_000,
            min_request: int = 10_000):
    """The serving workload: a resident set of n_resident x 100 bp reads (1%
    substitutions) from a seeded i.i.d. genome, and request read sets whose
    sizes are log-uniform in [min_request, max_request] reads (10k to 1M by
    default) of length U[100, 150] from the same genome.  Returns (resident
    Workload, list of (reads, offsets))."""
    g = genome(genome_size, seed_genome)
    reads, off = sampled_reads(g, n_resident, 100, 0.01, seed_reads)
    resident = Workload(f"serving-resident-{n_resident}x100-g{genome_size}", reads, off, 1 << 25, 64,
                        (0, n_resident))
    rng = _rng(seed_reads ^ 0xA5A5)
    sizes = np.exp(rng.uniform(np.log(min_request), np.log(max_request), size=n_requests)).astype(np.int64)
    requests = []
    for i, m in enumerate(sizes):
        lengths = rng.integers(100, 151, size=int(m))
        requests.append(sampled_reads(g, int(m), lengths, 0.01, seed_reads + 1 + i))
    return resident, requests


def serving_scaled(scale: int = 20):
    """The serving workload at 1/scale of its size in every dimension: the
    resident reads, the genome and the request sizes (so 1M resident reads
    from a 10 Mbp genome and requests of 500 to 50k reads at scale 20), with
    the same seeds, read lengths and request count."""
    return serving(n_resident=20_000_000 // scale, genome_size=200_000_000 // scale, n_requests=48,
                   max_request=1_000_000 // scale, min_request=10_000 // scale)
