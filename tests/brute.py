"""Brute-force BWT of a tiny string set by sorting rotations (pure Python).

This pins the oracle against something other than itself.  T is built as a
list of integers: terminator $_r becomes r and a symbol becomes m + its byte
value, so ``$_0 < ... < $_{m-1} < c_1`` holds (Section 2).  Because the
terminators are distinct, two rotations always differ by their first
terminator at the latest, so the order of the n rotations of T equals the
order of its suffixes and the last column of the sorted rotations is
``B[i] = T[(SA[i]-1) mod n]`` (Eq. 1).  Costs O(n^2 log n): tiny inputs only.
"""
from __future__ import annotations


def build_text(reads):
    """reads: list of bytes.  Returns (T as ints, list of (read, offset) per position)."""
    m = len(reads)
    T, where = [], []
    for r, s in enumerate(reads):
        for p, ch in enumerate(s):
            T.append(m + ch)
            where.append((r, p))
        T.append(r)
        where.append((r, len(s)))
    return T, where


def sorted_rotations(reads):
    """Positions of T in rotation (= suffix) order."""
    T, _ = build_text(reads)
    n = len(T)
    return sorted(range(n), key=lambda i: T[i:] + T[:i])


def bwt(reads) -> bytes:
    T, _ = build_text(reads)
    m = len(reads)
    n = len(T)
    out = bytearray()
    for i in sorted_rotations(reads):
        x = T[(i - 1) % n]
        out.append(ord("$") if x < m else x - m)
    return bytes(out)


def suffix_rows(reads):
    """dict (read, offset) -> row in the sorted order."""
    _, where = build_text(reads)
    return {where[i]: row for row, i in enumerate(sorted_rotations(reads))}


def g_values(old_reads, block_reads):
    """For each block suffix in block text order: how many suffixes of
    old_reads are smaller, read off the brute-force order of the union."""
    allr = list(old_reads) + list(block_reads)
    m_old = len(old_reads)
    _, where = build_text(allr)
    order = sorted_rotations(allr)
    g = {}
    old_seen = 0
    for i in order:
        r, p = where[i]
        if r < m_old:
            old_seen += 1
        else:
            g[(r - m_old, p)] = old_seen
    out = []
    for j, s in enumerate(block_reads):
        for p in range(len(s) + 1):
            out.append(g[(j, p)])
    return out


def to_set(reads_u8, offsets):
    return [bytes(reads_u8[int(offsets[j]):int(offsets[j + 1])]) for j in range(len(offsets) - 1)]
