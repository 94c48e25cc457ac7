/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for set-bwte
 * (Pantaleoni, "A massively parallel algorithm for constructing the BWT of
 * large string sets", arXiv 1410.0562).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - oracle_bwt: the BWT of a string set, straight from its definition
 *     (Section 2, Eq. 1): T = S_0 $_0 ... S_{m-1} $_{m-1} with
 *     $_0 < ... < $_{m-1} < c_1, suffixes sorted by direct comparison,
 *     B[i] = T[(SA[i]-1) mod n].  Every $_k is written as the byte '$'.
 *   - oracle_rank: rank(c,k,B) = |{i<k : B[i]=c}| (Section 2, Eq. 2),
 *     by counting.
 *   - oracle_block_sa / oracle_block_bint: SA_int and B_int of one block
 *     (Algorithm 1, ConstructSA and B(S_jk, SA_int)), by direct comparison.
 *   - oracle_block_g_direct: g[t] = number of suffixes of the previously
 *     added reads that are smaller than block suffix t (the quantity that
 *     Lemma 1 of Section 4 propagates), by binary search among the sorted
 *     old suffixes.
 *   - oracle_block_g_lemma1: the same g by Algorithm 2 (ComputeRanks),
 *     stepping Lemma 1 backwards from each terminator, with the start value
 *     i := m_ext (the reading of Algorithm 2's initial rank that agrees with
 *     the terminator order of Section 2).
 *   - oracle_insert: Insert of Algorithm 1 / Section 5 as a stable merge:
 *     new symbol i lands on row g_sa[i] + i, old rows keep their order.
 *   - oracle_setbwte: Algorithm 1 end to end, block by block, built from the
 *     four functions above; oracle_setbwte_reverse: the same loop over the
 *     blocks from the last to the first (Section 2 allows the reversal),
 *     each block going before the reads already inserted.
 *   - oracle_lf_invert / oracle_lf_invert_sampled: recover every read from B
 *     by LF steps (the FM-index inversion that Lemma 1 rests on), with a full
 *     prefix-count table or with counts every 64 rows.
 *   - oracle_count: occurrences of a pattern in the reads, by direct
 *     comparison (what FM-index backward search counts).
 *   - oracle_row_of_suffix: row of one suffix in the full sorted order, by
 *     counting the smaller suffixes one comparison at a time (for sampled
 *     checks at sizes where sorting everything is too slow).
 *
 * Readings taken where the paper is silent or garbled:
 *   - Algorithm 2 starts each read at i := m_ext, not n_ext: a new
 *     terminator is larger than exactly the m_ext old terminator suffixes
 *     and smaller than every suffix that starts with a symbol (Section 2).
 *   - Algorithm 2's text index offset + j + k, with offsets the prefix sum
 *     of |P_j|+1, counts j twice; the block-local position of P_j[k] is
 *     (exclusive prefix sum of |P_l|+1 over l<j) + k, and the terminator of
 *     P_j sits at k = |P_j|.
 *   - C[c] counts every symbol of B_ext smaller than c, the m_ext
 *     terminators included, so C[c_1] = m_ext.
 *   - Insert ties: new symbols with equal g_sa keep their SA_int order and
 *     go before old row g_sa; the final row of new symbol i is g_sa[i]+i.
 *   - Symbols are ordered by byte value (the alphabet, 1 to 16 bytes, is
 *     given in strictly increasing byte order); a byte outside the alphabet
 *     is an error.
 *   - Reverse order: a block added before every read already in B_ext has
 *     terminators smaller than every old one, so Algorithm 2 starts each of
 *     its reads at i := 0.
 *
 * Layout conventions (plain, nothing packed):
 *   reads   : the bytes of all reads, concatenated; read r is
 *             reads[offsets[r] .. offsets[r+1]).
 *   offsets : m+1 non-decreasing uint64 values, offsets[0] = 0.
 *   B       : one byte per row: an alphabet byte, or '$' for a terminator.
 *   block-local text position of read j's symbol k (block = reads
 *   [j0, j1)): start_j + k with start_j = sum over j0<=l<j of (|P_l|+1);
 *   the terminator of read j is at start_j + |P_j|.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ORACLE_PLANT selects one deliberate mistake, for the tests that show the
 * pins catch it; the shipped build leaves it at 0.
 *   1: Algorithm 2 starts at i := n_ext      2: terminator ties reversed
 *   3: a shorter suffix sorts after a longer one with the same prefix
 *   4: Insert puts new symbols after the old row g_sa (tie order flipped)
 *   5: C[c] leaves out the terminators
 *   6: the reverse order starts Algorithm 2 at i := m_ext, not 0
 *   7: counting skips overlapping occurrences
 *   8: the sampled inversion takes each checkpoint after its own row
 *   9: the row of a suffix counts the suffix itself
 *  10: rank(c, k) counts rows 0..k instead of 0..k-1
 *  11: Lemma 1's C[] only covers the first four symbols
 *  12: the direct g leaves out the last old read
 *  13: B_int holds '$' for a read's terminator suffix
 *  14: the full LF inversion's C[] leaves out the terminators             */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2

typedef struct {
    uint64_t r; /* global read id */
    uint64_t p; /* offset inside the read; p == |S_r| is the terminator */
} suffix_t;

/* One comparison context: qsort has no user pointer in ISO C, and the
 * oracle is single-threaded by design. */
static const uint8_t *g_reads;
static const uint64_t *g_offsets;

static uint64_t read_len(uint64_t r) { return g_offsets[r + 1] - g_offsets[r]; }

/* Direct comparison of suffixes (r,p) and (r',p') of T (Section 2): compare
 * symbol by symbol; the suffix that reaches its terminator first is smaller
 * (a terminator is smaller than every symbol); if both reach their
 * terminators at the same offset, $_r < $_r' iff r < r'.  A terminator stops
 * every comparison, so nothing past it is ever looked at. */
static int suffix_cmp(const suffix_t *a, const suffix_t *b) {
    uint64_t la = read_len(a->r) - a->p, lb = read_len(b->r) - b->p;
    const uint8_t *xa = g_reads + g_offsets[a->r] + a->p;
    const uint8_t *xb = g_reads + g_offsets[b->r] + b->p;
    uint64_t q = la < lb ? la : lb;
    for (uint64_t k = 0; k < q; ++k) {
        if (xa[k] != xb[k]) return xa[k] < xb[k] ? -1 : 1;
    }
#if ORACLE_PLANT == 3
    if (la != lb) return la < lb ? 1 : -1;
#else
    if (la != lb) return la < lb ? -1 : 1;
#endif
#if ORACLE_PLANT == 2
    if (a->r != b->r) return a->r < b->r ? 1 : -1;
#else
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
#endif
    return 0;
}

static int suffix_cmp_void(const void *a, const void *b) {
    return suffix_cmp((const suffix_t *)a, (const suffix_t *)b);
}

/* Check offsets and that every byte belongs to the alphabet. */
static int validate(const uint8_t *reads, const uint64_t *offsets, uint64_t m,
                    const uint8_t *alphabet, int sigma) {
    if (sigma < 1 || sigma > 16) return ORACLE_EINVAL;
    for (int a = 1; a < sigma; ++a)
        if (alphabet[a] <= alphabet[a - 1]) return ORACLE_EINVAL;
    if (offsets[0] != 0) return ORACLE_EINVAL;
    for (uint64_t r = 0; r < m; ++r) {
        if (offsets[r + 1] < offsets[r]) return ORACLE_EINVAL;
        for (uint64_t i = offsets[r]; i < offsets[r + 1]; ++i) {
            int ok = 0;
            for (int a = 0; a < sigma; ++a) ok |= reads[i] == alphabet[a];
            if (!ok) return ORACLE_EINVAL;
        }
    }
    return ORACLE_OK;
}

/* All suffixes of reads [r0, r1), in text order. */
static suffix_t *enumerate_suffixes(uint64_t r0, uint64_t r1, uint64_t *count) {
    uint64_t n = 0;
    for (uint64_t r = r0; r < r1; ++r) n += read_len(r) + 1;
    suffix_t *s = (suffix_t *)malloc((n ? n : 1) * sizeof(suffix_t));
    if (!s) return NULL;
    uint64_t t = 0;
    for (uint64_t r = r0; r < r1; ++r)
        for (uint64_t p = 0; p <= read_len(r); ++p) {
            s[t].r = r;
            s[t].p = p;
            ++t;
        }
    *count = n;
    return s;
}

/* B[i] = T[(SA[i]-1) mod n] (Eq. 1): the symbol before the suffix inside its
 * read, or a terminator when the suffix starts a read (for r = 0 that is
 * $_{m-1}, the wrap-around; for r > 0 it is $_{r-1}). */
static uint8_t preceding_symbol(const suffix_t *s) {
    if (s->p == 0) return (uint8_t)'$';
    return g_reads[g_offsets[s->r] + s->p - 1];
}

uint64_t oracle_num_suffixes(const uint64_t *offsets, uint64_t m) {
    return offsets[m] + m;
}

/* BWT of the whole set from the definition (Section 2, Eq. 1). */
int oracle_bwt(const uint8_t *reads, const uint64_t *offsets, uint64_t m,
               const uint8_t *alphabet, int sigma, uint8_t *B) {
    int rc = validate(reads, offsets, m, alphabet, sigma);
    if (rc) return rc;
    g_reads = reads;
    g_offsets = offsets;
    uint64_t n;
    suffix_t *s = enumerate_suffixes(0, m, &n);
    if (!s) return ORACLE_ENOMEM;
    qsort(s, n, sizeof(suffix_t), suffix_cmp_void);
    for (uint64_t i = 0; i < n; ++i) B[i] = preceding_symbol(&s[i]);
    free(s);
    return ORACLE_OK;
}

/* rank(c,k,B) = |{i<k : B[i]=c}| (Eq. 2). */
uint64_t oracle_rank(const uint8_t *B, uint64_t n, uint8_t c, uint64_t k) {
    uint64_t cnt = 0;
    if (k > n) k = n;
#if ORACLE_PLANT == 10
    for (uint64_t i = 0; i <= k && i < n; ++i) cnt += B[i] == c;
#else
    for (uint64_t i = 0; i < k; ++i) cnt += B[i] == c;
#endif
    return cnt;
}

static uint64_t block_start_of(uint64_t j0, uint64_t r) {
    /* block-local position of the first symbol of read r */
    return g_offsets[r] - g_offsets[j0] + (r - j0);
}

/* SA_int of the block of reads [j0, j1) (Algorithm 1, ConstructSA): the
 * block-local text positions of the block's suffixes in sorted order. */
int oracle_block_sa(const uint8_t *reads, const uint64_t *offsets, uint64_t j0,
                    uint64_t j1, uint64_t *sa) {
    g_reads = reads;
    g_offsets = offsets;
    uint64_t n;
    suffix_t *s = enumerate_suffixes(j0, j1, &n);
    if (!s) return ORACLE_ENOMEM;
    qsort(s, n, sizeof(suffix_t), suffix_cmp_void);
    for (uint64_t i = 0; i < n; ++i) sa[i] = block_start_of(j0, s[i].r) + s[i].p;
    free(s);
    return ORACLE_OK;
}

/* Maps a block-local position back to (read, offset) by walking the reads. */
static suffix_t locate(uint64_t j0, uint64_t j1, uint64_t t) {
    uint64_t lo = j0, hi = j1; /* last read whose start is <= t */
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (block_start_of(j0, mid) <= t) lo = mid; else hi = mid;
    }
    suffix_t s;
    s.r = lo;
    s.p = t - block_start_of(j0, lo);
    return s;
}

/* B_int[i] = the symbol preceding block suffix SA_int[i] inside its read,
 * '$' when the suffix starts its read (Algorithm 1, B(S_jk, SA_int)). */
int oracle_block_bint(const uint8_t *reads, const uint64_t *offsets, uint64_t j0,
                      uint64_t j1, const uint64_t *sa, uint64_t n_int,
                      uint8_t *bint) {
    g_reads = reads;
    g_offsets = offsets;
    for (uint64_t i = 0; i < n_int; ++i) {
        suffix_t s = locate(j0, j1, sa[i]);
#if ORACLE_PLANT == 13
        bint[i] = s.p == read_len(s.r) ? (uint8_t)'$' : preceding_symbol(&s);
#else
        bint[i] = preceding_symbol(&s);
#endif
    }
    return ORACLE_OK;
}

/* g[t] = |{old suffixes smaller than block suffix t}|, where the old
 * suffixes are those of reads [0, j0) and the block holds reads [j0, j1).
 * Old and new suffixes never compare equal (distinct terminators). */
int oracle_block_g_direct(const uint8_t *reads, const uint64_t *offsets,
                          uint64_t j0, uint64_t j1, uint64_t *g) {
    g_reads = reads;
    g_offsets = offsets;
    uint64_t n_old, n_new;
#if ORACLE_PLANT == 12
    suffix_t *old = enumerate_suffixes(0, j0 ? j0 - 1 : 0, &n_old);
#else
    suffix_t *old = enumerate_suffixes(0, j0, &n_old);
#endif
    suffix_t *neu = enumerate_suffixes(j0, j1, &n_new);
    if (!old || !neu) {
        free(old);
        free(neu);
        return ORACLE_ENOMEM;
    }
    qsort(old, n_old, sizeof(suffix_t), suffix_cmp_void);
    for (uint64_t t = 0; t < n_new; ++t) {
        uint64_t lo = 0, hi = n_old; /* first old suffix larger than neu[t] */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (suffix_cmp(&old[mid], &neu[t]) < 0) lo = mid + 1; else hi = mid;
        }
        g[t] = lo;
    }
    free(old);
    free(neu);
    return ORACLE_OK;
}

/* Code of a B byte: 0 for '$', 1 + alphabet index for a symbol. */
static int bcode(uint8_t b, const uint8_t *alphabet, int sigma) {
    if (b == '$') return 0;
    for (int a = 0; a < sigma; ++a)
        if (alphabet[a] == b) return 1 + a;
    return -1;
}

/* Algorithm 2 (ComputeRanks) over B_ext with Lemma 1 (Section 4):
 * for each read, i := m_ext at its terminator, then for k = |P|-1 .. 0:
 * i := C[c] + rank(c, i, B_ext) with c = P[k].  rank is read from a full
 * prefix-count table, C[c] counts every smaller symbol of B_ext including
 * its m_ext terminators. */
/* Algorithm 2 for the reads [j0, j1); `before` = 1 when the block goes
 * before every read of B_ext (the start rank is then 0, else m_ext). */
static int block_g_lemma1(const uint8_t *B_ext, uint64_t n_ext,
                          const uint8_t *reads, const uint64_t *offsets,
                          uint64_t j0, uint64_t j1, const uint8_t *alphabet,
                          int sigma, int before, uint64_t *g) {
    if (sigma < 1 || sigma > 16) return ORACLE_EINVAL; /* count arrays hold sigma + 1 <= 17 */
    g_reads = reads;
    g_offsets = offsets;
    uint64_t *occ = (uint64_t *)calloc((n_ext + 1) * (size_t)(sigma + 1), sizeof(uint64_t));
    if (!occ) return ORACLE_ENOMEM;
    /* occ[k*(sigma+1) + x] = number of code-x bytes in B_ext[0..k) */
    for (uint64_t k = 0; k < n_ext; ++k) {
        int x = bcode(B_ext[k], alphabet, sigma);
        if (x < 0) {
            free(occ);
            return ORACLE_EINVAL;
        }
        for (int y = 0; y <= sigma; ++y)
            occ[(k + 1) * (sigma + 1) + y] = occ[k * (sigma + 1) + y] + (x == y);
    }
    uint64_t C[17] = {0}; /* sigma + 1 <= 17 entries */
#if ORACLE_PLANT == 11
    for (int x = 1; x <= sigma && x <= 4; ++x) C[x] = C[x - 1] + occ[n_ext * (sigma + 1) + x - 1];
#else
    for (int x = 1; x <= sigma; ++x) C[x] = C[x - 1] + occ[n_ext * (sigma + 1) + x - 1];
#endif
    uint64_t m_ext = occ[n_ext * (sigma + 1) + 0];
#if ORACLE_PLANT == 5
    for (int x = 1; x <= sigma; ++x) C[x] -= m_ext;
#endif
    for (uint64_t j = j0; j < j1; ++j) {
        uint64_t start = block_start_of(j0, j);
        uint64_t k = read_len(j);
#if ORACLE_PLANT == 1
        uint64_t i = n_ext;
#elif ORACLE_PLANT == 6
        uint64_t i = m_ext;
        (void)before;
#else
        uint64_t i = before ? 0 : m_ext;
#endif
        g[start + k] = i;
        while (k > 0) {
            --k;
            int x = bcode(reads[offsets[j] + k], alphabet, sigma);
            if (x <= 0) {
                free(occ);
                return ORACLE_EINVAL;
            }
            i = C[x] + occ[i * (sigma + 1) + x];
            g[start + k] = i;
        }
    }
    free(occ);
    return ORACLE_OK;
}

int oracle_block_g_lemma1(const uint8_t *B_ext, uint64_t n_ext,
                          const uint8_t *reads, const uint64_t *offsets,
                          uint64_t j0, uint64_t j1, const uint8_t *alphabet,
                          int sigma, uint64_t *g) {
    return block_g_lemma1(B_ext, n_ext, reads, offsets, j0, j1, alphabet, sigma, 0, g);
}

/* Insert (Algorithm 1, Section 5) as a stable merge: new symbol i goes to row
 * g_sa[i] + i; the old rows fill the remaining rows in their own order.
 * g_sa must be non-decreasing with values in [0, n_ext]. */
int oracle_insert(const uint8_t *B_ext, uint64_t n_ext, const uint8_t *bint,
                  const uint64_t *g_sa, uint64_t n_int, uint8_t *out) {
    uint64_t n = n_ext + n_int;
    uint8_t *taken = (uint8_t *)calloc(n ? n : 1, 1);
    if (!taken) return ORACLE_ENOMEM;
    for (uint64_t i = 0; i < n_int; ++i) {
        if (g_sa[i] > n_ext || (i > 0 && g_sa[i] < g_sa[i - 1])) {
            free(taken);
            return ORACLE_EINVAL;
        }
#if ORACLE_PLANT == 4
        uint64_t row = (g_sa[i] < n_ext ? g_sa[i] + 1 : n_ext) + i;
#else
        uint64_t row = g_sa[i] + i;
#endif
        out[row] = bint[i];
        taken[row] = 1;
    }
    uint64_t r = 0;
    for (uint64_t row = 0; row < n; ++row)
        if (!taken[row]) out[row] = B_ext[r++];
    free(taken);
    return ORACLE_OK;
}

/* Algorithm 1 end to end over the given block boundaries
 * 0 = bounds[0] < ... < bounds[K] = m: per block ConstructSA, B_int,
 * ComputeRanks (Lemma 1), the g[SA_int] reordering and Insert. */
static int setbwte(const uint8_t *reads, const uint64_t *offsets, uint64_t m,
                   const uint8_t *alphabet, int sigma, const uint64_t *bounds,
                   uint64_t K, int reverse, uint8_t *B) {
    int rc = validate(reads, offsets, m, alphabet, sigma);
    if (rc) return rc;
    if (K == 0 || bounds[0] != 0 || bounds[K] != m) return ORACLE_EINVAL;
    uint64_t n_total = oracle_num_suffixes(offsets, m);
    uint8_t *ext = (uint8_t *)malloc(n_total + 1);
    uint8_t *nxt = (uint8_t *)malloc(n_total + 1);
    if (!ext || !nxt) {
        free(ext);
        free(nxt);
        return ORACLE_ENOMEM;
    }
    uint64_t n_ext = 0;
    for (uint64_t q = 0; q < K; ++q) {
        uint64_t b = reverse ? K - 1 - q : q;
        uint64_t j0 = bounds[b], j1 = bounds[b + 1];
        if (j1 < j0) rc = ORACLE_EINVAL;
        if (rc) break;
        uint64_t n_int = (offsets[j1] - offsets[j0]) + (j1 - j0);
        uint64_t *sa = (uint64_t *)malloc((n_int + 1) * sizeof(uint64_t));
        uint64_t *g = (uint64_t *)malloc((n_int + 1) * sizeof(uint64_t));
        uint64_t *gsa = (uint64_t *)malloc((n_int + 1) * sizeof(uint64_t));
        uint8_t *bint = (uint8_t *)malloc(n_int + 1);
        if (!sa || !g || !gsa || !bint) rc = ORACLE_ENOMEM;
        if (!rc) rc = oracle_block_sa(reads, offsets, j0, j1, sa);
        if (!rc) rc = oracle_block_bint(reads, offsets, j0, j1, sa, n_int, bint);
        if (!rc) rc = block_g_lemma1(ext, n_ext, reads, offsets, j0, j1, alphabet, sigma, reverse, g);
        if (!rc) {
            for (uint64_t i = 0; i < n_int; ++i) gsa[i] = g[sa[i]];
            rc = oracle_insert(ext, n_ext, bint, gsa, n_int, nxt);
        }
        free(sa);
        free(g);
        free(gsa);
        free(bint);
        if (rc) break;
        uint8_t *tmp = ext;
        ext = nxt;
        nxt = tmp;
        n_ext += n_int;
    }
    if (!rc) memcpy(B, ext, n_ext);
    free(ext);
    free(nxt);
    return rc;
}

int oracle_setbwte(const uint8_t *reads, const uint64_t *offsets, uint64_t m,
                   const uint8_t *alphabet, int sigma, const uint64_t *bounds,
                   uint64_t K, uint8_t *B) {
    return setbwte(reads, offsets, m, alphabet, sigma, bounds, K, 0, B);
}

int oracle_setbwte_reverse(const uint8_t *reads, const uint64_t *offsets, uint64_t m,
                           const uint8_t *alphabet, int sigma, const uint64_t *bounds,
                           uint64_t K, uint8_t *B) {
    return setbwte(reads, offsets, m, alphabet, sigma, bounds, K, 1, B);
}

/* Inverts B: for each r < m, start at row r (rows 0..m-1 hold the terminator
 * suffixes $_0..$_{m-1}, which sort first and in id order) and step
 * LF(i) = C[c] + rank(c, i) with c = B[i] until B[i] is a terminator; the
 * symbols met spell S_r backwards.  Writes the reads into reads_out
 * (capacity cap bytes) and their m+1 offsets.  Returns ORACLE_EINVAL when B
 * is not a consistent set BWT (an LF step leaves [0,n), a read runs longer
 * than n, or the number of '$' differs from m). */
int oracle_lf_invert(const uint8_t *B, uint64_t n, uint64_t m,
                     const uint8_t *alphabet, int sigma, uint8_t *reads_out,
                     uint64_t cap, uint64_t *offsets_out) {
    if (sigma < 1 || sigma > 16) return ORACLE_EINVAL; /* count arrays hold sigma + 1 <= 17 */
    uint64_t *occ = (uint64_t *)calloc((n + 1) * (size_t)(sigma + 1), sizeof(uint64_t));
    uint8_t *tmp = (uint8_t *)malloc(n + 1);
    if (!occ || !tmp) {
        free(occ);
        free(tmp);
        return ORACLE_ENOMEM;
    }
    int rc = ORACLE_OK;
    for (uint64_t k = 0; k < n && !rc; ++k) {
        int x = bcode(B[k], alphabet, sigma);
        if (x < 0) rc = ORACLE_EINVAL;
        for (int y = 0; y <= sigma && !rc; ++y)
            occ[(k + 1) * (sigma + 1) + y] = occ[k * (sigma + 1) + y] + (x == y);
    }
    if (!rc && occ[n * (sigma + 1)] != m) rc = ORACLE_EINVAL;
    uint64_t C[17] = {0}; /* sigma + 1 <= 17 entries */
    for (int x = 1; x <= sigma && !rc; ++x) C[x] = C[x - 1] + occ[n * (sigma + 1) + x - 1];
#if ORACLE_PLANT == 14
    for (int x = 1; x <= sigma && !rc; ++x) C[x] -= m;
#endif
    uint64_t w = 0;
    if (!rc) offsets_out[0] = 0;
    for (uint64_t r = 0; r < m && !rc; ++r) {
        uint64_t i = r, len = 0;
        for (;;) {
            int x = bcode(B[i], alphabet, sigma);
            if (x == 0) break;
            if (len >= n) {
                rc = ORACLE_EINVAL;
                break;
            }
            tmp[len++] = B[i];
            i = C[x] + occ[i * (sigma + 1) + x];
            if (i >= n) {
                rc = ORACLE_EINVAL;
                break;
            }
        }
        if (rc) break;
        if (w + len > cap) {
            rc = ORACLE_EINVAL;
            break;
        }
        for (uint64_t q = 0; q < len; ++q) reads_out[w + q] = tmp[len - 1 - q];
        w += len;
        offsets_out[r + 1] = w;
    }
    free(occ);
    free(tmp);
    return rc;
}

/* The same inversion with a lighter rank: counts of every code at each 64th
 * row, plus a plain count of the rows in between (for sets too large for
 * the full prefix-count table above).  Same contract as oracle_lf_invert. */
int oracle_lf_invert_sampled(const uint8_t *B, uint64_t n, uint64_t m, const uint8_t *alphabet, int sigma,
                             uint8_t *reads_out, uint64_t cap, uint64_t *offsets_out) {
    if (sigma < 1 || sigma > 16) return ORACLE_EINVAL; /* count arrays hold sigma + 1 <= 17 */
    const uint64_t nck = n / 64 + 1;
    uint64_t *ck = (uint64_t *)calloc(nck * (size_t)(sigma + 1), sizeof(uint64_t));
    int8_t *code = (int8_t *)malloc(n + 1);
    uint8_t *tmp = (uint8_t *)malloc(n + 1);
    if (!ck || !code || !tmp) {
        free(ck);
        free(code);
        free(tmp);
        return ORACLE_ENOMEM;
    }
    int rc = ORACLE_OK;
    uint64_t tot[17] = {0};
    for (uint64_t k = 0; k < n && !rc; ++k) {
#if ORACLE_PLANT != 8
        if (k % 64 == 0)
            for (int y = 0; y <= sigma; ++y) ck[(k / 64) * (sigma + 1) + y] = tot[y];
#endif
        int x = bcode(B[k], alphabet, sigma);
        if (x < 0) rc = ORACLE_EINVAL;
        else {
            code[k] = (int8_t)x;
            ++tot[x];
        }
#if ORACLE_PLANT == 8
        if (k % 64 == 0)
            for (int y = 0; y <= sigma; ++y) ck[(k / 64) * (sigma + 1) + y] = tot[y];
#endif
    }
    if (!rc && n % 64 == 0)
        for (int y = 0; y <= sigma; ++y) ck[(n / 64) * (sigma + 1) + y] = tot[y];
    if (!rc && tot[0] != m) rc = ORACLE_EINVAL;
    uint64_t C[17] = {0}; /* sigma + 1 <= 17 entries */
    for (int x = 1; x <= sigma && !rc; ++x) C[x] = C[x - 1] + tot[x - 1];
    uint64_t w = 0;
    if (!rc) offsets_out[0] = 0;
    for (uint64_t r = 0; r < m && !rc; ++r) {
        uint64_t i = r, len = 0;
        for (;;) {
            int x = code[i];
            if (x == 0) break;
            if (len >= n) {
                rc = ORACLE_EINVAL;
                break;
            }
            tmp[len++] = B[i];
            uint64_t rank = ck[(i / 64) * (sigma + 1) + x];
            for (uint64_t q = i - i % 64; q < i; ++q) rank += code[q] == x;
            i = C[x] + rank;
            if (i >= n) {
                rc = ORACLE_EINVAL;
                break;
            }
        }
        if (rc) break;
        if (w + len > cap) {
            rc = ORACLE_EINVAL;
            break;
        }
        for (uint64_t q = 0; q < len; ++q) reads_out[w + q] = tmp[len - 1 - q];
        w += len;
        offsets_out[r + 1] = w;
    }
    free(ck);
    free(code);
    free(tmp);
    return rc;
}

/* Occurrences of pattern P (bytes, no terminator) in the read set: every
 * (read, offset) where P starts, overlapping occurrences included, found by
 * direct comparison.  This is what FM-index backward search counts: the
 * suffixes of T that start with P (a terminator never matches a symbol, so
 * an occurrence never spans two reads). */
uint64_t oracle_count(const uint8_t *reads, const uint64_t *offsets, uint64_t m, const uint8_t *P, uint64_t len) {
    uint64_t cnt = 0;
    for (uint64_t r = 0; r < m; ++r) {
        const uint64_t L = offsets[r + 1] - offsets[r];
        if (len > L) continue;
#if ORACLE_PLANT == 7
        for (uint64_t p = 0; p + len <= L; ++p)
            if (memcmp(reads + offsets[r] + p, P, len) == 0) {
                ++cnt;
                if (len) p += len - 1;
            }
#else
        for (uint64_t p = 0; p + len <= L; ++p)
            cnt += memcmp(reads + offsets[r] + p, P, len) == 0;
#endif
    }
    return cnt;
}

/* Row of suffix (r, p) in the sorted order of all suffixes of the set:
 * the number of suffixes smaller than it, counted one comparison at a time
 * (O(n) comparisons, no sort). */
uint64_t oracle_row_of_suffix(const uint8_t *reads, const uint64_t *offsets,
                              uint64_t m, uint64_t r, uint64_t p) {
    g_reads = reads;
    g_offsets = offsets;
    suffix_t x;
    x.r = r;
    x.p = p;
    uint64_t row = 0;
    suffix_t y;
    for (y.r = 0; y.r < m; ++y.r)
        for (y.p = 0; y.p <= read_len(y.r); ++y.p)
#if ORACLE_PLANT == 9
            row += suffix_cmp(&y, &x) <= 0;
#else
            row += suffix_cmp(&y, &x) < 0;
#endif
    return row;
}

/* The symbol B holds at the row of suffix (r, p): Eq. 1 for one suffix. */
uint8_t oracle_bwt_symbol_of_suffix(const uint8_t *reads, const uint64_t *offsets,
                                    uint64_t r, uint64_t p) {
    g_reads = reads;
    g_offsets = offsets;
    suffix_t x;
    x.r = r;
    x.p = p;
    return preceding_symbol(&x);
}
