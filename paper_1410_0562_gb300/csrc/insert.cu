// insert.cu -- Insert (arXiv 1410.0562, Algorithm 1 and Section 5) as one
// stable parallel merge that writes the next rank dictionary.
//
// New symbol i (in SA_int order) lands on row g_sa[i] + i of the result: the
// g_sa[i] old rows below it plus the i new symbols before it.  New symbols
// with equal g_sa keep their SA_int order and go before old row g_sa (they
// are smaller: Lemma 1's g counts the old suffixes below the new one, and old
// and new suffixes never tie because their terminators differ).  Old rows
// keep their relative order.
//
// The 2-bit dictionary: one CTA builds one superblock (1024 occurrence blocks
// of 64 rows) from the new symbols that land in it, which bint_gather's plan
// names; it marks each output block's new rows in shared memory, derives
// where each block's old rows start from a scan of those marks, spreads the
// old rows around the new ones and scans the per-block counts for the 16-bit
// block counters (insert_kernel below).  The 4-bit dictionary (5 to 16
// symbols) splices the new symbols of each block one by one after a binary
// search for the first of them.  A one-CTA pass (three steps for many
// superblocks) then scans the superblock totals into the 64-bit superblock
// counters and C[] (Lemma 1's C[c] counts every smaller symbol, the
// terminators included).
#include <algorithm>

#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr int kInsertThreads = 512;        // threads of a 2-bit Insert CTA (one superblock), dense new rows
constexpr int kInsertThreadsSparse = 256;  // the same for sparse new rows
constexpr uint64_t kStageSupers = 512;      // superblocks per chunk of an in-place Insert
constexpr unsigned kStageGrid = 1216;       // CTAs of the staging copy (8 per SM)
constexpr uint64_t kStageBlocksW = 1ull << 19;  // output blocks per chunk of an in-place 4-bit Insert
constexpr int kRun = 8;              // consecutive new symbols a thread places at once
constexpr uint64_t kSparseSymbols = 4096;  // new symbols of a superblock (of 65536 rows) placed one by one

// 64 rows of the 2-bit dictionary as its three bit planes (bit p: row p).
struct Window {
    unsigned long long lo, hi, dm;
};

// The two 64-row parts a window starting at old row s reads (the second one
// zero past the old end), loaded before any of them is used.  Part P of a
// dictionary of sampling 64 K rows is words 3 (P % K) .. of block P / K.
struct OldPair {
    Window a, b;
};
template <int K>
__device__ __forceinline__ const unsigned long long* part_words(const unsigned long long* __restrict__ words,
                                                                uint64_t part) {
    return words + (part / K) * Occ<K>::kWords + 3 * (part % K);
}
// The old parts a window starting at row s reads, from blocks [base, base +
// avail) of the old dictionary held in old_words (the whole dictionary, or a
// staged copy of some of its blocks); a part outside them reads as zero and
// flags *d_err (an inconsistent plan).
template <int K>
__device__ __forceinline__ OldPair old_pair(const unsigned long long* __restrict__ old_words, uint64_t nparts_old,
                                            uint64_t s, uint64_t base, uint64_t avail, uint32_t* __restrict__ d_err) {
    const uint64_t P = s >> kOccShift;
    OldPair o;
    o.a = o.b = Window{0ull, 0ull, 0ull};
    const uint64_t ba = P / K;
    if (ba < base || ba - base >= avail) {
        atomicOr(d_err, 1024u);
        return o;
    }
    const bool has_b = P + 1 < nparts_old && (P + 1) / K - base < avail;
    if constexpr (K == 1) {
        const ulonglong2* A = reinterpret_cast<const ulonglong2*>(old_words) + 2 * (P - base);
        const ulonglong2 a0 = A[0], a1 = A[1];
        o.a = Window{a0.x, a0.y, a1.x};
        if (has_b) {
            const ulonglong2 b0 = A[2], b1 = A[3];
            o.b = Window{b0.x, b0.y, b1.x};
        }
    } else {
        const unsigned long long* pa = old_words + (ba - base) * Occ<K>::kWords + 3 * (P % K);
        o.a = Window{pa[0], pa[1], pa[2]};
        if (has_b) {
            const unsigned long long* pb = old_words + ((P + 1) / K - base) * Occ<K>::kWords + 3 * ((P + 1) % K);
            o.b = Window{pb[0], pb[1], pb[2]};
        }
    }
    return o;
}

// The old blocks that superblocks [S0, S1) of the next dictionary read,
// [b_lo, b_hi]: their windows start at old row S0 2^16 - ins_i0[S0] at the
// lowest and end within two parts of S1 2^16 - ins_i0[S1] (at most n_ext).
template <int K>
__device__ __forceinline__ void staged_range(const uint32_t* __restrict__ ins_i0, uint64_t n_ext, uint64_t S0,
                                             uint64_t S1, uint64_t& b_lo, uint64_t& b_hi) {
    const uint64_t o0 = S0 << kSuperShift, o1 = S1 << kSuperShift;
    const uint64_t lo_row = o0 - min((uint64_t)ins_i0[S0], o0);
    const uint64_t hi_row = min((uint64_t)n_ext, o1 - min((uint64_t)ins_i0[S1], o1)) + 2 * kOccSpan;
    const uint64_t rows_per_block = 64ull * K;
    const uint64_t last = n_ext / rows_per_block;  // the old dictionary's last block
    b_lo = min(lo_row / rows_per_block, last);
    b_hi = min(hi_row / rows_per_block, last);
}

// 64 old rows starting at row s, from the pair of parts holding them.
__device__ __forceinline__ Window old_window_of(const OldPair& o, uint64_t s) {
    const uint32_t off = (uint32_t)(s & (kOccSpan - 1));
    if (off == 0) return o.a;
    return Window{(o.a.lo >> off) | (o.b.lo << (64 - off)), (o.a.hi >> off) | (o.b.hi << (64 - off)),
                  (o.a.dm >> off) | (o.b.dm << (64 - off))};
}

// Opens an empty row at position p of the window: rows p.. move up by one
// and row 63 falls off (the same shift on each plane).
__device__ __forceinline__ unsigned long long open_bit(unsigned long long x, unsigned long long below) {
    return (x & below) | ((x & ~below) << 1);
}
__device__ __forceinline__ void open_row(Window& w, uint32_t p) {
    const unsigned long long below = (1ull << p) - 1ull;
    w.lo = open_bit(w.lo, below);
    w.hi = open_bit(w.hi, below);
    w.dm = open_bit(w.dm, below);
}

// Deposits the low popc(m) rows of w, in order, into the set bits of m on
// each plane (a parallel bit deposit): six stages that shift by 32, 16, ...,
// 1 rows, each moving the rows whose remaining distance has that bit.  The
// stage masks depend on m alone, so the three planes share them: stage i
// moves the bits of mv[i], where mv[i] marks (among the positions a
// compaction to the right would still move) those with an odd number of
// clear bits of m below them after the moves of stages 0 .. i-1 (the
// counts taken by a parallel suffix XOR).  This is the expand network of
// Hacker's Delight (Warren, 2nd ed., section 7-5).
__device__ __forceinline__ Window deposit_rows(Window w, unsigned long long m0) {
    unsigned long long m = m0, mk = ~m << 1, mv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned long long mp = mk ^ (mk << 1);
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        mp ^= mp << 32;
        mv[i] = mp & m;
        m = (m ^ mv[i]) | (mv[i] >> (1 << i));
        mk &= ~mp;
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        const int sh = 1 << i;
        w.lo = (w.lo & ~mv[i]) | ((w.lo << sh) & mv[i]);
        w.hi = (w.hi & ~mv[i]) | ((w.hi << sh) & mv[i]);
        w.dm = (w.dm & ~mv[i]) | ((w.dm << sh) & mv[i]);
    }
    return Window{w.lo & m0, w.hi & m0, w.dm & m0};
}

// Spreads the old rows of window w over the rows of an output part whose
// new rows are the set bits of F: the old rows keep their order and fill
// the clear bits of F, the rows of F are left empty.  Few new rows: open one
// row per set bit; few old rows: move each to its place; otherwise the
// deposit network.
constexpr uint32_t kOpenRows = 6;  // at most this many new rows: open them one by one
__device__ __forceinline__ Window spread_old(Window w, unsigned long long F) {
    const uint32_t k = __popcll(F);
    if (k <= kOpenRows) {
        while (F) {
            open_row(w, __ffsll((long long)F) - 1);
            F &= F - 1;
        }
        return w;
    }
    if (k < 64 - kOpenRows) return deposit_rows(w, ~F);
    Window o{0ull, 0ull, 0ull};
    unsigned long long z = ~F;
    uint32_t src = 0;
    while (z) {
        const uint32_t p = __ffsll((long long)z) - 1;
        z &= z - 1;
        o.lo |= ((w.lo >> src) & 1ull) << p;
        o.hi |= ((w.hi >> src) & 1ull) << p;
        o.dm |= ((w.dm >> src) & 1ull) << p;
        ++src;
    }
    return o;
}

// kRun consecutive g_sa values from a 16-byte aligned address.
template <class IdxT>
__device__ __forceinline__ void load_run(const IdxT* __restrict__ p, IdxT (&v)[kRun]) {
    static_assert(kRun == 8, "two 16-byte loads of 32-bit values, four of 64-bit ones");
    if constexpr (sizeof(IdxT) == 4) {
        const uint4 a = reinterpret_cast<const uint4*>(p)[0], b = reinterpret_cast<const uint4*>(p)[1];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const ulonglong2 a = reinterpret_cast<const ulonglong2*>(p)[q];
            v[2 * q] = a.x;
            v[2 * q + 1] = a.y;
        }
    }
}

// One CTA builds one superblock of the next dictionary (kBlocksPerSuper
// output parts of 64 rows, rows [O, O + 2^16)) from the new symbols
// [ins_i0[S], ins_i0[S+1]) that land in it (bint_gather wrote that plan):
//  1. the CTA reads those new symbols' rows g_sa[i] + i and codes (a run of
//     consecutive ones per thread) and sets, per output part, the mask F of
//     its new rows and their three planes at their rows (shared memory; a
//     thread merges the bits of its run per part first);
//  2. a scan of popcount(F) over the parts gives the new symbols before each
//     part, so part j's old rows are the contiguous run starting at old row
//     64 j - (new symbols before row 64 j);
//  3. each thread builds output parts (strided, so loads and stores of a
//     warp are contiguous): the 64-row old window, spread over the clear bits
//     of F, OR the new rows' planes;
//  4. a scan of the per-part counts gives the 16-bit block counters (the
//     count before the first part of each occurrence block);
//  5. the parts are written into their blocks of 64 K rows.
// Every index that comes from g_sa is checked; an inconsistent plan flags
// *d_err (bit 10) and never leads outside the arrays.
// With `staged`, the grid covers superblocks [sb_first, sb_first + grid)
// and old_words holds a staged copy of the old blocks they read
// (staged_range, at most stage_blocks of them); without it, old_words is the
// whole old dictionary and sb_first is 0.
template <class IdxT, int kT, int K>
__global__ void __launch_bounds__(kT, kT == 256 ? 4 : 2) insert_kernel(const unsigned long long* __restrict__ old_words,
                                                    unsigned long long n_ext, const uint8_t* __restrict__ bint,
                                                    const IdxT* __restrict__ gsa, unsigned long long n_int,
                                                    const uint32_t* __restrict__ ins_i0,
                                                    unsigned long long* __restrict__ new_words,
                                                    unsigned long long n_new, uint32_t* __restrict__ sb_tot,
                                                    uint32_t* __restrict__ d_err, unsigned long long sb_first,
                                                    int staged, unsigned long long stage_blocks) {
    constexpr int kNB = kBlocksPerSuper, kPer = kNB / kT;
    __shared__ uint32_t sF[2][kNB];  // new rows of each part (rows 0-31, 32-63); later its counts
    __shared__ uint32_t sD[2][kNB];  // terminator plane: of the new rows, later of the whole part
    __shared__ uint32_t sC[4][kNB];  // lo plane (words 0, 1) and hi plane (2, 3): of the new rows, then the part
    __shared__ uint32_t sP[2][kNB];  // new symbols before each part; later the block counters
    const int tid = threadIdx.x;
    const uint64_t S = sb_first + blockIdx.x;
    const uint64_t O = S << kSuperShift;
    const uint64_t p_first = S * kNB;
    const uint64_t np_new = dict_parts(n_new, K);
    const uint64_t np_old = dict_parts(n_ext, K);
    uint64_t base = 0, avail = n_ext / (64ull * K) + 1;  // old blocks old_words holds
    if (staged) {
        uint64_t b_hi;
        staged_range<K>(ins_i0, n_ext, sb_first, sb_first + gridDim.x, base, b_hi);
        avail = min(b_hi - base + 1, (uint64_t)stage_blocks);
    }
    for (int x = tid; x < kNB; x += kT) {
        sF[0][x] = sF[1][x] = sD[0][x] = sD[1][x] = 0u;
        sC[0][x] = sC[1][x] = sC[2][x] = sC[3][x] = 0u;
    }
    uint64_t i_begin = ins_i0[S], i_end = ins_i0[S + 1];
    if (i_end > n_int || i_begin > i_end) {
        if (tid == 0) atomicOr(d_err, 1024u);
        i_end = min(i_end, (uint64_t)n_int);
        i_begin = min(i_begin, i_end);
    }

    __syncthreads();

    // 1. the new rows of every part of this superblock: each thread takes
    //    runs of kRun consecutive new symbols (runs start at multiples of
    //    kRun, so the superblock's first and last runs may hold fewer; a
    //    whole run's g_sa and codes arrive as vector loads).  Their rows
    //    increase, so a run touches one or two parts when new rows are
    //    dense: the thread gathers each part's bits (new-row mask,
    //    terminator and code planes, as 32-bit halves) in registers and ORs
    //    them into shared memory once per part.  A run over one or two
    //    parts takes one pass per part over all of its symbols, so the lanes
    //    of a warp stay together (a divergent part change in the middle of
    //    a run cost more than the passes).  A superblock with few new rows
    //    skips the runs.
    if (i_end - i_begin <= kSparseSymbols) {
        // few new rows: one symbol per thread and step, its bits ORed into
        // shared memory directly (new rows rarely share a part, so the
        // atomics rarely meet); the loads of four steps go out together
        for (uint64_t i0 = i_begin + tid; i0 < i_end; i0 += 4 * (uint64_t)kT) {
            IdxT gv[4];
            uint32_t xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + (uint64_t)u * kT;
                gv[u] = i < i_end ? gsa[i] : (IdxT)0;
                xv[u] = i < i_end ? bint[i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + (uint64_t)u * kT;
                if (i >= i_end) break;
                const IdxT local = gv[u] + (IdxT)i - (IdxT)O;
                if (local >= (IdxT)(1u << kSuperShift)) {  // not in this superblock: the plan is inconsistent
                    atomicOr(d_err, 1024u);
                    continue;
                }
                const uint32_t l = (uint32_t)local, j = l >> kOccShift, h = (l >> 5) & 1u, bit = 1u << (l & 31u);
                const uint32_t x = xv[u];
                atomicOr(&sF[h][j], bit);
                if (x == kBintDollar) {
                    atomicOr(&sD[h][j], bit);
                } else {
                    if (x & 1u) atomicOr(&sC[h][j], bit);
                    if (x & 2u) atomicOr(&sC[2 + h][j], bit);
                }
            }
        }
    } else {
        uint32_t cj = 0xFFFFFFFFu;  // the part being gathered
        uint32_t f0 = 0, f1 = 0, d0 = 0, d1 = 0, l0 = 0, l1 = 0, h0 = 0, h1 = 0;
        auto flush = [&]() {
            if (cj == 0xFFFFFFFFu) return;
            if (f0) atomicOr(&sF[0][cj], f0);
            if (f1) atomicOr(&sF[1][cj], f1);
            if (d0) atomicOr(&sD[0][cj], d0);
            if (d1) atomicOr(&sD[1][cj], d1);
            if (l0) atomicOr(&sC[0][cj], l0);
            if (l1) atomicOr(&sC[1][cj], l1);
            if (h0) atomicOr(&sC[2][cj], h0);
            if (h1) atomicOr(&sC[3][cj], h1);
            f0 = f1 = d0 = d1 = l0 = l1 = h0 = h1 = 0;
        };
        // row q of the current part with code x (a terminator when x is kBintDollar)
        auto mark = [&](uint32_t q, uint32_t x, uint32_t on) {
            const uint32_t b = on << (q & 31u);
            const uint32_t blo = q < 32u ? b : 0u, bhi = q < 32u ? 0u : b;
            const uint32_t isd = x == kBintDollar ? 0xFFFFFFFFu : 0u;
            const uint32_t m1 = (x & 1u) ? ~isd : 0u, m2 = (x & 2u) ? ~isd : 0u;
            f0 |= blo;
            f1 |= bhi;
            d0 |= blo & isd;
            d1 |= bhi & isd;
            l0 |= blo & m1;
            l1 |= bhi & m1;
            h0 |= blo & m2;
            h1 |= bhi & m2;
        };
        for (uint64_t base = (i_begin & ~(uint64_t)(kRun - 1)) + (uint64_t)tid * kRun; base < i_end;
             base += (uint64_t)kT * kRun) {
            IdxT gv[kRun];
            uint32_t xs[kRun];
            uint32_t valid;
            if (base >= i_begin && base + kRun <= i_end) {
                load_run<IdxT>(gsa + base, gv);
                const uint2 b8 = *reinterpret_cast<const uint2*>(bint + base);
#pragma unroll
                for (int u = 0; u < kRun; ++u) xs[u] = ((u < 4 ? b8.x : b8.y) >> (8 * (u & 3))) & 0xFFu;
                valid = (1u << kRun) - 1u;
            } else {
                valid = 0;
#pragma unroll
                for (int u = 0; u < kRun; ++u) {
                    const uint64_t i = base + u;
                    const bool in = i >= i_begin && i < i_end;
                    gv[u] = in ? gsa[i] : (IdxT)0;
                    xs[u] = in ? bint[i] : 0u;
                    valid |= (uint32_t)in << u;
                }
            }
            // rows inside the superblock (row arithmetic in the index type: a
            // 32-bit index has fewer than 2^32 rows)
            uint32_t loc[kRun], j_lo = 0xFFFFFFFFu, j_hi = 0;
            const IdxT rel = (IdxT)base - (IdxT)O;
#pragma unroll
            for (int u = 0; u < kRun; ++u) {
                const IdxT local = gv[u] + rel + (IdxT)u;
                loc[u] = (uint32_t)local;
                if ((valid >> u) & 1u) {
                    if (local >= (IdxT)(1u << kSuperShift)) {  // not in this superblock: the plan is inconsistent
                        atomicOr(d_err, 1024u);
                        valid &= ~(1u << u);
                    } else {
                        j_lo = min(j_lo, loc[u] >> kOccShift);
                        j_hi = max(j_hi, loc[u] >> kOccShift);
                    }
                }
            }
            if (!valid) continue;
            if (j_hi - j_lo < 2) {
                // one or two parts (dense new rows): a pass over the run per
                // part, every pass the same for all lanes, so a warp does not
                // split at each part change
                for (uint32_t jj = j_lo; jj <= j_hi; ++jj) {
                    if (jj != cj) {
                        flush();
                        cj = jj;
                    }
#pragma unroll
                    for (int u = 0; u < kRun; ++u)
                        mark(loc[u] & 63u, xs[u], ((valid >> u) & 1u) & (uint32_t)((loc[u] >> kOccShift) == jj));
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < kRun; ++u) {
                if (!((valid >> u) & 1u)) continue;
                const uint32_t j = loc[u] >> kOccShift;
                if (j != cj) {
                    flush();
                    cj = j;
                }
                mark(loc[u] & 63u, xs[u], 1u);
            }
        }
        flush();
    }
    __syncthreads();

    // 2. new symbols before each part (parts kPer * tid .. in order)
    {
        uint32_t c[kPer], tot = 0;
#pragma unroll
        for (int bb = 0; bb < kPer; ++bb) {
            const int j = kPer * tid + bb;
            c[bb] = __popc(sF[0][j]) + __popc(sF[1][j]);
            tot += c[bb];
        }
        uint32_t all;
        uint32_t ex = cta_exclusive_scan<SumOp, kT>(tot, all);
#pragma unroll
        for (int bb = 0; bb < kPer; ++bb) {
            sP[0][kPer * tid + bb] = ex;
            ex += c[bb];
        }
        // two new symbols on one row, or one outside this superblock
        if (tid == 0 && all != (uint32_t)(i_end - i_begin)) atomicOr(d_err, 1024u);
    }
    __syncthreads();

    // 3. build parts tid, tid + kT, ...; keep them in shared memory
#pragma unroll
    for (int bb = 0; bb < kPer; ++bb) {
        const int j = tid + bb * kT;
        const uint64_t b = p_first + j;
        if (b >= np_new) {
            sF[0][j] = sF[1][j] = 0u;
            continue;
        }
        const uint64_t o = b << kOccShift;
        const uint64_t inew = i_begin + sP[0][j];  // new symbols before row o
        uint64_t s_old = o - inew;
        if (inew > o || s_old > n_ext) {
            // (parts past the last row, in the last block of 64 K rows,
            // hold nothing: their window is never used)
            if (o <= n_new) atomicOr(d_err, 1024u);
            s_old = inew > o ? 0ull : (uint64_t)n_ext;
        }
        const OldPair op = old_pair<K>(old_words, np_old, s_old, base, avail, d_err);
        const unsigned long long F = (unsigned long long)sF[0][j] | ((unsigned long long)sF[1][j] << 32);
        Window w = spread_old(old_window_of(op, s_old), F);
        w.lo |= (unsigned long long)sC[0][j] | ((unsigned long long)sC[1][j] << 32);
        w.hi |= (unsigned long long)sC[2][j] | ((unsigned long long)sC[3][j] << 32);
        w.dm |= (unsigned long long)sD[0][j] | ((unsigned long long)sD[1][j] << 32);
        const uint32_t valid = n_new > o ? (uint32_t)min((unsigned long long)kOccSpan, n_new - o) : 0u;
        const unsigned long long vm = low_bits(valid);
        w.lo &= vm;
        w.hi &= vm;
        w.dm &= vm;
        // per-code counts: c = 3 on both planes, 1 and 2 on one, 0 the rest
        const unsigned long long live = vm & ~w.dm;
        const uint32_t n3 = __popcll(w.lo & w.hi & live);
        const uint32_t n1 = __popcll(w.lo & live) - n3, n2 = __popcll(w.hi & live) - n3;
        const uint32_t n0 = __popcll(live) - n1 - n2 - n3;
        sC[0][j] = (uint32_t)w.lo;
        sC[1][j] = (uint32_t)(w.lo >> 32);
        sC[2][j] = (uint32_t)w.hi;
        sC[3][j] = (uint32_t)(w.hi >> 32);
        sD[0][j] = (uint32_t)w.dm;
        sD[1][j] = (uint32_t)(w.dm >> 32);
        sF[0][j] = n0 | (n1 << 16);
        sF[1][j] = n2 | (n3 << 16);
    }
    __syncthreads();

    // 4. 16-bit block counters: exclusive scan of the counts in part order
    {
        unsigned long long t01 = 0, t23 = 0;
        uint32_t a[kPer], d[kPer];
#pragma unroll
        for (int bb = 0; bb < kPer; ++bb) {
            a[bb] = sF[0][kPer * tid + bb];
            d[bb] = sF[1][kPer * tid + bb];
            t01 += (unsigned long long)(a[bb] & 0xFFFFu) | ((unsigned long long)(a[bb] >> 16) << 32);
            t23 += (unsigned long long)(d[bb] & 0xFFFFu) | ((unsigned long long)(d[bb] >> 16) << 32);
        }
        unsigned long long tot01, tot23;
        const unsigned long long e01 = cta_exclusive_scan<SumOp, kT>(t01, tot01);
        const unsigned long long e23 = cta_exclusive_scan<SumOp, kT>(t23, tot23);
        uint32_t p0 = (uint32_t)e01, p1 = (uint32_t)(e01 >> 32), p2 = (uint32_t)e23, p3 = (uint32_t)(e23 >> 32);
#pragma unroll
        for (int bb = 0; bb < kPer; ++bb) {
            sP[0][kPer * tid + bb] = p0 | (p1 << 16);
            sP[1][kPer * tid + bb] = p2 | (p3 << 16);
            p0 += a[bb] & 0xFFFFu;
            p1 += a[bb] >> 16;
            p2 += d[bb] & 0xFFFFu;
            p3 += d[bb] >> 16;
        }
        if (tid == 0) {
            uint32_t* t = sb_tot + 4ull * S;
            t[0] = (uint32_t)tot01;
            t[1] = (uint32_t)(tot01 >> 32);
            t[2] = (uint32_t)tot23;
            t[3] = (uint32_t)(tot23 >> 32);
        }
    }
    __syncthreads();

    // 5. write the parts out (a warp stores 32 consecutive parts); the first
    //    part of each occurrence block also writes the block's counters
#pragma unroll
    for (int bb = 0; bb < kPer; ++bb) {
        const int j = tid + bb * kT;
        const uint64_t b = p_first + j;
        if (b >= np_new) break;
        const unsigned long long lo = (unsigned long long)sC[0][j] | ((unsigned long long)sC[1][j] << 32);
        const unsigned long long hi = (unsigned long long)sC[2][j] | ((unsigned long long)sC[3][j] << 32);
        const unsigned long long dm = (unsigned long long)sD[0][j] | ((unsigned long long)sD[1][j] << 32);
        const unsigned long long cnt = (unsigned long long)sP[0][j] | ((unsigned long long)sP[1][j] << 32);
        if constexpr (K == 1) {
            ulonglong2* dst = reinterpret_cast<ulonglong2*>(new_words) + 2 * b;
            dst[0] = make_ulonglong2(lo, hi);
            dst[1] = make_ulonglong2(dm, cnt);
        } else {
            unsigned long long* dst = new_words + (b / K) * Occ<K>::kWords;
            const uint32_t q = (uint32_t)(b % K);
            dst[3 * q] = lo;
            dst[3 * q + 1] = hi;
            dst[3 * q + 2] = dm;
            if (q == 0) dst[3 * K] = cnt;
        }
    }
}

// Copies the old blocks that superblocks [S0, S1) of the next dictionary
// read (staged_range) from the dictionary being rewritten in place into the
// staging buffer, before those superblocks overwrite any of them.
template <int K>
__global__ void __launch_bounds__(kThreads) stage_old_kernel(const unsigned long long* __restrict__ old_words,
                                                             unsigned long long n_ext,
                                                             const uint32_t* __restrict__ ins_i0,
                                                             unsigned long long S0, unsigned long long S1,
                                                             unsigned long long* __restrict__ stage,
                                                             unsigned long long stage_blocks,
                                                             uint32_t* __restrict__ d_err) {
    uint64_t b_lo, b_hi;
    staged_range<K>(ins_i0, n_ext, S0, S1, b_lo, b_hi);
    uint64_t blocks = b_hi - b_lo + 1;
    if (blocks > stage_blocks) {  // cannot happen for a consistent plan: the chunk's parts need fewer
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(d_err, 1024u);
        blocks = stage_blocks;
    }
    const uint64_t words = blocks * Occ<K>::kWords;
    const unsigned long long* src = old_words + b_lo * Occ<K>::kWords;
    for (uint64_t w = (uint64_t)blockIdx.x * kThreads + threadIdx.x; w < words; w += (uint64_t)gridDim.x * kThreads)
        stage[w] = src[w];
}

// ---------------------------------------------------------------------------
// The same merge for the 4-bit dictionary (5 to 16 symbols): one output
// block per thread, a CTA of 256 threads builds four 64-block superblocks;
// the 12-bit block counters are scanned per code across the 64 threads of a
// superblock (two warps).

__device__ __forceinline__ unsigned long long funnel_r(unsigned long long lo, unsigned long long hi, uint32_t bs) {
    return bs == 0 ? lo : (lo >> bs) | (hi << (64 - bs));
}

struct WindowW {
    unsigned long long w[4], dm;
};

// 64 old rows starting at row s (rows past the old end read as zero).
// old_blocks holds old blocks [base, base + avail) (all of them, or a
// staged copy); a block outside reads as zero and flags *d_err.
__device__ __forceinline__ WindowW old_window_w(const OccBlockW* __restrict__ old_blocks, uint64_t nb_old, uint64_t s,
                                                uint64_t base, uint64_t avail, uint32_t* __restrict__ d_err) {
    const uint64_t bs = s >> kOccShift;
    const uint32_t off = (uint32_t)(s & (kOccSpan - 1));
    if (bs < base || bs - base >= avail) {
        atomicOr(d_err, 1024u);
        WindowW z;
        z.w[0] = z.w[1] = z.w[2] = z.w[3] = z.dm = 0ull;
        return z;
    }
    const OccBlockW& A = old_blocks[bs - base];
    unsigned long long x[9];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = A.sym[k];
    unsigned long long da = A.dmask, db = 0;
#pragma unroll
    for (int k = 4; k < 9; ++k) x[k] = 0;
    if (bs + 1 < nb_old && bs + 1 - base < avail) {
        const OccBlockW& B = old_blocks[bs + 1 - base];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[4 + k] = B.sym[k];
        db = B.dmask;
    }
    // shift the 512-bit pair right by 4 * off bits: whole words first
    const uint32_t sh = 4 * off, ws = sh >> 6, bsh = sh & 63;
    if (ws & 2) {
#pragma unroll
        for (int k = 0; k < 7; ++k) x[k] = k + 2 < 9 ? x[k + 2] : 0ull;
    }
    if (ws & 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = x[k + 1];
    }
    WindowW w;
#pragma unroll
    for (int k = 0; k < 4; ++k) w.w[k] = funnel_r(x[k], x[k + 1], bsh);
    w.dm = off == 0 ? da : ((da >> off) | (db << (64 - off)));
    return w;
}

// Splice one row holding `code` (terminator when dollar) in at position p.
__device__ __forceinline__ void splice_w(WindowW& w, uint32_t p, uint32_t code, uint32_t dollar) {
    const uint32_t k = p >> 4, b = 4 * (p & 15);
#pragma unroll
    for (int j = 3; j > 0; --j)
        if ((uint32_t)j > k) w.w[j] = (w.w[j] << 4) | (w.w[j - 1] >> 60);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((uint32_t)j == k) {
            const unsigned long long keep = low_bits(b);
            w.w[j] = (w.w[j] & keep) | ((unsigned long long)code << b) | ((w.w[j] & ~keep) << 4);
        }
    }
    const unsigned long long keepd = low_bits(p);
    w.dm = (w.dm & keepd) | ((unsigned long long)dollar << p) | ((w.dm & ~keepd) << 1);
}

// The first new symbol at or after row o: |{i : g_sa[i] + i < o}|.
template <class IdxT>
__device__ __forceinline__ uint64_t first_new_at(const IdxT* __restrict__ gsa, uint64_t n_int, uint64_t o) {
    uint64_t lo = 0, hi = n_int;
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if ((uint64_t)gsa[mid] + mid < o) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The old blocks [b_lo, b_hi] that output blocks [b0, b1) of the 4-bit
// dictionary read (as staged_range for the 2-bit one).
template <class IdxT>
__device__ __forceinline__ void staged_range_w(const IdxT* __restrict__ gsa, uint64_t n_int, uint64_t n_ext,
                                               uint64_t b0, uint64_t b1, uint64_t& b_lo, uint64_t& b_hi) {
    const uint64_t o0 = b0 << kOccShift, o1 = b1 << kOccShift;
    const uint64_t i0 = first_new_at(gsa, n_int, o0), i1 = first_new_at(gsa, n_int, o1);
    const uint64_t nb = (n_ext >> kOccShift) + 1;
    b_lo = min((o0 - min(i0, o0)) >> kOccShift, nb - 1);
    b_hi = min((min((uint64_t)n_ext, o1 - min(i1, o1)) + 2 * kOccSpan) >> kOccShift, nb - 1);
}

template <class IdxT>
__global__ void __launch_bounds__(kThreads) stage_old_w_kernel(const OccBlockW* __restrict__ old_blocks,
                                                               unsigned long long n_ext, const IdxT* __restrict__ gsa,
                                                               unsigned long long n_int, unsigned long long b0,
                                                               unsigned long long b1, OccBlockW* __restrict__ stage,
                                                               unsigned long long stage_blocks,
                                                               uint32_t* __restrict__ d_err) {
    __shared__ unsigned long long s_lo, s_n;
    if (threadIdx.x == 0) {
        uint64_t lo, hi;
        staged_range_w(gsa, n_int, n_ext, b0, b1, lo, hi);
        uint64_t nblk = hi - lo + 1;
        if (nblk > stage_blocks) {
            if (blockIdx.x == 0) atomicOr(d_err, 1024u);
            nblk = stage_blocks;
        }
        s_lo = lo;
        s_n = nblk;
    }
    __syncthreads();
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(old_blocks + s_lo);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(stage);
    for (uint64_t v = (uint64_t)blockIdx.x * kThreads + threadIdx.x; v < 4 * s_n; v += (uint64_t)gridDim.x * kThreads)
        dst[v] = src[v];
}

template <class IdxT>
__global__ void __launch_bounds__(kThreads) insert_w_kernel(const OccBlockW* __restrict__ old_blocks,
                                                            unsigned long long n_ext, const uint8_t* __restrict__ bint,
                                                            const IdxT* __restrict__ gsa, unsigned long long n_int,
                                                            OccBlockW* __restrict__ new_blocks,
                                                            unsigned long long n_new, unsigned long long nsb,
                                                            uint32_t* __restrict__ sb_tot, uint32_t* __restrict__ d_err,
                                                            unsigned long long b_first, int staged,
                                                            unsigned long long stage_blocks) {
    __shared__ uint32_t warp_tot[kThreads / 32][kSigmaW];
    __shared__ unsigned long long s_base, s_avail;
    const uint64_t nb_new = (n_new >> kOccShift) + 1;
    const uint64_t nb_old = (n_ext >> kOccShift) + 1;
    const uint64_t b = b_first + (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (threadIdx.x == 0) {
        uint64_t lo = 0, hi = nb_old - 1;
        if (staged) staged_range_w(gsa, n_int, n_ext, b_first, b_first + (uint64_t)gridDim.x * kThreads, lo, hi);
        s_base = lo;
        s_avail = staged ? min(hi - lo + 1, (uint64_t)stage_blocks) : nb_old;
    }
    __syncthreads();
    const uint64_t base = s_base, avail = s_avail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WindowW w;
    w.w[0] = w.w[1] = w.w[2] = w.w[3] = w.dm = 0;
    uint32_t cnt[kSigmaW];
#pragma unroll
    for (int c = 0; c < kSigmaW; ++c) cnt[c] = 0;
    if (b < nb_new) {
        const uint64_t o = b << kOccShift;
        uint64_t lo = 0, hi = n_int;  // first i with g_sa[i] + i >= o
        while (lo < hi) {
            const uint64_t mid = lo + ((hi - lo) >> 1);
            if ((uint64_t)gsa[mid] + mid < o) lo = mid + 1; else hi = mid;
        }
        uint64_t i = lo;
        const uint64_t s_old = o >= i ? min((unsigned long long)(o - i), n_ext) : 0ull;
        w = old_window_w(old_blocks, nb_old, s_old, base, avail, d_err);
        while (i < n_int) {
            const uint64_t row = (uint64_t)gsa[i] + i;
            if (row >= o + kOccSpan) break;
            const uint8_t x = bint[i];
            splice_w(w, (uint32_t)(row - o), x == kBintDollar ? 0u : x, x == kBintDollar ? 1u : 0u);
            ++i;
        }
        const uint32_t valid = n_new > o ? (uint32_t)min((unsigned long long)kOccSpan, n_new - o) : 0u;
        unsigned long long vm[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t rows = valid > 16u * k ? min(valid - 16u * k, 16u) : 0u;
            vm[k] = low_bits(4 * rows);
            w.w[k] &= vm[k];
        }
        w.dm &= low_bits(valid);
#pragma unroll
        for (int c = 0; c < kSigmaW; ++c) {
            uint32_t s = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) s += __popcll(match_code4(w.w[k], c) & vm[k]);
            cnt[c] = s;
        }
        cnt[0] -= __popcll(w.dm);
    }
    // per code: inclusive scan over the superblock's 64 threads (two warps)
    uint32_t incl[kSigmaW];
#pragma unroll
    for (int c = 0; c < kSigmaW; ++c) {
        uint32_t x = cnt[c];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        incl[c] = x;
        if (lane == 31) warp_tot[warp][c] = x;
    }
    __syncthreads();
    if (warp & 1) {
#pragma unroll
        for (int c = 0; c < kSigmaW; ++c) incl[c] += warp_tot[warp - 1][c];
    }
    if (b < nb_new) {
        unsigned long long cw[3] = {0ull, 0ull, 0ull};
#pragma unroll
        for (int c = 0; c < kSigmaW; ++c) {
            const unsigned long long v = (incl[c] - cnt[c]) & 0xFFFu;  // exclusive: below 4096
            const int o = 12 * c, wd = o >> 6, sh = o & 63;
            cw[wd] |= v << sh;
            if (sh > 52) cw[wd + 1] |= v >> (64 - sh);
        }
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(new_blocks + b);
        dst[0] = make_ulonglong2(w.w[0], w.w[1]);
        dst[1] = make_ulonglong2(w.w[2], w.w[3]);
        dst[2] = make_ulonglong2(w.dm, cw[0]);
        dst[3] = make_ulonglong2(cw[1], cw[2]);
    }
    const uint64_t s = b >> (kSuperShiftW - kOccShift);
    if ((b & (kBlocksPerSuperW - 1)) == kBlocksPerSuperW - 1 && s < nsb) {
#pragma unroll
        for (int c = 0; c < kSigmaW; ++c) sb_tot[(uint64_t)kSigmaW * s + c] = incl[c];
    }
}

constexpr int kScanThreads = 256;

// Superblock counters from the per-superblock totals in three steps: each
// CTA scans 256 superblocks (one scan per code) and keeps its totals; one
// CTA scans those totals and writes C[] (Lemma 1's C counts the terminators
// too); each CTA adds its offsets.  Up to kSmallScan superblocks take one
// CTA instead (below).
template <int kCodes>
__global__ void __launch_bounds__(kScanThreads) super_local_kernel(const uint32_t* __restrict__ sb_tot,
                                                                   unsigned long long nsb,
                                                                   unsigned long long* __restrict__ super,
                                                                   unsigned long long* __restrict__ chunk_tot) {
    const unsigned long long s = (unsigned long long)blockIdx.x * kScanThreads + threadIdx.x;
#pragma unroll 1
    for (int c = 0; c < kCodes; ++c) {
        const unsigned long long v = s < nsb ? sb_tot[kCodes * s + c] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = cta_exclusive_scan<SumOp, kScanThreads>(v, tot);
        if (s < nsb) super[kCodes * s + c] = ex;
        if (threadIdx.x == 0) chunk_tot[(unsigned long long)kCodes * blockIdx.x + c] = tot;
    }
}

template <int kCodes>
__global__ void __launch_bounds__(kScanThreads) super_chunks_kernel(unsigned long long* __restrict__ chunk_tot,
                                                                    unsigned long long nchunks,
                                                                    unsigned long long* __restrict__ C,
                                                                    unsigned long long m) {
    __shared__ unsigned long long code_tot[kCodes];
#pragma unroll 1
    for (int c = 0; c < kCodes; ++c) {
        unsigned long long carry = 0;
        for (unsigned long long b = 0; b < nchunks; b += kScanThreads) {
            const unsigned long long k = b + threadIdx.x;
            const unsigned long long v = k < nchunks ? chunk_tot[kCodes * k + c] : 0ull;
            unsigned long long tot;
            const unsigned long long ex = cta_exclusive_scan<SumOp, kScanThreads>(v, tot);
            if (k < nchunks) chunk_tot[kCodes * k + c] = carry + ex;
            carry += tot;
        }
        if (threadIdx.x == 0) code_tot[c] = carry;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = m;
        for (int c = 0; c < kCodes; ++c) {
            C[c] = acc;
            acc += code_tot[c];
        }
    }
}

template <int kCodes>
__global__ void __launch_bounds__(kScanThreads) super_add_kernel(unsigned long long* __restrict__ super,
                                                                 unsigned long long nsb,
                                                                 const unsigned long long* __restrict__ chunk_tot) {
    const unsigned long long s = (unsigned long long)blockIdx.x * kScanThreads + threadIdx.x;
    if (s >= nsb) return;
#pragma unroll
    for (int c = 0; c < kCodes; ++c) super[kCodes * s + c] += chunk_tot[(unsigned long long)kCodes * blockIdx.x + c];
}

// The same in one CTA for a few superblocks: each thread takes a contiguous
// range, sums it per code, the CTA scans the sums and each thread writes
// its range's prefixes.
constexpr uint64_t kSmallScan = 8 * kScanThreads;

template <int kCodes>
__global__ void __launch_bounds__(kScanThreads) super_scan_small_kernel(const uint32_t* __restrict__ sb_tot,
                                                                        unsigned long long nsb,
                                                                        unsigned long long* __restrict__ super,
                                                                        unsigned long long* __restrict__ C,
                                                                        unsigned long long m) {
    __shared__ unsigned long long code_tot[kCodes];
    const unsigned long long per = (nsb + kScanThreads - 1) / kScanThreads;
    const unsigned long long s0 = min(nsb, (unsigned long long)threadIdx.x * per), s1 = min(nsb, s0 + per);
    unsigned long long run[kCodes];
#pragma unroll
    for (int c = 0; c < kCodes; ++c) run[c] = 0;
    for (unsigned long long s = s0; s < s1; ++s) {
#pragma unroll
        for (int c = 0; c < kCodes; ++c) run[c] += sb_tot[kCodes * s + c];
    }
#pragma unroll
    for (int c = 0; c < kCodes; ++c) {
        unsigned long long tot;
        run[c] = cta_exclusive_scan<SumOp, kScanThreads>(run[c], tot);
        if (threadIdx.x == 0) code_tot[c] = tot;
    }
    for (unsigned long long s = s0; s < s1; ++s) {
#pragma unroll
        for (int c = 0; c < kCodes; ++c) {
            super[kCodes * s + c] = run[c];
            run[c] += sb_tot[kCodes * s + c];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = m;
        for (int c = 0; c < kCodes; ++c) {
            C[c] = acc;
            acc += code_tot[c];
        }
    }
}

template <int kCodes>
void super_scan(Launcher& L, const uint32_t* sb_tot, uint64_t nsb, unsigned long long* super, unsigned long long* C,
                uint64_t m, unsigned long long* chunk_tot) {
    if (nsb <= kSmallScan) {
        SBWT_LAUNCH(L, "super_scan", (4.0 + 8.0) * kCodes * nsb, 0, nullptr, super_scan_small_kernel<kCodes>, 1,
                    kScanThreads, 0, sb_tot, (unsigned long long)nsb, super, C, (unsigned long long)m);
        return;
    }
    const unsigned nchunks = ceil_div_u(nsb, kScanThreads);
    SBWT_LAUNCH(L, "super_scan", (4.0 + 16.0) * kCodes * nsb, 0, nullptr, super_local_kernel<kCodes>, nchunks,
                kScanThreads, 0, sb_tot, (unsigned long long)nsb, super, chunk_tot);
    SBWT_LAUNCH(L, "super_scan", 16.0 * kCodes * nchunks, 0, nullptr, super_chunks_kernel<kCodes>, 1, kScanThreads, 0,
                chunk_tot, (unsigned long long)nchunks, C, (unsigned long long)m);
    SBWT_LAUNCH(L, "super_scan", (16.0 + 8.0) * kCodes * nsb, 0, nullptr, super_add_kernel<kCodes>, nchunks,
                kScanThreads, 0, super, (unsigned long long)nsb, chunk_tot);
}

}  // namespace

// Old blocks a chunk can read: the chunk's rows in blocks plus a few; a
// dictionary smaller than a chunk needs only its own blocks.
uint64_t insert_stage_blocks(int code_bits, int occ_k, uint64_t n_final) {
    const uint64_t chunk = code_bits == 4 ? kStageBlocksW : (uint64_t)kStageSupers * kBlocksPerSuper / occ_k;
    return std::min<uint64_t>(chunk, dict_blocks(n_final, occ_k)) + 8;
}

template <class IdxT>
void launch_insert(Launcher& L, const void* old_blocks, uint64_t n_ext, const uint8_t* bint, const IdxT* gsa,
                   uint64_t n_int, const uint32_t* ins_i0, void* new_blocks, unsigned long long* new_super,
                   unsigned long long* new_C, uint64_t m_new, uint32_t* sb_tot, uint32_t* d_err, int code_bits,
                   int occ_k, unsigned long long* stage, uint64_t stage_blocks, int insert_threads) {
    const uint64_t n_new = n_ext + n_int;
    // the superblock scan's per-chunk totals live after the superblock totals
    const uint64_t nsb_all = dict_supers_of(n_new, code_bits);
    unsigned long long* chunk_tot =
        reinterpret_cast<unsigned long long*>(sb_tot + ((nsb_all * dict_codes(code_bits) + 3) & ~3ull));
    if (code_bits == 4) {
        const uint64_t nsb = dict_supers_w(n_new);
        const uint64_t nb_all = nsb * kBlocksPerSuperW;  // output blocks the grid covers
        const auto* old_b = static_cast<const OccBlockW*>(old_blocks);
        auto* new_b = static_cast<OccBlockW*>(new_blocks);
        if (!stage) {
            const double bytes = 64.0 * dict_blocks(n_ext) + (1.0 + sizeof(IdxT)) * n_int + 64.0 * dict_blocks(n_new);
            SBWT_LAUNCH(L, "insert_merge", bytes, 0, nullptr, insert_w_kernel<IdxT>, ceil_div_u(nb_all, kThreads),
                        kThreads, 0, old_b, (unsigned long long)n_ext, bint, gsa, (unsigned long long)n_int, new_b,
                        (unsigned long long)n_new, (unsigned long long)nsb, sb_tot, d_err, 0ull, 0, 0ull);
        } else {
            // in place, from the top down in chunks of kStageBlocksW output
            // blocks (a multiple of the CTA's blocks), as for 2-bit codes
            const uint64_t top = (nb_all + kThreads - 1) / kThreads * kThreads;
            for (uint64_t b1 = top; b1 > 0;) {
                const uint64_t b0 = b1 > kStageBlocksW ? b1 - kStageBlocksW : 0;
                SBWT_LAUNCH(L, "insert_stage", 128.0 * (b1 - b0), 0, nullptr, stage_old_w_kernel<IdxT>, kStageGrid,
                            kThreads, 0, old_b, (unsigned long long)n_ext, gsa, (unsigned long long)n_int,
                            (unsigned long long)b0, (unsigned long long)b1, reinterpret_cast<OccBlockW*>(stage),
                            (unsigned long long)stage_blocks, d_err);
                SBWT_LAUNCH(L, "insert_merge", 128.0 * (b1 - b0), 0, nullptr, insert_w_kernel<IdxT>,
                            (unsigned)((b1 - b0) / kThreads), kThreads, 0, reinterpret_cast<const OccBlockW*>(stage),
                            (unsigned long long)n_ext, bint, gsa, (unsigned long long)n_int, new_b,
                            (unsigned long long)n_new, (unsigned long long)nsb, sb_tot, d_err, (unsigned long long)b0,
                            1, (unsigned long long)stage_blocks);
                b1 = b0;
            }
        }
        super_scan<kSigmaW>(L, sb_tot, nsb, new_super, new_C, m_new, chunk_tot);
        return;
    }
    const uint64_t nsb = dict_supers(n_new);
    const double bb = (double)dict_block_bytes(2, occ_k);
    // Dense new rows (a quarter of the result or more): 512 threads, so the
    // runs of new symbols spread over more threads.  Sparse: 256 threads of
    // four parts each, so more CTAs (superblocks) are resident per SM and
    // their load latencies overlap.
    const bool dense = insert_threads ? insert_threads == kInsertThreads : 4 * n_int >= n_new;
    const int threads = dense ? kInsertThreads : kInsertThreadsSparse;
    auto* const kern = dense ? (occ_k == 4 ? insert_kernel<IdxT, kInsertThreads, 4>
                                           : (occ_k == 2 ? insert_kernel<IdxT, kInsertThreads, 2>
                                                         : insert_kernel<IdxT, kInsertThreads, 1>))
                             : (occ_k == 4 ? insert_kernel<IdxT, kInsertThreadsSparse, 4>
                                           : (occ_k == 2 ? insert_kernel<IdxT, kInsertThreadsSparse, 2>
                                                         : insert_kernel<IdxT, kInsertThreadsSparse, 1>));
    const auto* old_w = static_cast<const unsigned long long*>(old_blocks);
    auto* new_w = static_cast<unsigned long long*>(new_blocks);
    if (!stage) {
        const double bytes = bb * dict_blocks(n_ext, occ_k) + (1.0 + sizeof(IdxT)) * n_int +
                             bb * dict_blocks(n_new, occ_k) + 4.0 * (nsb + 1);
        SBWT_LAUNCH(L, "insert_merge", bytes, 0, nullptr, kern, (unsigned)nsb, threads, 0, old_w,
                    (unsigned long long)n_ext, bint, gsa, (unsigned long long)n_int, ins_i0, new_w,
                    (unsigned long long)n_new, sb_tot, d_err, 0ull, 0, 0ull);
    } else {
        // In place (the host tier keeps one dictionary): superblocks from the
        // top down in chunks of kStageSupers; each chunk first copies the old
        // blocks it reads to the staging buffer.  A chunk's old rows all lie
        // below its first output row (new rows only push old rows up), so
        // the chunks above it never overwrite them before they are staged.
        auto* const stage_kern = occ_k == 4 ? stage_old_kernel<4> : (occ_k == 2 ? stage_old_kernel<2>
                                                                                 : stage_old_kernel<1>);
        for (uint64_t s1 = nsb; s1 > 0;) {
            const uint64_t s0 = s1 > kStageSupers ? s1 - kStageSupers : 0;
            const double rows = (double)(s1 - s0) * (1 << kSuperShift);
            SBWT_LAUNCH(L, "insert_stage", 2.0 * rows / (64.0 * occ_k) * bb, 0, nullptr, stage_kern, kStageGrid,
                        kThreads, 0, old_w, (unsigned long long)n_ext, ins_i0, (unsigned long long)s0,
                        (unsigned long long)s1, stage, (unsigned long long)stage_blocks, d_err);
            SBWT_LAUNCH(L, "insert_merge", 2.0 * rows / (64.0 * occ_k) * bb + (1.0 + sizeof(IdxT)) * rows *
                                              ((double)n_int / (double)n_new), 0, nullptr, kern, (unsigned)(s1 - s0),
                        threads, 0, stage, (unsigned long long)n_ext, bint, gsa, (unsigned long long)n_int, ins_i0,
                        new_w, (unsigned long long)n_new, sb_tot, d_err, (unsigned long long)s0, 1,
                        (unsigned long long)stage_blocks);
            s1 = s0;
        }
    }
    super_scan<4>(L, sb_tot, nsb, new_super, new_C, m_new, chunk_tot);
}

template void launch_insert<uint32_t>(Launcher&, const void*, uint64_t, const uint8_t*, const uint32_t*, uint64_t,
                                      const uint32_t*, void*, unsigned long long*, unsigned long long*, uint64_t,
                                      uint32_t*, uint32_t*, int, int, unsigned long long*, uint64_t, int);
template void launch_insert<unsigned long long>(Launcher&, const void*, uint64_t, const uint8_t*,
                                                const unsigned long long*, uint64_t, const uint32_t*, void*,
                                                unsigned long long*, unsigned long long*, uint64_t, uint32_t*,
                                                uint32_t*, int, int, unsigned long long*, uint64_t, int);

}  // namespace sbwt
