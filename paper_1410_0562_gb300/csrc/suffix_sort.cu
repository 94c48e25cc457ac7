// suffix_sort.cu -- ConstructSA of one block (Algorithm 1; Section 3 of
// arXiv 1410.0562 asks for any suffix sort and uses an MSD radix sort over
// packed symbols that sieves out finished suffixes).  Here: an MSD bucket
// split, CTA-local sorts of the buckets, then prefix doubling whose rounds are
// again CTA-local wherever a group fits one CTA.
//
// Suffix order (Section 2): symbols compare by code; a suffix that reaches
// its terminator first is smaller; two suffixes that reach their terminators
// at the same offset compare by read index ($_j order), which inside a block
// is the order of their text positions.
//
// Key of the suffix at block position t: its first 29 codes, MSB first, with
// codes at and past its terminator zeroed, then min(len, 29) in the low 5
// bits, len = distance to the terminator.  Equal keys with len < 29 end at
// the same offset, so ordered by t they are in read order: each is a
// finished singleton.  Keys with len >= 29 that are equal form the unsorted
// groups.  rank[t] is the row of the first member of t's group (the
// Larsson-Sadakane convention), so ranks stay valid while groups split.
//
// 1. Bucket split.  The bucket of a suffix is (p, l): p its first P codes
//    (zeroed past the terminator), l = min(len, P).  Ordered by (p, l) the
//    buckets are ordered like the keys, and the valid pairs are numbered
//    densely (the digit below): P = 11 fits 24 bits.
//    A stable LSD sort of (digit, t) on those bits partitions the block into
//    buckets, each in t order; a bucket's rows are final.  A suffix with
//    len < P (a "short" one) is alone in a bucket of equal keys: it is
//    finished where it lands.
// 2. Units.  The digit-sorted array is cut into windows of kWindow rows; unit
//    w is every bucket that starts inside window w.  A unit holds whole
//    buckets, so its rows are final as a set, and as long as its buckets are
//    at most kWindow long it holds at most 2 kWindow = kLCap rows.
// 3. Local sort of every unit with at most kLCap long suffixes: each bucket
//    is sorted by (key, t), and SA, rank and the unit's still-unsorted
//    members (in row order, in place in the unit's own range of loc_act)
//    are written.  One warp per unit does it in chunks of whole buckets of
//    at most kWChunk rows, with no CTA barrier; a unit with a longer bucket
//    is left to a CTA-batch kernel (counting for buckets of at most kSeg, a
//    merge sort of the batch otherwise).  A unit with more long suffixes
//    goes to the global path: its suffixes (with their rows) are gathered
//    into one list that the device-wide radix sort orders by the full key.
// 4. Round with offset h (29, 58, ...): each unsorted member t is re-sorted
//    inside its group by rank[t + h]; t + h never leaves the read because an
//    unsorted member has len >= h.  All next-ranks are read before any rank
//    of the round is written (a separate gather launch).  Unit-local groups:
//    the unit's members are sorted by (rank[t], rank[t + h]), by one warp
//    when they fit one chunk, else in a CTA batch; a group whose head row is
//    H keeps rows H .. H + size - 1.  Groups from the
//    global path: one device-wide radix sort of all of them by the same pair,
//    as one list, so the k-th sorted element goes to the k-th active row.
//    Rounds continue until the resolved prefix exceeds the longest read of
//    the block.
// At the end rank[] is the inverse suffix array of the block.
#include <algorithm>

#include "sbwt_internal.cuh"
#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kH0 = 29;
constexpr int kGItems = 16;
constexpr int kGTile = kThreads * kGItems;  // elements per group-kernel tile
constexpr unsigned kMaxGroupChunks = 2048;

// CTA-batch local sorts (the units the warp kernels leave): kLThreads x
// kLItems pairs per CTA, four CTAs per SM.
constexpr int kLThreads = 256;
constexpr int kLItems = 8;
constexpr uint32_t kLCap = kLThreads * kLItems;  // 2048 long suffixes per unit at most
constexpr uint32_t kWindow = kLCap / 2;          // rows per window
constexpr uint32_t kLSlots = kLCap + kLCap / kLItems;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kFallback = 0xFFFFFFFEu;  // u.cnt of a unit the warp local sort left to the CTA one
constexpr uint32_t kShortFlag = 0x80000000u;  // digit flag: the bucket holds suffixes with len < P
constexpr int kScanThreads = 1024;  // the unit scan: one CTA, kScanPer windows per thread
// Buckets: the first P codes and min(len, P); their dense numbers need
// kDigitBits bits (5,592,405 valid pairs for 11 two-bit codes, 1,118,481 for
// 5 four-bit codes).  Two long suffixes share a bucket iff their keys agree
// above kBucketShift.
constexpr int kDigitBits = 24;
constexpr uint32_t kDigitMask = (1u << kDigitBits) - 1;
constexpr int kBucketShift = 41;

// Unit table: one entry per window of kWindow rows of the digit-sorted
// array, stored as one array per field so a scan over windows reads it with
// vector loads.  Unit w is every bucket that starts inside window w.
struct Units {
    uint32_t* beg;    // first bucket start in the window (kNone: no unit starts here)
    uint32_t* lcb;    // long suffixes in the window before beg
    uint32_t* lct;    // long suffixes in the window
    uint32_t* end;    // end of the unit (first row of the next unit)
    uint32_t* nlong;  // long suffixes in the unit (during the scan: in the block before beg)
    uint32_t* lofs;   // offset of the unit in the global-path list, kNone for a local unit
    uint32_t* cnt;    // unsorted members of a local unit: loc_act[beg .. beg + cnt)
    uint32_t* owner;  // the unit whose rows include the window's first row
};
constexpr int kUnitFields = 8;
// words per field: every field starts on a 32-byte boundary
inline uint64_t unit_stride(uint64_t cap) { return (cap / kWindow + 2 + 7) & ~7ull; }
inline Units units_at(void* base, uint64_t cap) {
    uint32_t* p = static_cast<uint32_t*>(base);
    const uint64_t s = unit_stride(cap);
    return Units{p, p + s, p + 2 * s, p + 3 * s, p + 4 * s, p + 5 * s, p + 6 * s, p + 7 * s};
}

// Key geometry per code width kB (2 bits for up to 4 symbols, 4 bits for 5
// to 16): H codes in the key (H kB <= 58 bits) and buckets of P codes (for
// 4-bit codes P is the smallest bucket length, for 16 symbols; fewer
// symbols take longer buckets, chosen per index), digits of 24 bits.
template <int kB>
struct KeyGeom {
    static constexpr uint32_t H = kB == 2 ? 29 : 14;
    static constexpr uint32_t P = kB == 2 ? 11 : 5;
    static constexpr uint32_t CB = H * kB;           // code bits of a key
    static constexpr int kLog = kB == 2 ? 4 : 3;     // log2 of codes per text word
    static_assert(H <= kH0, "length field");
};

// The length field of a key: min(len, H), except that a suffix reaching at
// least H codes stores kH0 — so "terminated inside the key" is field < kH0
// for either width, and the order of keys is unchanged.
template <int kB>
__device__ __forceinline__ uint32_t len_field(uint32_t len) {
    return len < KeyGeom<kB>::H ? len : kH0;
}

// The key's H codes from the three text words w0 w1 w2 that hold position
// P, with the codes at and past the terminator zeroed.
template <int kB>
__device__ __forceinline__ unsigned long long key_codes(uint32_t w0, uint32_t w1, uint32_t w2, uint64_t P,
                                                        uint32_t field) {
    using G = KeyGeom<kB>;
    const uint32_t s = kB * (uint32_t)(P & ((1u << G::kLog) - 1));
    const unsigned long long hi = ((unsigned long long)w0 << 32) | w1;
    const unsigned long long v = (hi << s) | (((unsigned long long)w2 << s) >> 32);  // codes from P, MSB first
    unsigned long long k = v >> (64 - G::CB);
    if (field < G::H) k &= ~((1ull << (kB * (G::H - field))) - 1ull);
    return (k << 5) | field;
}

template <int kB>
__device__ __forceinline__ unsigned long long initial_key(const uint32_t* __restrict__ text,
                                                          const uint32_t* __restrict__ term, uint64_t P) {
    using G = KeyGeom<kB>;
    // distance to the terminator, capped at H (terminator bitmap window)
    const uint64_t tw = P >> 5;
    const unsigned long long tb = (((unsigned long long)term[tw + 1] << 32) | term[tw]) >> (P & 31);
    const unsigned long long near = tb & ((1ull << G::H) - 1);
    const uint32_t len = near ? (uint32_t)(__ffsll((long long)near) - 1) : G::H;
    const uint64_t wi = P >> G::kLog;
    return key_codes<kB>(text[wi], text[wi + 1], text[wi + 2], P, len_field<kB>(len));
}

// The same key when its length field is known: only the text window is
// read, as one 16-byte load (plus 8 bytes when the three words cross it; the
// text array starts on a 16-byte boundary and carries 4 padding words).
template <int kB>
__device__ __forceinline__ unsigned long long key_with_len(const uint32_t* __restrict__ text, uint64_t P,
                                                           uint32_t field) {
    const uint64_t wi = P >> KeyGeom<kB>::kLog;
    const uint32_t q = (uint32_t)(wi & 3);
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(text + (wi - q)));
    uint2 b = make_uint2(0u, 0u);
    if (q >= 2) b = __ldg(reinterpret_cast<const uint2*>(text + (wi - q) + 4));
    uint32_t w0, w1, w2;
    if (q == 0) {
        w0 = a.x, w1 = a.y, w2 = a.z;
    } else if (q == 1) {
        w0 = a.y, w1 = a.z, w2 = a.w;
    } else if (q == 2) {
        w0 = a.z, w1 = a.w, w2 = b.x;
    } else {
        w0 = a.w, w1 = b.x, w2 = b.y;
    }
    return key_codes<kB>(w0, w1, w2, P, field);
}

// Dense number of the bucket (p, l) of key K among all valid pairs in (p, l)
// order, P = 11 two-bit codes.  A pair is valid when the codes of p at and
// past l are zero.  Pairs before (p, l): the p pairs (p' < p, l' = P); for
// each l' < P the multiples of 4^(P - l') below p (short pairs with p' < p),
// in all sum_{k=1..P} ceil(p / 4^k), which for p >= 1 is P + sum_k
// floor((p-1) / 4^k) = P + ((p-1) - s4(p-1)) / 3 with s4 the base-4 digit
// sum (Legendre's formula); and the short pairs (p, l') with l' < l, i.e.
// those whose zero tail p has.  Bit 31 flags a short bucket.
__device__ __forceinline__ uint32_t bucket_digit(unsigned long long K) {
    using G = KeyGeom<2>;
    constexpr uint32_t pc = G::P;
    const uint32_t l = min((uint32_t)(K & 31), pc);
    const uint32_t p = (uint32_t)((K >> 5) >> (G::CB - 2 * pc));
    const uint32_t zero_codes = p ? (uint32_t)(__ffs(p) - 1) >> 1 : pc;
    uint32_t o = p;
    if (p) {
        const uint32_t x = p - 1;
        const uint32_t s4 = (uint32_t)__popc(x & 0x55555555u) + 2u * (uint32_t)__popc(x & 0xAAAAAAAAu);
        o += pc + (x - s4) / 3;
    }
    const uint32_t first_valid = pc > zero_codes ? pc - zero_codes : 0;
    o += l > first_valid ? l - first_valid : 0;
    return o | (l < pc ? kShortFlag : 0u);
}

// The bucket number for 4-bit codes of an alphabet of sigma symbols, in
// base sigma so that the pairs are as dense as for 2-bit codes: buckets of
// the first pw codes (pw chosen on the host so that every valid pair fits
// kDigitBits bits).  With p the pw codes read as a base-sigma number, s(p)
// their digit sum and z the zero codes at the end of p, the count of pairs
// before (p, l) above becomes, for p >= 1, p + pw + (p - s(p)) / (sigma - 1)
// - z, since s(p - 1) = s(p) - 1 + z (sigma - 1); plus the short pairs
// (p, l') with pw - z <= l' < l.
__device__ __forceinline__ uint32_t bucket_digit_sigma(unsigned long long K, uint32_t sigma, uint32_t pw) {
    using G = KeyGeom<4>;
    const uint32_t l = min((uint32_t)(K & 31), pw);
    const unsigned long long codes = (K >> 5) >> (G::CB - 4 * pw);  // the first pw codes
    uint32_t p = 0, s = 0;
    for (uint32_t q = 0; q < pw; ++q) {
        const uint32_t c = (uint32_t)(codes >> (4 * (pw - 1 - q))) & 15u;
        p = p * sigma + c;
        s += c;
    }
    const uint32_t z = codes ? (uint32_t)(__ffsll((long long)codes) - 1) / 4 : pw;
    uint32_t o = p;
    if (p) o += pw + (p - s) / (sigma - 1) - z;
    const uint32_t first_valid = pw > z ? pw - z : 0;
    o += l > first_valid ? l - first_valid : 0;
    return o | (l < pw ? kShortFlag : 0u);
}

// Element of block position t for the bucket split: its bucket digit (bits
// 0..23, bit 31 the short flag) and the key's length field (bits 24..28) in
// the low word, t in the high word.  The sort orders by the low kDigitBits bits and
// carries the rest.
constexpr int kKeyThreads = 512;  // threads of a sa_digit_keys CTA (one radix chunk)

template <int kB>
__global__ void __launch_bounds__(kKeyThreads) sa_digit_keys_kernel(const uint32_t* __restrict__ text,
                                                                 const uint32_t* __restrict__ term,
                                                                 unsigned long long base, uint32_t n,
                                                                 uint32_t sigma, uint32_t pw,
                                                                 unsigned long long* __restrict__ elems,
                                                                 uint32_t* __restrict__ d_n,
                                                                 uint32_t* __restrict__ counts,
                                                                 uint32_t* __restrict__ totals) {
    static_assert(kKeyThreads % kRadixBins == 0, "whole digit sets per thread group");
    __shared__ uint32_t h[kKeyThreads / 32][kRadixBins];
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = n;
    uint32_t tile0, tile1;
    radix_chunk_tiles(n, gridDim.x, blockIdx.x, tile0, tile1);
    if (tile0 >= tile1) return;
    for (int i = threadIdx.x; i < (kKeyThreads / 32) * kRadixBins; i += kKeyThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    uint32_t* my = h[threadIdx.x >> 5];
    const uint32_t t_end = (uint32_t)min((uint64_t)n, (uint64_t)tile1 * kRadixTile);
#pragma unroll 4
    for (uint32_t t = tile0 * kRadixTile + threadIdx.x; t < t_end; t += kKeyThreads) {
        const unsigned long long K = initial_key<kB>(text, term, base + t);
        uint32_t d;
        if constexpr (kB == 2) {
            d = bucket_digit(K);
        } else {
            d = bucket_digit_sigma(K, sigma, pw);
        }
        elems[t] = d | ((uint32_t)(K & 31) << 24) | ((unsigned long long)t << 32);
        atomicAdd(&my[d & (kRadixBins - 1)], 1u);
    }
    __syncthreads();
    // the first radix pass's counts of this chunk (digit bits 0..7)
    if (threadIdx.x < kRadixBins) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kKeyThreads / 32; ++w) c += h[w][threadIdx.x];
        counts[(uint64_t)blockIdx.x * kRadixBins + threadIdx.x] = c;
        if (c) atomicAdd(&totals[threadIdx.x], c);
    }
}

// One warp per window of the digit-sorted array: the first bucket start in
// the window and the long-suffix counts before it and in the whole window.
// Short suffixes are finished where they landed: SA and rank are written
// here.  The k-th long row i of window w, suffix t, is listed as (ll_t,
// ll_row, ll_key)[w kWindow + k] = (t, i, its key), so a unit's long rows
// are a few contiguous runs.
template <int kB>
__global__ void __launch_bounds__(kThreads) sa_unit_begin_kernel(const uint32_t* __restrict__ text,
                                                                 unsigned long long base,
                                                                 const unsigned long long* __restrict__ elems,
                                                                 uint32_t n, uint32_t nwin, Units u,
                                                                 uint32_t* __restrict__ sa,
                                                                 uint32_t* __restrict__ rank,
                                                                 uint32_t* __restrict__ ll_t,
                                                                 uint32_t* __restrict__ ll_row,
                                                                 unsigned long long* __restrict__ ll_key,
                                                                 uint32_t* __restrict__ d_err) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (kThreads / 32);
    for (uint32_t w = (blockIdx.x * kThreads + threadIdx.x) >> 5; w < nwin; w += warps) {
        const uint32_t lo = w * kWindow, hi = min(n, lo + kWindow);
        uint32_t first = kNone, lcb = 0, lct = 0;
        for (uint32_t b = lo; b < hi; b += 32) {
            const uint32_t i = b + lane;
            const bool valid = i < hi;
            const unsigned long long e = valid ? elems[i] : 0ull;
            const uint32_t d = (uint32_t)e;
            const uint32_t prev = (valid && i > 0) ? (uint32_t)elems[i - 1] : d;
            const uint32_t len = (d >> 24) & 31u;
            const uint32_t t = (uint32_t)(e >> 32);
            const bool bnd = valid && (i == 0 || ((d ^ prev) & kDigitMask) != 0);
            const bool lng = valid && !(d & kShortFlag);
            const uint32_t bb = __ballot_sync(0xffffffffu, bnd), bl = __ballot_sync(0xffffffffu, lng);
            if (valid && t >= n) atomicOr(d_err, 64u);
            if (valid && !lng && t < n) {
                sa[i] = t;
                rank[t] = i;
            }
            if (lng) {
                const uint32_t k = lo + lct + __popc(bl & ((1u << lane) - 1u));
                ll_t[k] = t;
                ll_row[k] = i;
                ll_key[k] = key_with_len<kB>(text, base + (t < n ? t : 0u), len);
            }
            if (first == kNone) {
                if (bb) {
                    const int fb = __ffs(bb) - 1;
                    first = b + fb;
                    lcb += __popc(bl & ((1u << fb) - 1u));
                } else {
                    lcb += __popc(bl);
                }
            }
            lct += __popc(bl);
        }
        if (lane == 0) {
            u.beg[w] = first;
            u.lcb[w] = lcb;
            u.lct[w] = lct;
        }
    }
}

// kScanPer consecutive windows of one field (vector accesses when whole)
constexpr int kScanPer = 8;
static_assert(kScanPer % 4 == 0, "whole 16-byte vectors");
__device__ __forceinline__ void load_run(const uint32_t* p, uint32_t w0, uint32_t nwin, uint32_t fill,
                                         uint32_t (&v)[kScanPer]) {
    if (w0 + kScanPer <= nwin) {
#pragma unroll
        for (int q = 0; q < kScanPer; q += 4) {
            const uint4 a = *reinterpret_cast<const uint4*>(p + w0 + q);
            v[q] = a.x, v[q + 1] = a.y, v[q + 2] = a.z, v[q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) v[q] = w0 + q < nwin ? p[w0 + q] : fill;
    }
}
__device__ __forceinline__ void store_run(uint32_t* p, uint32_t w0, uint32_t nwin, const uint32_t (&v)[kScanPer]) {
    if (w0 + kScanPer <= nwin) {
#pragma unroll
        for (int q = 0; q < kScanPer; q += 4)
            *reinterpret_cast<uint4*>(p + w0 + q) = make_uint4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < kScanPer; ++q)
            if (w0 + q < nwin) p[w0 + q] = v[q];
    }
}

// One CTA over all windows, kScanPer consecutive windows per thread: unit
// ends, long counts, owners, and the offsets of the units that take the
// global path.  Also zeroes the per-round counts of local unsorted members
// (zero_slots[k * zero_stride], k < nzero) and the per-round counts of units
// left to the CTA kernel (left_slots[k], k < nleft).
constexpr uint32_t kScanSpan = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) sa_unit_scan_kernel(Units u, uint32_t nwin, uint32_t n,
                                                                    uint32_t* __restrict__ d_large_n,
                                                                    uint32_t* __restrict__ zero_slots, int nzero,
                                                                    int zero_stride,
                                                                    uint32_t* __restrict__ left_slots, int nleft) {
    __shared__ unsigned long long xch[kScanThreads];
    if ((int)threadIdx.x < nzero) zero_slots[threadIdx.x * zero_stride] = 0;
    if ((int)threadIdx.x < nleft) left_slots[threadIdx.x] = 0;
    // forward: long suffixes in the block before each unit start (kept in
    // nlong until the backward pass), owner of each window's first row
    uint32_t carry_sum = 0, carry_last = 0;  // carry_last: 1 + index of the last unit so far
    for (uint32_t base = 0; base < nwin; base += kScanSpan) {
        const uint32_t w0 = base + threadIdx.x * kScanPer;
        uint32_t beg[kScanPer], lcb[kScanPer], lct[kScanPer], g[kScanPer], own[kScanPer];
        load_run(u.beg, w0, nwin, kNone, beg);
        load_run(u.lcb, w0, nwin, 0u, lcb);
        load_run(u.lct, w0, nwin, 0u, lct);
        uint32_t sum = 0, last = 0;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            sum += lct[q];
            if (beg[q] != kNone) last = w0 + q + 1;
        }
        uint32_t tot, mtot;
        uint32_t run = carry_sum + cta_exclusive_scan<SumOp, kScanThreads>(sum, tot);
        uint32_t run_last = max(carry_last, cta_exclusive_scan<MaxOp, kScanThreads>(last, mtot));
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            const uint32_t w = w0 + q;
            const bool ne = beg[q] != kNone;
            g[q] = ne ? run + lcb[q] : 0u;
            own[q] = (ne && beg[q] == w * kWindow) ? w : run_last - 1;  // window 0 always starts a unit
            run += lct[q];
            if (ne) run_last = w + 1;
        }
        if (w0 < nwin) {
            store_run(u.nlong, w0, nwin, g);
            store_run(u.owner, w0, nwin, own);
        }
        carry_sum += tot;
        carry_last = max(carry_last, mtot);
    }
    const uint32_t total_long = carry_sum;
    __syncthreads();
    // backward, chunks from the last: the next unit's (start, long prefix)
    // gives each unit's end and long count.  The minimum over later threads
    // is an exclusive scan in reversed thread order.
    unsigned long long carry = ~0ull;
    const uint32_t nchunks = (nwin + kScanSpan - 1) / kScanSpan;
    for (uint32_t ci = nchunks; ci-- > 0;) {
        const uint32_t w0 = ci * kScanSpan + threadIdx.x * kScanPer;
        uint32_t beg[kScanPer], g[kScanPer], end[kScanPer], nl[kScanPer];
        load_run(u.beg, w0, nwin, kNone, beg);
        load_run(u.nlong, w0, nwin, 0u, g);
        unsigned long long mine = ~0ull;
#pragma unroll
        for (int q = kScanPer - 1; q >= 0; --q)
            if (beg[q] != kNone) mine = ((unsigned long long)beg[q] << 32) | g[q];
        xch[threadIdx.x] = mine;
        __syncthreads();
        unsigned long long tot;
        const unsigned long long rex =
            cta_exclusive_scan<MinOp, kScanThreads>(xch[kScanThreads - 1 - threadIdx.x], tot);
        __syncthreads();
        xch[kScanThreads - 1 - threadIdx.x] = rex;  // min over the threads after that one
        __syncthreads();
        unsigned long long nx = min(carry, xch[threadIdx.x]);
#pragma unroll
        for (int q = kScanPer - 1; q >= 0; --q) {
            end[q] = 0;
            nl[q] = 0;
            if (beg[q] != kNone) {
                end[q] = nx == ~0ull ? n : (uint32_t)(nx >> 32);
                nl[q] = (nx == ~0ull ? total_long : (uint32_t)nx) - g[q];
                nx = ((unsigned long long)beg[q] << 32) | g[q];
            }
        }
        if (w0 < nwin) {
            store_run(u.end, w0, nwin, end);
            store_run(u.nlong, w0, nwin, nl);
        }
        carry = min(carry, tot);
        __syncthreads();
    }
    __syncthreads();
    // forward: offsets of the global-path units
    uint32_t lcarry = 0;
    for (uint32_t base = 0; base < nwin; base += kScanSpan) {
        const uint32_t w0 = base + threadIdx.x * kScanPer;
        uint32_t beg[kScanPer], end[kScanPer], nl[kScanPer], lofs[kScanPer], zero[kScanPer], sum = 0;
        load_run(u.beg, w0, nwin, kNone, beg);
        load_run(u.end, w0, nwin, 0u, end);
        load_run(u.nlong, w0, nwin, 0u, nl);
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            const bool big = beg[q] != kNone && nl[q] > kLCap;
            lofs[q] = big ? end[q] - beg[q] : 0u;  // size for now
            sum += lofs[q];
            zero[q] = 0;
        }
        uint32_t tot;
        uint32_t run = lcarry + cta_exclusive_scan<SumOp, kScanThreads>(sum, tot);
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            const uint32_t size = lofs[q];
            lofs[q] = size ? run : kNone;
            run += size;
        }
        if (w0 < nwin) {
            store_run(u.lofs, w0, nwin, lofs);
            store_run(u.cnt, w0, nwin, zero);
        }
        lcarry += tot;
    }
    if (threadIdx.x == 0) *d_large_n = lcarry;
}

// one spare slot per kLItems: blocked accesses (thread x, item j at
// kLItems x + j) then fall into distinct banks
__device__ __forceinline__ uint32_t skew(uint32_t i) { return i + i / kLItems; }

// Stable merge sort of `count` <= kLCap (key, value) pairs held blocked in
// registers: thread x holds items kLItems x .. kLItems x + kLItems - 1, and
// every item at or past `count` holds key ~0 (larger than any real key).
// First each thread sorts its items (odd-even transposition, swapping only
// strictly larger keys), then runs of kLItems, 2 kLItems, ... are merged
// pairwise: each thread finds where its kLItems outputs start on the merge
// path (a binary search between the two runs, ties taken from the left run)
// and merges them serially.  skey/sval are kLSlots-entry shared arrays,
// indexed through skew() so blocked accesses do not collide in banks.
__device__ __forceinline__ void block_merge_sort(unsigned long long (&k)[kLItems], uint32_t (&v)[kLItems],
                                                 uint32_t count, unsigned long long* skey, uint32_t* sval) {
#pragma unroll
    for (int r = 0; r < kLItems; ++r) {
#pragma unroll
        for (int j = r & 1; j + 1 < kLItems; j += 2) {
            const unsigned long long ka = k[j], kb = k[j + 1];
            const uint32_t va = v[j], vb = v[j + 1];
            const bool sw = ka > kb;
            k[j] = sw ? kb : ka;
            k[j + 1] = sw ? ka : kb;
            v[j] = sw ? vb : va;
            v[j + 1] = sw ? va : vb;
        }
    }
    const uint32_t base = threadIdx.x * kLItems;
    for (uint32_t w = kLItems; w < count; w <<= 1) {
        __syncthreads();  // the previous pass's readers are done
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            skey[skew(base + j)] = k[j];
            sval[skew(base + j)] = v[j];
        }
        __syncthreads();
        const uint32_t a0 = base & ~(2 * w - 1);  // the pair of runs [a0, a0 + w), [a0 + w, a0 + 2w)
        if (a0 >= count) continue;                // padding only: already in order
        const uint32_t a1 = a0 + w, b0 = a1, b1 = a1 + w;
        const uint32_t d = base - a0;  // this thread's first output within the pair
        uint32_t lo = d > w ? d - w : 0, hi = d < w ? d : w;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (skey[skew(a0 + mid)] <= skey[skew(b0 + d - 1 - mid)]) lo = mid + 1;
            else hi = mid;
        }
        uint32_t ai = a0 + lo, bi = b0 + (d - lo);
        unsigned long long ka = ai < a1 ? skey[skew(ai)] : 0ull;
        unsigned long long kb = bi < b1 ? skey[skew(bi)] : 0ull;
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const bool take_a = ai < a1 && (bi >= b1 || ka <= kb);
            if (take_a) {
                k[j] = ka;
                v[j] = sval[skew(ai)];
                ++ai;
                ka = ai < a1 ? skey[skew(ai)] : 0ull;
            } else {
                k[j] = kb;
                v[j] = sval[skew(bi)];
                ++bi;
                kb = bi < b1 ? skey[skew(bi)] : 0ull;
            }
        }
    }
    __syncthreads();
}

// Running head positions over a sorted CTA list: heads (bit j: item j of
// this thread starts a group) -> for each item the index of its group's first
// item, returned through `first` (the value for item 0; later items update it
// as they meet heads).
__device__ __forceinline__ uint32_t carry_in_head(uint32_t heads, uint32_t g0) {
    const uint32_t last = heads ? g0 + 31 - __clz(heads) : 0u;
    uint32_t tot;
    return cta_exclusive_scan<MaxOp, kLThreads>(last, tot);
}

// Sort of `count` <= kLCap (key, value) pairs held blocked in registers
// (as for block_merge_sort) when the list is cut into segments of equal
// key >> shift, contiguous and in segment order, none longer than kSeg: an
// item's place is its segment's first index plus the number of items of its
// segment before it in (key, value) order (values are distinct, so the order
// is total).  Returns false, with the registers untouched, when a segment is
// longer than kSeg.  On success skey/sval hold the sorted list too.
constexpr uint32_t kSeg = 64;

__device__ __forceinline__ bool block_segment_sort(unsigned long long (&k)[kLItems], uint32_t (&v)[kLItems],
                                                   uint32_t count, unsigned long long* skey, uint32_t* sval,
                                                   uint32_t* sseg, int shift) {
    const uint32_t g0 = threadIdx.x * kLItems;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        skey[skew(g0 + j)] = k[j];
        sval[skew(g0 + j)] = v[j];
    }
    __syncthreads();
    // segment starts, then each segment's end stored at its start
    const unsigned long long kprev = (g0 > 0 && g0 <= count) ? skey[skew(g0 - 1)] : 0ull;
    uint32_t starts = 0;
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        const uint32_t g = g0 + j;
        const unsigned long long pk = j ? k[j - 1] : kprev;
        starts |= (uint32_t)(g < count && (g == 0 || (k[j] >> shift) != (pk >> shift))) << j;
    }
    bool next_start = true;
    if (g0 + kLItems < count) next_start = (skey[skew(g0 + kLItems)] >> shift) != (k[kLItems - 1] >> shift);
    uint32_t s0 = carry_in_head(starts, g0);
    uint32_t pos[kLItems];  // first the segment's first index, then the item's place
    bool big = false;
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        const uint32_t g = g0 + j;
        if ((starts >> j) & 1u) s0 = g;
        pos[j] = s0;
        const bool last = j + 1 < kLItems ? (((starts >> (j + 1)) & 1u) || g + 1 >= count) : next_start;
        if (g < count && last) {
            sseg[skew(s0)] = g + 1;
            big |= g + 1 - s0 > kSeg;
        }
    }
    if (__syncthreads_or(big)) return false;
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        const uint32_t g = g0 + j;
        if (g >= count) continue;
        const uint32_t s1 = sseg[skew(pos[j])];
        uint32_t r = pos[j];
        for (uint32_t x = pos[j]; x < s1; ++x) {
            const unsigned long long kx = skey[skew(x)];
            r += (kx < k[j] || (kx == k[j] && sval[skew(x)] < v[j])) ? 1u : 0u;
        }
        pos[j] = r;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        if (g0 + j < count) {
            skey[skew(pos[j])] = k[j];
            sval[skew(pos[j])] = v[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        if (g0 + j < count) {
            k[j] = skey[skew(g0 + j)];
            v[j] = sval[skew(g0 + j)];
        }
    }
    return true;
}

// Sorts the blocked items by (key, value): segment by segment as above,
// else by a merge sort of the list; leaves the sorted keys in skey.
__device__ __forceinline__ void block_sort(unsigned long long (&k)[kLItems], uint32_t (&v)[kLItems],
                                           uint32_t count, unsigned long long* skey, uint32_t* sval,
                                           uint32_t* sseg, int shift) {
    if (block_segment_sort(k, v, count, skey, sval, sseg, shift)) {
        __syncthreads();
        return;
    }
    block_merge_sort(k, v, count, skey, sval);
#pragma unroll
    for (int j = 0; j < kLItems; ++j) skey[skew(threadIdx.x * kLItems + j)] = k[j];
    __syncthreads();
}

// Batches: a CTA walks its share of the windows, taking each time the
// longest run of windows [w, w + k) whose element counts (c, one window per
// thread; a count above kLCap stops a batch) sum to at most kLCap.  Fills
// b_pref[i] = elements before window w + i in the batch; returns k (0 when
// the first window cannot join a batch) and the batch's element total.
struct Batch {
    uint32_t pref[kLThreads];  // elements before window w + i
    uint32_t beg[kLThreads];   // the unit start of window w + i
    uint32_t abase[kLThreads];  // unsorted members before the window's first slot
    uint32_t acnt[kLThreads];   // unsorted members of the window's unit
    uint32_t misc[4];
};

__device__ __forceinline__ uint32_t form_batch(Batch& b, uint32_t c, uint32_t beg, uint32_t& total) {
    uint32_t tot;
    const uint32_t ex = cta_exclusive_scan<SumOp, kLThreads>(c, tot);
    const uint32_t incl = ex + c;
    const uint32_t k = (uint32_t)__syncthreads_count(incl <= kLCap);
    if (threadIdx.x < k) {
        b.pref[threadIdx.x] = ex;
        b.beg[threadIdx.x] = beg;
        b.acnt[threadIdx.x] = 0;
    }
    if (k && threadIdx.x == k - 1) b.misc[0] = incl;
    __syncthreads();
    total = k ? b.misc[0] : 0u;
    return k;
}

// The batch window of slot g: the last i < k with pref[i] <= g (windows
// with no elements share the next one's prefix, so it is never empty).
__device__ __forceinline__ uint32_t batch_window(const Batch& b, uint32_t k, uint32_t g) {
    uint32_t lo = 0, hi = k - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (b.pref[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Writes the unsorted members (act bit j: item j of this thread) of every
// unit in the batch to its range of loc_act, in sorted order, and sets the
// units' counts.  Items stay inside their unit's slots when sorted.
__device__ __forceinline__ void batch_write_unsorted(Batch& b, uint32_t k, uint32_t w, const uint32_t (&v)[kLItems],
                                                     uint32_t act, uint32_t count, uint32_t* __restrict__ loc_act,
                                                     uint32_t* __restrict__ unit_cnt, uint32_t* __restrict__ d_cnt) {
    const uint32_t g0 = threadIdx.x * kLItems;
    uint32_t atot;
    uint32_t a = cta_exclusive_scan<SumOp, kLThreads>((uint32_t)__popc(act), atot);
    uint32_t wi = g0 < count ? batch_window(b, k, g0) : 0u;
    uint32_t ai = a;
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        const uint32_t g = g0 + j;
        if (g >= count) break;
        while (wi + 1 < k && b.pref[wi + 1] <= g) ++wi;
        if (g == b.pref[wi]) b.abase[wi] = ai;
        if ((act >> j) & 1u) {
            atomicAdd(&b.acnt[wi], 1u);
            ++ai;
        }
    }
    __syncthreads();
    wi = g0 < count ? batch_window(b, k, g0) : 0u;
    ai = a;
#pragma unroll
    for (int j = 0; j < kLItems; ++j) {
        const uint32_t g = g0 + j;
        if (g >= count) break;
        while (wi + 1 < k && b.pref[wi + 1] <= g) ++wi;
        if ((act >> j) & 1u) loc_act[b.beg[wi] + (ai - b.abase[wi])] = v[j];
        ai += (act >> j) & 1u;
    }
    if (threadIdx.x < k) {
        const uint32_t before = threadIdx.x + 1 < k ? b.pref[threadIdx.x + 1] : count;
        if (before > b.pref[threadIdx.x]) unit_cnt[w + threadIdx.x] = b.acnt[threadIdx.x];
    }
    if (threadIdx.x == 0 && atot) atomicAdd(d_cnt, atot);
    __syncthreads();
}

// Local sort of the units with at most kLCap long suffixes, a batch of
// consecutive units per CTA step.  A batch's long rows are the runs
// (ll_t, ll_row, ll_key)[x kWindow + k0 ...) of the windows x = ws, ws + 1, ... from
// its first unit start ws (k0 = lcb in window ws, 0 after), in row order;
// the sorted j-th long suffix takes the j-th of those rows, srow[j].  A
// global-path unit ends a batch and is skipped.
__global__ void __launch_bounds__(kLThreads, 4) sa_local_sort_kernel(
    uint32_t n, const uint32_t* __restrict__ ll_t, const uint32_t* __restrict__ ll_row,
    const unsigned long long* __restrict__ ll_key, Units u, uint32_t nwin, uint32_t* __restrict__ sa,
    uint32_t* __restrict__ rank, uint32_t* __restrict__ loc_act, uint32_t* __restrict__ d_cnt,
    uint32_t* __restrict__ d_err, int seg_shift) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kLSlots);
    uint32_t* srow = sval + kLSlots;
    uint32_t* sseg = srow + kLSlots;
    __shared__ Batch b;
    __shared__ uint32_t run_start[kLThreads], run_src[kLThreads];
    __shared__ uint32_t first_left;

    const uint32_t per = (nwin + gridDim.x - 1) / gridDim.x;
    const uint32_t wbeg = min(nwin, blockIdx.x * per), wend = min(nwin, wbeg + per);
    for (uint32_t w = wbeg; w < wend;) {
        const uint32_t x = w + threadIdx.x;
        // only the units the warp kernel left here (u.cnt = kFallback) are
        // sorted; every other unit ends a batch like a global-path unit
        uint32_t c = kLCap + 1, ub = kNone;
        bool left = false;
        if (x < wend) {
            ub = u.beg[x];
            left = ub != kNone && u.lofs[x] == kNone && u.cnt[x] == kFallback;
            c = ub == kNone ? 0u : (left ? u.nlong[x] : kLCap + 1);
        }
        if (threadIdx.x == 0) first_left = kNone;
        __syncthreads();
        if (left) atomicMin(&first_left, x);
        __syncthreads();
        const uint32_t fl = first_left;
        __syncthreads();  // read by every thread before thread 0 resets it
        if (fl == kNone) {
            w += kLThreads;
            continue;
        }
        if (fl > w) {
            w = fl;
            continue;
        }
        uint32_t total;
        const uint32_t k = form_batch(b, c, ub, total);
        if (k == 0) {
            ++w;
            continue;
        }
        if (total == 0) {
            w += k;
            continue;
        }
        // the batch's first unit start
        if (threadIdx.x == 0) b.misc[1] = kNone;
        __syncthreads();
        if (threadIdx.x < k && ub != kNone) atomicMin(&b.misc[1], x);
        __syncthreads();
        const uint32_t ws = b.misc[1];
        // this thread's slots g0 .. g0 + kLItems - 1 of the batch's long rows:
        // list positions first (the run table is built kLThreads windows at
        // a time), then all loads at once
        const uint32_t g0 = threadIdx.x * kLItems;
        uint32_t src[kLItems];
#pragma unroll
        for (int j = 0; j < kLItems; ++j) src[j] = kNone;
        uint32_t cc = 0;
        for (uint32_t x0 = ws; cc < total && x0 < nwin; x0 += kLThreads) {
            const uint32_t xx = x0 + threadIdx.x;
            const uint32_t k0 = xx == ws ? u.lcb[ws] : 0u;
            const uint32_t avail = xx < nwin ? u.lct[xx] - k0 : 0u;
            uint32_t tot;
            const uint32_t ex = cta_exclusive_scan<SumOp, kLThreads>(avail, tot);
            const uint32_t take = min(tot, total - cc);
            run_start[threadIdx.x] = cc + ex;
            run_src[threadIdx.x] = xx * kWindow + k0;
            const uint32_t nruns = (uint32_t)__syncthreads_count(ex < take);
            if (g0 + kLItems > cc && g0 < cc + take) {
                const uint32_t gs = max(g0, cc);
                uint32_t lo = 0, hi = nruns - 1;  // the last run starting at or before slot gs
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (run_start[mid] <= gs) lo = mid;
                    else hi = mid - 1;
                }
#pragma unroll
                for (int j = 0; j < kLItems; ++j) {
                    const uint32_t g = g0 + j;
                    if (g < cc || g >= cc + take) continue;
                    while (lo + 1 < nruns && run_start[lo + 1] <= g) ++lo;
                    src[j] = run_src[lo] + (g - run_start[lo]);
                }
            }
            cc += take;
            __syncthreads();
        }
        const uint32_t cnt = cc;
        unsigned long long kk[kLItems];
        uint32_t v[kLItems], rw[kLItems];
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            v[j] = src[j] != kNone ? ll_t[src[j]] : 0u;
            rw[j] = src[j] != kNone ? ll_row[src[j]] : 0u;
            kk[j] = src[j] != kNone ? ll_key[src[j]] : ~0ull;
        }
#pragma unroll
        for (int j = 0; j < kLItems; ++j) srow[skew(g0 + j)] = rw[j];  // an out-of-range t is skipped when written
        block_sort(kk, v, cnt, skey, sval, sseg, seg_shift);  // segments: buckets

        // group heads: a new key, or a key that contains its terminator
        const unsigned long long kprev = (g0 > 0 && g0 <= cnt) ? skey[skew(g0 - 1)] : 0ull;
        uint32_t heads = 0;
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const uint32_t g = g0 + j;
            const unsigned long long pk = j ? kk[j - 1] : kprev;
            const bool h = g < cnt && (g == 0 || kk[j] != pk || (uint32_t)(kk[j] & 31) < kH0);
            heads |= (uint32_t)h << j;
        }
        bool next_head = true;
        if (g0 + kLItems < cnt) {
            const unsigned long long kn = skey[skew(g0 + kLItems)];
            next_head = kn != kk[kLItems - 1] || (uint32_t)(kn & 31) < kH0;
        }
        uint32_t first = carry_in_head(heads, g0);
        uint32_t act = 0;
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const uint32_t g = g0 + j;
            if (g >= cnt) break;
            const bool h = (heads >> j) & 1u;
            if (h) first = g;
            const bool e = j + 1 < kLItems ? (((heads >> (j + 1)) & 1u) || g + 1 >= cnt) : next_head;
            const uint32_t row = srow[skew(g)];
            if (row < n && v[j] < n) {
                sa[row] = v[j];
                rank[v[j]] = srow[skew(first)];
            }
            if (!(h && e)) act |= 1u << j;
        }
        batch_write_unsorted(b, k, w, v, act, cnt, loc_act, u.cnt, d_cnt);
        w += k;
    }
}

// Warp-per-unit local sort.  Each warp takes whole local units and sorts
// their buckets in chunks of at most kWChunk long rows held in warp-private
// shared memory, with no CTA barrier.  A chunk ends at a bucket start, so
// its slots are exactly its sorted positions.  Inside a bucket an item's
// place is the count of bucket members below it in (key, t) order; its
// group head (equal unresolved keys) the count below it in key order; it
// is an unsorted member when its key is unresolved (length field kH0) and
// shared.  A unit with a bucket longer than one chunk, or with more list
// runs than the run table holds, is marked kFallback in u.cnt and left to
// sa_local_sort_kernel; what the warp wrote for it before giving up is
// written again, identically, there.  The results are those of the CTA
// kernel: SA, rank (the head's row), the unsorted members in sorted order
// at loc_act[beg ..], the unit's count and the block total.
constexpr int kWChunk = 256;
constexpr int kWStripes = kWChunk / 32;
constexpr int kWRuns = 32;
constexpr int kWWarps = 8;

struct WarpTile {
    unsigned long long key[kWChunk];
    uint32_t t[kWChunk];
    uint32_t row[kWChunk];
    uint32_t tpos[kWChunk];      // t of the suffix at each sorted position
    uint32_t run_start[kWRuns];  // first unit slot of each list run
    uint32_t run_src[kWRuns];    // list index of that slot
    uint8_t act[kWChunk];        // the suffix at this sorted position is an unsorted member
};

// List index of unit slot g (runs in slot order, r the run of an earlier
// slot of this lane or 0).
__device__ __forceinline__ uint32_t warp_list_index(const WarpTile& T, uint32_t nruns, uint32_t g, uint32_t& r) {
    while (r + 1 < nruns && T.run_start[r + 1] <= g) ++r;
    return T.run_src[r] + (g - T.run_start[r]);
}

__global__ void __launch_bounds__(kWWarps * 32) sa_local_sort_warp_kernel(
    uint32_t n, const uint32_t* __restrict__ ll_t, const uint32_t* __restrict__ ll_row,
    const unsigned long long* __restrict__ ll_key, Units u, uint32_t nwin, uint32_t* __restrict__ sa,
    uint32_t* __restrict__ rank, uint32_t* __restrict__ loc_act, uint32_t* __restrict__ d_cnt, int seg_shift) {
    __shared__ WarpTile tiles[kWWarps];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    WarpTile& T = tiles[threadIdx.x >> 5];
    const uint32_t warps = gridDim.x * kWWarps;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwin; w += warps) {
        const uint32_t beg = u.beg[w];
        if (beg == kNone || u.lofs[w] != kNone) continue;
        const uint32_t N = u.nlong[w];
        if (N == 0) continue;
        // the unit's list runs: window w from its unit start, then the
        // windows up to the next unit start (their rows before it)
        uint32_t nruns = 0, got = 0;
        for (uint32_t x0 = w; x0 < nwin; x0 += 32) {
            const uint32_t x = x0 + lane;
            uint32_t avail = 0, k0 = 0;
            bool stop = true;
            if (x < nwin) {
                if (x == w) {
                    k0 = u.lcb[w];
                    avail = u.lct[w] - k0;
                    stop = false;
                } else {
                    stop = u.beg[x] != kNone;
                    avail = stop ? u.lcb[x] : u.lct[x];
                }
            }
            const uint32_t stops = __ballot_sync(0xffffffffu, stop);
            const uint32_t first_stop = stops ? (uint32_t)__ffs(stops) - 1 : 32u;
            if (lane > first_stop) avail = 0;
            uint32_t inc = avail;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= (uint32_t)o) inc += y;
            }
            const uint32_t nonempty = __ballot_sync(0xffffffffu, avail > 0);
            if (avail > 0) {
                const uint32_t r = nruns + __popc(nonempty & below);
                if (r < kWRuns) {
                    T.run_start[r] = got + inc - avail;
                    T.run_src[r] = x * kWindow + k0;
                }
            }
            nruns += __popc(nonempty);
            got += __shfl_sync(0xffffffffu, inc, 31);
            if (first_stop < 32) break;
        }
        __syncwarp();
        bool ok = nruns <= kWRuns && got == N;
        uint32_t acnt = 0;  // unsorted members of the unit so far
        for (uint32_t s = 0; ok && s < N;) {
            const uint32_t c = min((uint32_t)kWChunk, N - s);
            uint32_t r = 0;
#pragma unroll
            for (int j = 0; j < kWStripes; ++j) {
                if ((uint32_t)j * 32 >= c) break;  // past the last stripe (warp-uniform)
                const uint32_t q = j * 32 + lane;
                if (q < c) {
                    const uint32_t src = warp_list_index(T, nruns, s + q, r);
                    T.key[q] = ll_key[src];
                    T.t[q] = ll_t[src];
                    T.row[q] = ll_row[src];
                }
            }
            unsigned long long next_key = 0;
            const bool more = s + c < N;
            if (more) {
                uint32_t r2 = 0;
                next_key = ll_key[warp_list_index(T, nruns, s + c, r2)];
            }
            __syncwarp();
            // end the chunk at its last bucket start when its last bucket
            // goes on past it
            uint32_t cut = c;
            if (more && (next_key >> seg_shift) == (T.key[c - 1] >> seg_shift)) {
                uint32_t last = 0;
#pragma unroll
                for (int j = 0; j < kWStripes; ++j) {
                    if ((uint32_t)j * 32 >= c) break;  // past the last stripe (warp-uniform)
                    const uint32_t q = j * 32 + lane;
                    if (q >= 1 && q < c && (T.key[q] >> seg_shift) != (T.key[q - 1] >> seg_shift)) last = q;
                }
                last = __reduce_max_sync(0xffffffffu, last);
                if (last == 0) {  // one bucket fills the chunk
                    ok = false;
                    break;
                }
                cut = last;
            }
            uint32_t bs_carry = 0;
#pragma unroll
            for (int j = 0; j < kWStripes; ++j) {
                if ((uint32_t)j * 32 >= cut) break;  // past the last stripe (warp-uniform)
                const uint32_t q = j * 32 + lane;
                const bool in = q < cut;
                const unsigned long long K = in ? T.key[q] : 0ull;
                const unsigned long long B = K >> seg_shift;
                const bool head = in && (q == 0 || (T.key[q - 1] >> seg_shift) != B);
                uint32_t bs = head ? q : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, bs, o);
                    if (lane >= (uint32_t)o) bs = max(bs, y);
                }
                bs = max(bs, bs_carry);
                bs_carry = __shfl_sync(0xffffffffu, bs, 31);
                if (in) {
                    const uint32_t t = T.t[q];
                    // a bucket's members are in t order in the chunk, so the
                    // equal keys below t are the equal keys at slots below q
                    uint32_t lt_key = 0, eq = 0, eq_below = 0;
                    for (uint32_t x = bs; x < cut; ++x) {
                        const unsigned long long kx = T.key[x];
                        if ((kx >> seg_shift) != B) break;
                        lt_key += kx < K;
                        eq += kx == K;
                        eq_below += (kx == K && x < q) ? 1u : 0u;
                    }
                    const uint32_t lt_pair = lt_key + eq_below;
                    const uint32_t p = bs + lt_pair;
                    const bool unresolved = (uint32_t)(K & 31) >= kH0;
                    const uint32_t hp = unresolved ? bs + lt_key : p;
                    const uint32_t row = T.row[p];
                    if (row < n && t < n) {
                        sa[row] = t;
                        rank[t] = T.row[hp];
                    }
                    T.tpos[p] = t;
                    T.act[p] = (unresolved && eq >= 2) ? 1 : 0;
                }
            }
            __syncwarp();
            // the chunk's unsorted members, in sorted order
#pragma unroll
            for (int j = 0; j < kWStripes; ++j) {
                if ((uint32_t)j * 32 >= cut) break;  // past the last stripe (warp-uniform)
                const uint32_t q = j * 32 + lane;
                const bool a = q < cut && T.act[q];
                const uint32_t bal = __ballot_sync(0xffffffffu, a);
                if (a) loc_act[beg + acnt + __popc(bal & below)] = T.tpos[q];
                acnt += __popc(bal);
            }
            __syncwarp();
            s += cut;
        }
        if (lane == 0) {
            if (!ok) {
                u.cnt[w] = kFallback;
            } else {
                u.cnt[w] = acnt;
                if (acnt) atomicAdd(d_cnt, acnt);
            }
        }
        __syncwarp();
    }
}

// The global-path list: every row of a unit with more than kLCap long
// suffixes, in row order, as (key, t, row).  One CTA per window; a window's
// rows belong to its owner unit up to the window's own unit start.
template <int kB>
__global__ void __launch_bounds__(kThreads) sa_large_gather_kernel(
    const uint32_t* __restrict__ text, unsigned long long base, uint32_t n,
    const unsigned long long* __restrict__ elems, Units u, uint32_t nwin, unsigned long long* __restrict__ lkeys,
    uint32_t* __restrict__ lvals, uint32_t* __restrict__ lpos, const uint32_t* __restrict__ d_large) {
    if (*d_large == 0) return;  // no unit takes the device-wide path (the usual case)
    for (uint32_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const uint32_t lo = w * kWindow, hi = min(n, lo + kWindow);
        const uint32_t beg = u.beg[w];
        const uint32_t split = beg == kNone ? hi : beg;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const uint32_t q = part == 0 ? u.owner[w] : w;
            const uint32_t r0 = part == 0 ? lo : split, r1 = part == 0 ? split : hi;
            if (r0 >= r1 || u.lofs[q] == kNone) continue;
            const uint32_t lofs = u.lofs[q], qbeg = u.beg[q];
            for (uint32_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
                const unsigned long long e = elems[i];
                const uint32_t t = (uint32_t)(e >> 32);
                const uint32_t o = lofs + (i - qbeg);
                lkeys[o] = key_with_len<kB>(text, base + (t < n ? t : 0u), ((uint32_t)e >> 24) & 31u);
                lvals[o] = t;
                lpos[o] = i;
            }
        }
    }
}

// next-ranks of the local unsorted members (one warp per unit), read before
// any rank of the round changes
__global__ void __launch_bounds__(kThreads) sa_round_gather_local_kernel(
    const uint32_t* __restrict__ loc_act, Units u, uint32_t nwin, const uint32_t* __restrict__ rank, uint32_t h,
    uint32_t n, uint32_t* __restrict__ loc_next, uint32_t* __restrict__ d_err) {
    constexpr int kG = 4;  // 32-member steps whose loads are in flight together
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (kThreads / 32);
    for (uint32_t w = (blockIdx.x * kThreads + threadIdx.x) >> 5; w < nwin; w += warps) {
        const uint32_t beg = u.beg[w], lofs = u.lofs[w], cnt = u.cnt[w];
        if (beg == kNone || lofs != kNone) continue;
        for (uint32_t k0 = 0; k0 < cnt; k0 += 32 * kG) {
            uint32_t t[kG], nx[kG];
#pragma unroll
            for (int i = 0; i < kG; ++i) {
                const uint32_t k = k0 + i * 32 + lane;
                t[i] = k < cnt ? loc_act[beg + k] : kNone;
            }
#pragma unroll
            for (int i = 0; i < kG; ++i) {
                const bool in = k0 + i * 32 + lane < cnt;
                const bool ok = (uint64_t)t[i] + h < n;
                if (in && !ok) atomicOr(d_err, 128u);
                nx[i] = in && ok ? rank[t[i] + h] : 0u;
            }
#pragma unroll
            for (int i = 0; i < kG; ++i) {
                const uint32_t k = k0 + i * 32 + lane;
                if (k < cnt) loc_next[beg + k] = nx[i];
            }
        }
    }
}

// One round for the local units, a batch of units per CTA step: sort the
// unsorted members by (rank[t], rank[t + h]); a member of the group whose
// head row is H that lands at offset x of its group takes row H + x.
__global__ void __launch_bounds__(kLThreads, 4) sa_round_local_kernel(
    uint32_t* __restrict__ loc_act, const uint32_t* __restrict__ loc_next, Units u, uint32_t nwin, uint32_t n,
    uint32_t* __restrict__ rank, uint32_t* __restrict__ sa, uint32_t* __restrict__ d_cnt,
    uint32_t* __restrict__ d_err, const uint32_t* __restrict__ d_left) {
    if (*d_left == 0) return;  // the warp kernel left no unit of more than kWChunk members
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kLSlots);
    uint32_t* sseg = sval + kLSlots;
    __shared__ Batch b;
    __shared__ uint32_t first_left;

    const uint32_t per = (nwin + gridDim.x - 1) / gridDim.x;
    const uint32_t wbeg = min(nwin, blockIdx.x * per), wend = min(nwin, wbeg + per);
    for (uint32_t w = wbeg; w < wend;) {
        const uint32_t x = w + threadIdx.x;
        // units of at most kWChunk members are the warp kernel's (it ran
        // first; their counts only shrank); they end a batch
        uint32_t c = kLCap + 1, ub = kNone;
        bool left = false;
        if (x < wend) {
            ub = u.beg[x];
            const uint32_t cx = (ub != kNone && u.lofs[x] == kNone) ? u.cnt[x] : 0u;
            left = cx > (uint32_t)kWChunk;
            c = left ? min(cx, kLCap) : (cx ? kLCap + 1 : 0u);
        }
        if (threadIdx.x == 0) first_left = kNone;
        __syncthreads();
        if (left) atomicMin(&first_left, x);
        __syncthreads();
        const uint32_t fl = first_left;
        __syncthreads();  // read by every thread before thread 0 resets it
        if (fl == kNone) {
            w += kLThreads;
            continue;
        }
        if (fl > w) {
            w = fl;
            continue;
        }
        uint32_t total;
        const uint32_t k = form_batch(b, c, ub, total);
        if (k == 0) {
            ++w;
            continue;
        }
        if (total == 0) {
            w += k;
            continue;
        }
        // key (rank[t], rank[t + h]) of each slot, loaded blocked: every
        // item's member and next rank first, then the members' ranks, so a
        // thread's loads are in flight together
        const uint32_t g0 = threadIdx.x * kLItems;
        unsigned long long kk[kLItems];
        uint32_t v[kLItems], nx[kLItems], src[kLItems];
        uint32_t wi = g0 < total ? batch_window(b, k, g0) : 0u;
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const uint32_t g = g0 + j;
            src[j] = 0;
            if (g < total) {
                while (wi + 1 < k && b.pref[wi + 1] <= g) ++wi;
                src[j] = b.beg[wi] + (g - b.pref[wi]);
            }
        }
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const bool in = g0 + j < total;
            v[j] = in ? loc_act[src[j]] : 0u;
            nx[j] = in ? loc_next[src[j]] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const bool in = g0 + j < total;
            const uint32_t here = in && v[j] < n ? rank[v[j]] : 0u;
            kk[j] = in ? (((unsigned long long)here << 32) | nx[j]) : ~0ull;
        }
        block_sort(kk, v, total, skey, sval, sseg, 32);  // segments: the old groups (equal rank[t])

        const unsigned long long kprev = (g0 > 0 && g0 <= total) ? skey[skew(g0 - 1)] : 0ull;
        uint32_t heads = 0, starts = 0;  // new groups; old groups (a new head row)
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const uint32_t g = g0 + j;
            const unsigned long long pk = j ? kk[j - 1] : kprev;
            heads |= (uint32_t)(g < total && (g == 0 || kk[j] != pk)) << j;
            starts |= (uint32_t)(g < total && (g == 0 || (kk[j] >> 32) != (pk >> 32))) << j;
        }
        bool next_head = true;
        if (g0 + kLItems < total) next_head = skey[skew(g0 + kLItems)] != kk[kLItems - 1];
        uint32_t hfirst = carry_in_head(heads, g0);
        uint32_t ofirst = carry_in_head(starts, g0);
        uint32_t act = 0;
#pragma unroll
        for (int j = 0; j < kLItems; ++j) {
            const uint32_t g = g0 + j;
            if (g >= total) break;
            const bool h = (heads >> j) & 1u;
            if (h) hfirst = g;
            if ((starts >> j) & 1u) ofirst = g;
            const bool e = j + 1 < kLItems ? (((heads >> (j + 1)) & 1u) || g + 1 >= total) : next_head;
            const uint32_t here = (uint32_t)(kk[j] >> 32);
            const uint32_t row = here + (g - ofirst);
            if (row < n && v[j] < n) {
                sa[row] = v[j];
                rank[v[j]] = here + (hfirst - ofirst);
            } else {
                atomicOr(d_err, 64u);
            }
            if (!(h && e)) act |= 1u << j;
        }
        batch_write_unsorted(b, k, w, v, act, total, loc_act, u.cnt, d_cnt);
        w += k;
    }
}

// One round for the local units of at most kWChunk unsorted members, one
// warp per unit: the members and their keys (rank[t], rank[t + h]) are
// loaded into the warp's tile before any rank of the unit changes; inside
// an old group (equal rank[t], consecutive in the member list) a member's
// place is the count below it in (key, t) order, its new group head the
// count below it in key order.  Same results as sa_round_local_kernel,
// which takes the larger units.
__global__ void __launch_bounds__(kWWarps * 32) sa_round_local_warp_kernel(
    uint32_t* __restrict__ loc_act, const uint32_t* __restrict__ loc_next, Units u, uint32_t nwin, uint32_t n,
    uint32_t* __restrict__ rank, uint32_t* __restrict__ sa, uint32_t* __restrict__ d_cnt,
    uint32_t* __restrict__ d_err, uint32_t* __restrict__ d_left) {
    __shared__ WarpTile tiles[kWWarps];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    WarpTile& T = tiles[threadIdx.x >> 5];
    const uint32_t warps = gridDim.x * kWWarps;
    // the (start, global-path offset, count) of the warp's next window is
    // fetched while the current one is sorted (the counts this kernel writes
    // are its own windows' only)
    uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nbeg = kNone, nlofs = kNone, ncnt = 0;
    if (w < nwin) {
        nbeg = u.beg[w];
        nlofs = u.lofs[w];
        ncnt = u.cnt[w];
    }
    for (; w < nwin; w += warps) {
        const uint32_t beg = nbeg, lofs = nlofs, cnt = ncnt;
        if (w + warps < nwin) {
            nbeg = u.beg[w + warps];
            nlofs = u.lofs[w + warps];
            ncnt = u.cnt[w + warps];
        }
        if (beg == kNone || lofs != kNone) continue;
        if (cnt > (uint32_t)kWChunk && lane == 0) atomicAdd(d_left, 1u);  // the CTA kernel's unit
        if (cnt == 0 || cnt > (uint32_t)kWChunk) continue;
        // the loads of four stripes issued before any is used: members and
        // next ranks, then the members' ranks
        constexpr int kHalf = kWStripes / 2;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            if ((uint32_t)hf * 32 * kHalf >= cnt) break;  // warp-uniform
            uint32_t mt[kHalf], nx[kHalf], hr[kHalf];
#pragma unroll
            for (int i = 0; i < kHalf; ++i) {
                const uint32_t q = (hf * kHalf + i) * 32 + lane;
                mt[i] = q < cnt ? loc_act[beg + q] : kNone;
                nx[i] = q < cnt ? loc_next[beg + q] : 0u;
            }
#pragma unroll
            for (int i = 0; i < kHalf; ++i) hr[i] = mt[i] < n ? rank[mt[i]] : 0u;
#pragma unroll
            for (int i = 0; i < kHalf; ++i) {
                const uint32_t q = (hf * kHalf + i) * 32 + lane;
                if (q < cnt) {
                    T.key[q] = ((unsigned long long)hr[i] << 32) | nx[i];
                    T.t[q] = mt[i];
                }
            }
        }
        __syncwarp();
        uint32_t bs_carry = 0;
#pragma unroll
        for (int j = 0; j < kWStripes; ++j) {
            if ((uint32_t)j * 32 >= cnt) break;  // past the last stripe (warp-uniform)
            const uint32_t q = j * 32 + lane;
            const bool in = q < cnt;
            const unsigned long long K = in ? T.key[q] : 0ull;
            const uint32_t here = (uint32_t)(K >> 32);
            const bool head = in && (q == 0 || (uint32_t)(T.key[q - 1] >> 32) != here);
            uint32_t bs = head ? q : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, bs, o);
                if (lane >= (uint32_t)o) bs = max(bs, y);
            }
            bs = max(bs, bs_carry);
            bs_carry = __shfl_sync(0xffffffffu, bs, 31);
            if (in) {
                const uint32_t t = T.t[q];
                // an old group's members are listed in t order, so the equal
                // keys below t are the equal keys at slots below q
                uint32_t lt_key = 0, eq = 0, eq_below = 0;
                for (uint32_t x = bs; x < cnt; ++x) {
                    const unsigned long long kx = T.key[x];
                    if ((uint32_t)(kx >> 32) != here) break;
                    lt_key += kx < K;
                    eq += kx == K;
                    eq_below += (kx == K && x < q) ? 1u : 0u;
                }
                const uint32_t lt_pair = lt_key + eq_below;
                const uint32_t row = here + lt_pair;
                if (row < n && t < n) {
                    sa[row] = t;
                    rank[t] = here + lt_key;
                } else {
                    atomicOr(d_err, 64u);
                }
                T.tpos[bs + lt_pair] = t;
                T.act[bs + lt_pair] = eq >= 2 ? 1 : 0;
            }
        }
        __syncwarp();
        uint32_t acnt = 0;
#pragma unroll
        for (int j = 0; j < kWStripes; ++j) {
            if ((uint32_t)j * 32 >= cnt) break;  // past the last stripe (warp-uniform)
            const uint32_t q = j * 32 + lane;
            const bool a = q < cnt && T.act[q];
            const uint32_t bal = __ballot_sync(0xffffffffu, a);
            if (a) loc_act[beg + acnt + __popc(bal & below)] = T.tpos[q];
            acnt += __popc(bal);
        }
        if (lane == 0) {
            u.cnt[w] = acnt;
            if (acnt) atomicAdd(d_cnt, acnt);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kThreads) sa_round_keys_kernel(const uint32_t* __restrict__ act_suf,
                                                                 const uint32_t* __restrict__ d_cnt,
                                                                 const uint32_t* __restrict__ rank, uint32_t h,
                                                                 uint32_t n, int bits,
                                                                 unsigned long long* __restrict__ keys,
                                                                 uint32_t* __restrict__ vals,
                                                                 uint32_t* __restrict__ d_err) {
    const uint32_t cnt = *d_cnt;
    for (uint32_t k = blockIdx.x * kThreads + threadIdx.x; k < cnt; k += gridDim.x * kThreads) {
        const uint32_t t = act_suf[k];
        // an unsorted member has at least h symbols before its terminator, so
        // t + h stays inside the block; anything else is a fault of the caller
        uint32_t next = 0, here = 0;
        if ((uint64_t)t + h < n) {
            next = rank[t + h];
            here = rank[t];
        } else {
            atomicOr(d_err, 4u);
        }
        keys[k] = ((unsigned long long)here << bits) | next;
        vals[k] = t;
    }
}

// Group bookkeeping of the global path after a device-wide sort.  Element i
// of the sorted list (keys, vals) sits on row act_pos_in[i] of the block SA.
// It writes SA[pos] = t, rank[t] = row of t's group head, and appends the
// members of groups with two or more elements to (act_pos_out, act_suf_out).
// kInit: the list of the initial keys, where a key that contains its
// terminator is a group of its own.  Reduce-then-scan over chunks of whole
// tiles: groups_reduce gives each chunk's last head row and member count,
// groups_scan turns them into per-chunk prefixes (and the total into
// *d_cnt_out), groups_apply walks each chunk with running values.
struct ElemInfo {
    unsigned long long k[kGItems];
    uint32_t pos[kGItems];
    uint32_t heads;  // bit q: element q starts a group
    uint32_t ends;   // bit q: element q is the last of its group
};

template <bool kInit>
__device__ __forceinline__ void load_tile_info(const unsigned long long* __restrict__ keys,
                                               const uint32_t* __restrict__ act_pos_in, uint32_t n, uint32_t i0,
                                               ElemInfo& e) {
#pragma unroll
    for (int q = 0; q < kGItems; ++q) {
        const uint32_t i = i0 + q;
        e.k[q] = i < n ? keys[i] : 0ull;
        e.pos[q] = i < n ? act_pos_in[i] : 0u;
    }
    const unsigned long long kprev = (i0 > 0 && i0 - 1 < n) ? keys[i0 - 1] : 0ull;
    // is the element after this thread's last one a group head?
    bool next_head = true;
    if ((uint64_t)i0 + kGItems < n) {
        const unsigned long long kn = keys[i0 + kGItems];
        next_head = kn != e.k[kGItems - 1] || (kInit && (uint32_t)(kn & 31) < kH0);
    }
    e.heads = 0;
#pragma unroll
    for (int q = 0; q < kGItems; ++q) {
        const uint32_t i = i0 + q;
        const unsigned long long prev = q == 0 ? kprev : e.k[q - 1];
        const bool h = i < n && (i == 0 || e.k[q] != prev || (kInit && (uint32_t)(e.k[q] & 31) < kH0));
        e.heads |= (uint32_t)h << q;
    }
    e.ends = 0;
#pragma unroll
    for (int q = 0; q < kGItems; ++q) {
        const uint32_t i = i0 + q;
        const bool hn = q + 1 < kGItems ? (((e.heads >> (q + 1)) & 1u) || i + 1 >= n) : next_head;
        e.ends |= (uint32_t)hn << q;
    }
}

__device__ __forceinline__ void chunk_tiles(uint32_t ntiles, uint32_t& t0, uint32_t& t1) {
    const uint32_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    t0 = min(ntiles, blockIdx.x * per);
    t1 = min(ntiles, t0 + per);
}

template <bool kInit>
__global__ void __launch_bounds__(kThreads) sa_groups_reduce_kernel(const unsigned long long* __restrict__ keys,
                                                                    const uint32_t* __restrict__ act_pos_in,
                                                                    const uint32_t* __restrict__ d_cnt,
                                                                    uint2* __restrict__ chunk_agg) {
    const uint32_t n = *d_cnt;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kGTile - 1) / kGTile);
    uint32_t t0, t1;
    chunk_tiles(ntiles, t0, t1);
    uint32_t tmax = 0, tsum = 0;
    for (uint32_t tile = t0; tile < t1; ++tile) {
        ElemInfo e;
        const uint32_t i0 = tile * kGTile + threadIdx.x * kGItems;
        load_tile_info<kInit>(keys, act_pos_in, n, i0, e);
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            if (i0 + q >= n) continue;
            const bool h = (e.heads >> q) & 1u, en = (e.ends >> q) & 1u;
            if (h) tmax = max(tmax, e.pos[q]);
            tsum += (h && en) ? 0u : 1u;
        }
    }
    uint32_t totmax, totsum;
    cta_exclusive_scan<MaxOp, kThreads>(tmax, totmax);
    cta_exclusive_scan<SumOp, kThreads>(tsum, totsum);
    if (threadIdx.x == 0) chunk_agg[blockIdx.x] = make_uint2(totmax, totsum);
}

__global__ void __launch_bounds__(kThreads) sa_groups_scan_kernel(uint2* __restrict__ chunk_agg, int nchunks,
                                                                  uint32_t* __restrict__ d_cnt_out) {
    uint32_t cmax = 0, csum = 0;
    for (int base = 0; base < nchunks; base += kThreads) {
        const int c = base + threadIdx.x;
        const uint2 v = c < nchunks ? chunk_agg[c] : make_uint2(0u, 0u);
        uint32_t tmax, tsum;
        const uint32_t emax = cta_exclusive_scan<MaxOp, kThreads>(v.x, tmax);
        const uint32_t esum = cta_exclusive_scan<SumOp, kThreads>(v.y, tsum);
        if (c < nchunks) chunk_agg[c] = make_uint2(max(cmax, emax), csum + esum);
        cmax = max(cmax, tmax);
        csum += tsum;
    }
    if (threadIdx.x == 0) *d_cnt_out = csum;
}

template <bool kInit>
__global__ void __launch_bounds__(kThreads) sa_groups_apply_kernel(
    const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ act_pos_in, const uint32_t* __restrict__ d_cnt, uint32_t n_block,
    const uint2* __restrict__ chunk_prefix, uint32_t* __restrict__ sa, uint32_t* __restrict__ rank,
    uint32_t* __restrict__ act_pos_out, uint32_t* __restrict__ act_suf_out, uint32_t* __restrict__ d_err) {
    const uint32_t n = *d_cnt;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kGTile - 1) / kGTile);
    uint32_t t0, t1;
    chunk_tiles(ntiles, t0, t1);
    uint32_t run_max = chunk_prefix[blockIdx.x].x, run_sum = chunk_prefix[blockIdx.x].y;
    for (uint32_t tile = t0; tile < t1; ++tile) {
        ElemInfo e;
        const uint32_t i0 = tile * kGTile + threadIdx.x * kGItems;
        load_tile_info<kInit>(keys, act_pos_in, n, i0, e);
        uint32_t tmax = 0, tsum = 0;
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            if (i0 + q >= n) continue;
            const bool h = (e.heads >> q) & 1u, en = (e.ends >> q) & 1u;
            if (h) tmax = max(tmax, e.pos[q]);
            tsum += (h && en) ? 0u : 1u;
        }
        uint32_t totmax, totsum;
        const uint32_t exmax = cta_exclusive_scan<MaxOp, kThreads>(tmax, totmax);
        const uint32_t exsum = cta_exclusive_scan<SumOp, kThreads>(tsum, totsum);
        uint32_t cur = max(run_max, exmax);
        uint32_t out = run_sum + exsum;
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            const uint32_t i = i0 + q;
            if (i >= n) continue;
            const bool h = (e.heads >> q) & 1u, en = (e.ends >> q) & 1u;
            if (h) cur = e.pos[q];
            const uint32_t t = vals[i];
            if (t < n_block && e.pos[q] < n_block) {
                sa[e.pos[q]] = t;
                rank[t] = cur;
            } else {
                atomicOr(d_err, 32u);
            }
            if (!(h && en)) {
                if (out < n_block) {
                    act_pos_out[out] = e.pos[q];
                    act_suf_out[out] = t;
                } else {
                    atomicOr(d_err, 32u);
                }
                ++out;
            }
        }
        run_max = max(run_max, totmax);
        run_sum += totsum;
    }
}

constexpr size_t kLocalSortSmem = (size_t)kLSlots * (8 + 4 + 4 + 4);
constexpr size_t kRoundLocalSmem = (size_t)kLSlots * (8 + 4 + 4);

unsigned g_window_ctas[64] = {0};
unsigned g_round_keys_ctas[64] = {0};
unsigned g_groups_ctas[64] = {0};
unsigned g_local_ctas[64] = {0};
unsigned g_local_warp_ctas[64] = {0};
unsigned g_round_warp_ctas[64] = {0};
unsigned g_round_local_ctas[64] = {0};

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

}  // namespace

void suffix_sort_init() {
    radix_init();
    const int dev = current_device();
    cudaFuncSetAttribute(sa_local_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLocalSortSmem);
    cudaFuncSetAttribute(sa_round_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRoundLocalSmem);
    g_window_ctas[dev] = persistent_ctas((const void*)sa_unit_begin_kernel<2>, kThreads, 0);
    g_round_keys_ctas[dev] = persistent_ctas((const void*)sa_round_keys_kernel, kThreads, 0);
    g_groups_ctas[dev] = std::min<unsigned>(kMaxGroupChunks,
                                            persistent_ctas((const void*)sa_groups_apply_kernel<false>, kThreads, 0));
    g_local_ctas[dev] = persistent_ctas((const void*)sa_local_sort_kernel, kLThreads, kLocalSortSmem);
    g_local_warp_ctas[dev] = persistent_ctas((const void*)sa_local_sort_warp_kernel, kWWarps * 32, 0);
    g_round_warp_ctas[dev] = persistent_ctas((const void*)sa_round_local_warp_kernel, kWWarps * 32, 0);
    g_round_local_ctas[dev] = persistent_ctas((const void*)sa_round_local_kernel, kLThreads, kRoundLocalSmem);
}

uint32_t suffix_sort_rounds(uint32_t max_len, int code_bits) {
    uint32_t r = 0;
    uint64_t resolved = code_bits == 4 ? KeyGeom<4>::H : KeyGeom<2>::H;
    while (resolved <= max_len) {
        resolved *= 2;
        ++r;
    }
    return r;
}

// slot 0: n; 1: size of the global-path list; 2 + 2r: global-path unsorted
// members after round r (r = 0: the initial sort); 3 + 2r: local ones;
// 3 + 2R + r (R rounds, r >= 1): units of round r left to the CTA kernel
size_t suffix_sort_log_slots(uint32_t max_len, int code_bits) {
    return 4 + 3 * (size_t)suffix_sort_rounds(max_len, code_bits);
}

size_t suffix_sort_chunk_words(uint64_t cap) {
    (void)cap;
    return kMaxGroupChunks;  // one (max, count) pair per chunk, 8 bytes each
}

size_t suffix_sort_unit_bytes(uint64_t cap) { return (size_t)kUnitFields * unit_stride(cap) * 4; }

namespace {

template <bool kInit>
void run_groups(Launcher& L, const SuffixSortBuffers& b, const unsigned long long* keys, const uint32_t* vals,
                const uint32_t* act_pos_in, const uint32_t* d_cnt, uint32_t n_block, uint32_t* act_pos_out,
                uint32_t* act_suf_out, uint32_t* d_cnt_out, unsigned grid) {
    uint2* agg = reinterpret_cast<uint2*>(b.chunks);
    const char* names[3] = {kInit ? "sa_large_groups_reduce" : "sa_round_groups_reduce", "sa_groups_scan",
                            kInit ? "sa_large_groups_apply" : "sa_round_groups_apply"};
    SBWT_LAUNCH(L, names[0], 0, 12, d_cnt, sa_groups_reduce_kernel<kInit>, grid, kThreads, 0, keys, act_pos_in,
                d_cnt, agg);
    SBWT_LAUNCH(L, names[1], 16.0 * grid, 0, nullptr, sa_groups_scan_kernel, 1, kThreads, 0, agg, (int)grid,
                d_cnt_out);
    // per element: key (+ neighbours), value, position, SA and rank writes,
    // and the compacted pair of an unsorted member
    SBWT_LAUNCH(L, names[2], 0, 36, d_cnt, sa_groups_apply_kernel<kInit>, grid, kThreads, 0, keys, vals, act_pos_in,
                d_cnt, n_block, agg, b.sa, b.rank, act_pos_out, act_suf_out, b.err);
}

}  // namespace

void suffix_sort_block(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, uint32_t n,
                       uint32_t max_len, int code_bits, int sigma, const SuffixSortBuffers& b) {
    if (n == 0) return;
    const int dev = current_device();
    const uint64_t gtiles = (uint64_t)n / kGTile + 1;
    auto grid_of = [](unsigned ctas, uint64_t need) {
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(std::max(1u, ctas), need));
    };
    const bool wide = code_bits == 4;
    const uint32_t rounds = suffix_sort_rounds(max_len, code_bits);
    // 4-bit codes: buckets of pw codes numbered in base sigma, pw as large as
    // the 24-bit digits allow (pairs: sum_{l <= pw} sigma^l)
    uint32_t pw = KeyGeom<4>::P;
    if (wide && sigma >= 2) {
        pw = 1;
        for (uint32_t P = 1; P <= KeyGeom<4>::H; ++P) {
            uint64_t pairs = 0, pow = 1;
            for (uint32_t l = 0; l <= P; ++l, pow *= (uint64_t)sigma) pairs += pow;
            if (pairs > (1ull << kDigitBits)) break;
            pw = P;
        }
    }
    const int seg_shift = wide ? 5 + (int)KeyGeom<4>::CB - 4 * (int)pw : kBucketShift;
    const uint32_t nwin = (uint32_t)(((uint64_t)n + kWindow - 1) / kWindow);
    const unsigned warp_grid = grid_of(g_window_ctas[dev], (uint64_t)nwin / (kThreads / 32) + 1);
    const Units units = units_at(b.units, n);
    const int digit_bits = kDigitBits;
    auto* const digit_keys = wide ? sa_digit_keys_kernel<4> : sa_digit_keys_kernel<2>;
    auto* const unit_begin = wide ? sa_unit_begin_kernel<4> : sa_unit_begin_kernel<2>;
    auto* const large_gather = wide ? sa_large_gather_kernel<4> : sa_large_gather_kernel<2>;

    uint32_t* d_n = b.count_log;
    uint32_t* d_large = b.count_log + 1;
    // the keys, and the digit counts of the sort's first pass over them
    radix_clear(L, b.radix_temp);
    SBWT_LAUNCH(L, "sa_digit_keys", (double)n * 8 + n * code_bits / 8.0 + n / 8.0, 0, nullptr, digit_keys,
                radix_keys_grid(n), kKeyThreads, 0, text, term, (unsigned long long)base, n,
                (uint32_t)std::max(sigma, 2), pw, b.keys, d_n, radix_first_counts(b.radix_temp),
                radix_first_totals(b.radix_temp));
    const bool da = radix_sort_keys(L, b.keys, b.keys_alt, d_n, n, 0, digit_bits, b.radix_temp, b.err, true);
    const unsigned long long* elems = da ? b.keys_alt : b.keys;  // (digit, t) in row order
    // the other 64-bit array holds the keys of the listed long rows, then the
    // device-wide path's list
    unsigned long long* other = da ? b.keys : b.keys_alt;
    // the long rows of each window, listed in the block's free arrays (the
    // next-rank array and the device-wide path's second member list are not
    // used before the first round)
    uint32_t* ll_t = b.loc_next;
    uint32_t* ll_row = b.act_suf[0];
    unsigned long long* ll_key = other;
    SBWT_LAUNCH(L, "sa_unit_begin", (double)n * 24 + 32.0 * nwin, 0, nullptr, unit_begin,
                warp_grid, kThreads, 0, text, (unsigned long long)base, elems, n, nwin, units, b.sa, b.rank,
                ll_t, ll_row, ll_key, b.err);
    SBWT_LAUNCH(L, "sa_unit_scan", 96.0 * nwin, 0, nullptr, sa_unit_scan_kernel, 1, kScanThreads, 0, units, nwin, n,
                d_large, b.count_log + 3, (int)rounds + 1, 2, b.count_log + 4 + 2 * rounds, (int)rounds);
    // per long row: its list entry (t, row, key), SA and rank writes; per
    // unsorted member the compacted entry
    SBWT_LAUNCH(L, "sa_local_sort", (double)n * 24, 4, b.count_log + 3, sa_local_sort_warp_kernel,
                grid_of(g_local_warp_ctas[dev], (uint64_t)nwin / kWWarps + 1), kWWarps * 32, 0, n, ll_t, ll_row,
                ll_key, units, nwin, b.sa, b.rank, b.loc_act, b.count_log + 3, seg_shift);
    // the units with a bucket longer than a warp chunk
    SBWT_LAUNCH(L, "sa_local_sort_cta", 0, 0, nullptr, sa_local_sort_kernel, grid_of(g_local_ctas[dev], nwin),
                kLThreads, kLocalSortSmem, n, ll_t, ll_row, ll_key, units, nwin, b.sa, b.rank, b.loc_act,
                b.count_log + 3, b.err, seg_shift);
    // the list of the device-wide path goes to the other array (the long
    // rows' keys are dead once the local sort has run)
    SBWT_LAUNCH(L, "sa_large_gather", 32.0 * nwin, 24, d_large, large_gather, grid_of(g_local_ctas[dev], nwin),
                kThreads, 0, text, (unsigned long long)base, n, elems, units, nwin, other, b.vals,
                b.act_pos[0], d_large);
    unsigned long long* spare = da ? b.keys_alt : b.keys;  // the elements are dead now
    const bool la = radix_sort_pairs_fused(L, other, b.vals, spare, b.vals_alt, d_large, n, 0, 63, b.radix_temp,
                                           b.err);
    run_groups<true>(L, b, la ? spare : other, la ? b.vals_alt : b.vals, b.act_pos[0], d_large, n, b.act_pos[1],
                     b.act_suf[1], b.count_log + 2, grid_of(g_groups_ctas[dev], gtiles));

    const int bits = n > 1 ? 32 - __builtin_clz(n - 1) : 1;
    uint32_t h = wide ? KeyGeom<4>::H : KeyGeom<2>::H;
    int cur = 1;
    for (uint32_t r = 1; r <= rounds; ++r, h *= 2) {
        const uint32_t* cnt = b.count_log + 2 + 2 * (r - 1);
        uint32_t* next_cnt = b.count_log + 2 + 2 * r;
        const uint32_t* loc_cnt = b.count_log + 3 + 2 * (r - 1);
        uint32_t* left = b.count_log + 3 + 2 * rounds + r;
        SBWT_LAUNCH(L, "sa_round_gather", 0, 12, loc_cnt, sa_round_gather_local_kernel, warp_grid, kThreads, 0,
                    b.loc_act, units, nwin, b.rank, h, n, b.loc_next, b.err);
        SBWT_LAUNCH(L, "sa_round_keys", 0, 24, cnt, sa_round_keys_kernel,
                    grid_of(g_round_keys_ctas[dev], (uint64_t)n / kThreads + 1), kThreads, 0, b.act_suf[cur], cnt,
                    b.rank, h, n, bits, b.keys, b.vals, b.err);
        SBWT_LAUNCH(L, "sa_round_local", 0, 24, loc_cnt, sa_round_local_warp_kernel,
                    grid_of(g_round_warp_ctas[dev], (uint64_t)nwin / kWWarps + 1), kWWarps * 32, 0, b.loc_act,
                    b.loc_next, units, nwin, n, b.rank, b.sa, b.count_log + 3 + 2 * r, b.err, left);
        SBWT_LAUNCH(L, "sa_round_local_cta", 0, 0, nullptr, sa_round_local_kernel,
                    grid_of(g_round_local_ctas[dev], nwin), kLThreads, kRoundLocalSmem, b.loc_act, b.loc_next,
                    units, nwin, n, b.rank, b.sa, b.count_log + 3 + 2 * r, b.err, left);
        const bool a = radix_sort_pairs_fused(L, b.keys, b.vals, b.keys_alt, b.vals_alt, cnt, n, 0, 2 * bits,
                                              b.radix_temp, b.err);
        run_groups<false>(L, b, a ? b.keys_alt : b.keys, a ? b.vals_alt : b.vals, b.act_pos[cur], cnt, n,
                          b.act_pos[cur ^ 1], b.act_suf[cur ^ 1], next_cnt, grid_of(g_groups_ctas[dev], gtiles));
        cur ^= 1;
    }
}

}  // namespace sbwt
