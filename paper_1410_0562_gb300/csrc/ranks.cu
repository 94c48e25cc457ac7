// ranks.cu -- B_int extraction, ComputeRanks, the g[SA_int] gather, rank
// queries and the unpacking of B (arXiv 1410.0562, Algorithm 1 and
// Algorithm 2 with Lemma 1).
#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;

// B_int[i]: the symbol before block suffix SA[i] inside its read, or a
// terminator when the suffix starts its read (Eq. 1 restricted to the block).
__global__ void __launch_bounds__(kThreads) bint_kernel(const uint32_t* __restrict__ text,
                                                        const uint32_t* __restrict__ term, unsigned long long base,
                                                        const uint32_t* __restrict__ sa, uint32_t n,
                                                        uint8_t* __restrict__ bint) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = sa[i] < n ? sa[i] : 0u;
    const uint64_t P = base + t;
    bint[i] = (t == 0 || is_term(term, P - 1)) ? kBintDollar : (uint8_t)text_code(text, P - 1);
}

// Algorithm 2, one thread per read: start at i = m_ext on the read's
// terminator (it is larger than exactly the m_ext old terminators and smaller
// than every old suffix that starts with a symbol), then walk the read
// backwards with Lemma 1: i := C[c] + rank(c, i, B_ext), c = P[k-1].
// With kStage the superblock counters (at most kSuperStageBytes) are first
// copied to shared memory, so a step reads one occurrence block and nothing
// else.  The g values of a read are produced at descending positions; they
// are kept in registers and written 16 bytes at a time wherever a group of
// 16 / sizeof(IdxT) positions is complete (g starts on a 16-byte boundary).
constexpr uint32_t kSuperStageBytes = 48 * 1024;

// rank(c, i) within i's superblock of the 2-bit dictionary, with row
// arithmetic in the index type I (32 bits for a 32-bit index).
template <class I, int K>
__device__ __forceinline__ I occ_in_super_i(const unsigned long long* __restrict__ words, uint32_t c, I i) {
    if constexpr (K == 1) {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(words) + 2 * (i >> kOccShift);
        const ulonglong2 s = __ldg(p);      // lo, hi
        const ulonglong2 d = __ldg(p + 1);  // dm, counts
        const uint32_t r = (uint32_t)i & (kOccSpan - 1);
        const unsigned long long m = plane_match(s.x, s.y, d.x, c) & ((1ull << r) - 1ull);
        return (I)(((uint32_t)(d.y >> (16 * c)) & 0xFFFFu) + (uint32_t)__popcll(m));
    } else {
        return (I)occ_rank_in_super<K>(words, c, (unsigned long long)i);
    }
}

template <class IdxT, bool kStage, int kB, int K>
__global__ void __launch_bounds__(kThreads) compute_ranks_kernel(const uint32_t* __restrict__ text,
                                                                 const unsigned long long* __restrict__ offsets,
                                                                 unsigned long long j_begin,
                                                                 unsigned long long nreads,
                                                                 const typename DictLayout<kB, K>::Block* blocks,
                                                                 const unsigned long long* __restrict__ super,
                                                                 const unsigned long long* __restrict__ d_C,
                                                                 unsigned long long n_ext,
                                                                 unsigned long long m_ext, IdxT* __restrict__ g,
                                                                 uint32_t* __restrict__ d_err) {
    // row and position arithmetic in the index type: a 32-bit index has
    // fewer than 2^32 rows and text positions
    using I = IdxT;
    constexpr int kSS = DictLayout<kB, K>::kSuperShift, kCodes = DictLayout<kB, K>::kCodes;
    constexpr uint32_t kPer = 32 / kB;  // codes per text word
    extern __shared__ unsigned long long s_raw[];
    I* s_super = reinterpret_cast<I*>(s_raw);
    if (kStage) {
        const uint32_t words = ((uint32_t)(n_ext >> kSS) + 1) * kCodes;
        for (uint32_t x = threadIdx.x; x < words; x += kThreads) s_super[x] = (I)super[x];
        __syncthreads();
    }
    const uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j >= nreads) return;
    const uint64_t jj = j_begin + j;
    const uint64_t o0 = offsets[j_begin];
    const uint64_t oj = offsets[jj];
    const I len = (I)(offsets[jj + 1] - oj);
    const I rs = (I)(oj - o0 + j);  // block-local position of the read's first symbol
    const I P = (I)(oj + jj);       // the same position in the append's text
    const I C0 = (I)d_C[0], C1 = (I)d_C[1], C2 = (I)d_C[2], C3 = (I)d_C[3];
    const I nx = (I)n_ext;

    constexpr int G = 16 / (int)sizeof(IdxT);
    IdxT s[G];  // s[0]: the newest value (lowest position)
    int held = 0;
    auto push = [&](I pos, IdxT v) {
#pragma unroll
        for (int r = G - 1; r > 0; --r) s[r] = s[r - 1];
        s[0] = v;
        ++held;
        if ((pos & (G - 1)) == 0) {
            if (held == G) {
                if constexpr (G == 4) {
                    *reinterpret_cast<uint4*>(g + pos) = make_uint4(s[0], s[1], s[2], s[3]);
                } else {
                    *reinterpret_cast<ulonglong2*>(g + pos) = make_ulonglong2(s[0], s[1]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < G; ++r)
                    if (r < held) g[pos + r] = s[r];
            }
            held = 0;
        }
    };

    I i = (I)m_ext;
    push(rs + len, i);
    // the text word of the current position and the one below it, fetched
    // a word ahead so the walk never waits for the text
    I wcur = len > 0 ? (P + len - 1) / kPer : (I)0;
    uint32_t word = len > 0 ? __ldg(text + wcur) : 0u;
    uint32_t below = (len > 0 && wcur > 0) ? __ldg(text + wcur - 1) : 0u;
    for (I k = len; k > 0; --k) {
        const I t = P + k - 1;
        if (t / kPer != wcur) {  // one word down
            wcur = t / kPer;
            word = below;
            below = wcur > 0 ? __ldg(text + wcur - 1) : 0u;
        }
        const uint32_t c = (word >> (32u - kB - kB * (uint32_t)(t % kPer))) & ((1u << kB) - 1u);
        I Cc, in;
        if constexpr (kB == 2) {
            Cc = (c & 2) ? ((c & 1) ? C3 : C2) : ((c & 1) ? C1 : C0);
            in = occ_in_super_i<I, K>(blocks, c, i);
        } else {
            Cc = (I)__ldg(d_C + c);
            in = (I)DictLayout<kB, K>::in_super(blocks, c, i);
        }
        const I sup = kStage ? s_super[(i >> kSS) * kCodes + c] : (I)__ldg(super + (i >> kSS) * kCodes + c);
        i = Cc + sup + in;
        if (i > nx) {
            atomicOr(d_err, 8u);
            i = nx;
        }
        push(rs + k - 1, i);
    }
    // the lowest positions of the read, below its first complete group
#pragma unroll
    for (int r = 0; r < G; ++r)
        if (r < held) g[rs + r] = s[r];
}

// ComputeRanks for long reads, one thread per segment of seg_rows positions
// of a read (256 unless the tile shapes say otherwise), so a block of few
// long reads still runs many LF chains at once.  Segment q of read j covers
// positions [a, b) = [q seg_rows, min((q+1) seg_rows, len + 1)), the
// terminator at len.  The last segment starts, as
// Algorithm 2 does, from the terminator's rank start.  Any other segment first
// needs g at b exactly: backward search (Lemma 1 applied to the interval of
// old suffixes that start with P[b .. e)) over the L symbols from b on; once
// that interval is empty, its lower end is the number of old suffixes
// smaller than P[b ..] whatever follows e, which is g[b] (with L doubled while
// the L-mer still occurs in B_ext, and the exact chain from the terminator
// once e would pass the read's end).  From g[b] it steps down to a with
// Lemma 1, like the per-read kernel.  Reads of up to 2 seg_rows symbols take
// the per-read kernel.
constexpr uint32_t kProbe0 = 32;  // first backward-search window

template <class IdxT, bool kStage, int kB, int K>
__global__ void __launch_bounds__(kThreads) compute_ranks_seg_kernel(const uint32_t* __restrict__ text,
                                                                     const unsigned long long* __restrict__ offsets,
                                                                     unsigned long long j_begin,
                                                                     unsigned long long nreads, uint32_t segs,
                                                                     uint32_t seg_rows,
                                                                     const typename DictLayout<kB, K>::Block* blocks,
                                                                     const unsigned long long* __restrict__ super,
                                                                     const unsigned long long* __restrict__ d_C,
                                                                     unsigned long long n_ext,
                                                                     unsigned long long m_start,
                                                                     IdxT* __restrict__ g, uint32_t* __restrict__ d_err) {
    using I = IdxT;
    using D = DictLayout<kB, K>;
    constexpr int kSS = D::kSuperShift, kCodes = D::kCodes;
    constexpr uint32_t kPer = 32 / kB;
    extern __shared__ unsigned long long s_raw[];
    I* s_super = reinterpret_cast<I*>(s_raw);
    if (kStage) {
        const uint32_t words = ((uint32_t)(n_ext >> kSS) + 1) * kCodes;
        for (uint32_t x = threadIdx.x; x < words; x += kThreads) s_super[x] = (I)super[x];
        __syncthreads();
    }
    const uint64_t t = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t j = t / segs;
    const uint32_t q = (uint32_t)(t % segs);
    if (j >= nreads) return;
    const uint64_t jj = j_begin + j;
    const uint64_t o0 = offsets[j_begin];
    const uint64_t oj = offsets[jj];
    const I len = (I)(offsets[jj + 1] - oj);
    const I a = (I)q * seg_rows;
    if (a > len) return;  // this read has fewer segments
    const I b = min((I)(a + seg_rows), (I)(len + 1));
    const I rs = (I)(oj - o0 + j);  // block-local position of the read's first symbol
    const I P = (I)(oj + jj);       // the same position in the append's text
    const I nx = (I)n_ext;
    auto code_at = [&](I k) -> uint32_t {  // symbol at read position k < len
        const I tt = P + k;
        return (__ldg(text + tt / kPer) >> (32u - kB - kB * (uint32_t)(tt % kPer))) & ((1u << kB) - 1u);
    };
    const I C0 = (I)d_C[0], C1 = (I)d_C[1], C2 = (I)d_C[2], C3 = (I)d_C[3];
    // Lemma 1: rank of c P[k..] among the old suffixes from the rank i of P[k..]
    auto step = [&](uint32_t c, I i) -> I {
        I Cc;
        if constexpr (kB == 2) {
            Cc = (c & 2) ? ((c & 1) ? C3 : C2) : ((c & 1) ? C1 : C0);
        } else {
            Cc = (I)__ldg(d_C + c);
        }
        const I sup = kStage ? s_super[(i >> kSS) * kCodes + c] : (I)__ldg(super + (i >> kSS) * kCodes + c);
        I r = Cc + sup + (I)D::in_super(blocks, c, i);
        if (r > nx) {
            atomicOr(d_err, 8u);
            r = nx;
        }
        return r;
    };
    // the chain from the terminator (exact start) down to position `to`
    auto chain_from_end = [&](I to) -> I {
        I i = (I)m_start;
        for (I k = len; k > to; --k) i = step(code_at(k - 1), i);
        return i;
    };
    I i, top;  // i = g at position top
    if (b == len + 1) {
        i = (I)m_start;  // the segment holds the terminator
        top = len;
        g[rs + len] = i;
    } else {
        top = b;
        i = 0;
        for (uint64_t L = kProbe0;; L *= 4) {
            if ((uint64_t)b + L > (uint64_t)len) {
                i = chain_from_end(b);
                break;
            }
            I lo = 0, hi = nx;
            I k = (I)(b + L);
            for (; k > b && lo < hi; --k) {
                const uint32_t c = code_at(k - 1);
                lo = step(c, lo);
                hi = step(c, hi);
            }
            if (lo == hi) {  // no old suffix starts with P[k .. b + L): lo is exact from here
                for (; k > b; --k) lo = step(code_at(k - 1), lo);
                i = lo;
                break;
            }
        }
    }
    // the segment's own walk, the text word below fetched a word ahead
    if (top > a) {
        I wcur = (P + top - 1) / kPer;
        uint32_t word = __ldg(text + wcur);
        uint32_t below = wcur > 0 ? __ldg(text + wcur - 1) : 0u;
        for (I k = top; k > a; --k) {
            const I tt = P + k - 1;
            if (tt / kPer != wcur) {
                wcur = tt / kPer;
                word = below;
                below = wcur > 0 ? __ldg(text + wcur - 1) : 0u;
            }
            i = step((word >> (32u - kB - kB * (uint32_t)(tt % kPer))) & ((1u << kB) - 1u), i);
            g[rs + k - 1] = i;
        }
    }
}

// B_int and g_sa in one pass over SA_int (both index by SA_int[i]).  With
// ins_i0 set, it also writes Insert's plan: new symbol i lands on row
// r_i = g_sa[i] + i of the next dictionary (strictly increasing in i), and
// ins_i0[S] = |{i : r_i < S * 2^super_shift}| for S = 0 .. nsb, so the CTA
// that builds superblock S takes the new symbols [ins_i0[S], ins_i0[S+1]).
// Element i writes the entries S with r_{i-1} < S * 2^super_shift <= r_i
// (all S up to r_0 for i = 0; the last element also those past r_{n-1}).
// A thread takes kGather consecutive elements: their SA entries arrive as
// one vector, and all of their random reads (g, the text word and the
// terminator word of each) are in flight together.
constexpr int kGather = 4;

template <class IdxT, int kB>
__global__ void __launch_bounds__(kThreads) bint_gather_kernel(const uint32_t* __restrict__ text,
                                                               const uint32_t* __restrict__ term,
                                                               unsigned long long base,
                                                               const uint32_t* __restrict__ sa,
                                                               const IdxT* __restrict__ g, uint32_t n,
                                                               uint8_t* __restrict__ bint,
                                                               IdxT* __restrict__ gsa, uint32_t* __restrict__ ins_i0,
                                                               unsigned long long nsb, int super_shift) {
    const uint32_t i0 = (blockIdx.x * kThreads + threadIdx.x) * kGather;
    const bool whole = i0 + kGather <= n;
    uint32_t t[kGather];
    if (whole) {
        const uint4 s4 = *reinterpret_cast<const uint4*>(sa + i0);
        t[0] = s4.x, t[1] = s4.y, t[2] = s4.z, t[3] = s4.w;
    } else {
#pragma unroll
        for (int u = 0; u < kGather; ++u) t[u] = i0 + u < n ? sa[i0 + u] : 0u;
    }
    IdxT v[kGather];
    uint32_t code[kGather];
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
        t[u] = t[u] < n ? t[u] : 0u;
        const uint64_t P = base + t[u];
        v[u] = (i0 + u < n) ? g[t[u]] : (IdxT)0;
        code[u] = (t[u] == 0 || is_term(term, P - 1)) ? kBintDollar : text_code_b<kB>(text, P - 1);
    }
    if (whole) {
        *reinterpret_cast<uint32_t*>(bint + i0) = code[0] | (code[1] << 8) | (code[2] << 16) | (code[3] << 24);
        if constexpr (sizeof(IdxT) == 4) {
            *reinterpret_cast<uint4*>(gsa + i0) = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
            reinterpret_cast<ulonglong2*>(gsa + i0)[0] = make_ulonglong2(v[0], v[1]);
            reinterpret_cast<ulonglong2*>(gsa + i0)[1] = make_ulonglong2(v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int u = 0; u < kGather; ++u)
            if (i0 + u < n) {
                bint[i0 + u] = (uint8_t)code[u];
                gsa[i0 + u] = v[u];
            }
    }
    if (ins_i0 == nullptr) return;
    // r of the element before this thread's first: the previous lane's last
    // (every lane of the warp is still here: the grid is whole warps)
    unsigned long long r[kGather];
#pragma unroll
    for (int u = 0; u < kGather; ++u) r[u] = (unsigned long long)v[u] + i0 + u;
    unsigned long long prev = __shfl_up_sync(0xffffffffu, r[kGather - 1], 1);
    if (i0 >= n) return;
    if ((threadIdx.x & 31) == 0 && i0 > 0) {
        const uint32_t tp = sa[i0 - 1] < n ? sa[i0 - 1] : 0u;
        prev = (unsigned long long)g[tp] + (i0 - 1);
    }
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
        const uint32_t i = i0 + u;
        if (i >= n) break;
        const unsigned long long s_lo = i == 0 ? 0ull : (prev >> super_shift) + 1;
        const unsigned long long s_hi = min(r[u] >> super_shift, nsb);
        for (unsigned long long S = s_lo; S <= s_hi; ++S) ins_i0[S] = i;
        if (i == n - 1)
            for (unsigned long long S = (r[u] >> super_shift) + 1; S <= nsb; ++S) ins_i0[S] = n;
        prev = r[u];
    }
}

// rank(c, k) queries, codes 0..kCodes-1, or kCodes for the terminator.
template <int kB, int K>
__global__ void __launch_bounds__(kThreads) rank_batch_kernel(const typename DictLayout<kB, K>::Block* blocks,
                                                              const unsigned long long* __restrict__ super,
                                                              const uint8_t* __restrict__ codes,
                                                              const unsigned long long* __restrict__ ks,
                                                              unsigned long long q,
                                                              unsigned long long* __restrict__ out) {
    constexpr uint32_t kCodes = DictLayout<kB, K>::kCodes;
    const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= q) return;
    const uint32_t c = codes[i];
    const unsigned long long k = ks[i];
    if (c < kCodes) {
        out[i] = dict_rank<kB, K>(blocks, super, c, k);
    } else {  // terminators: every row before k that holds no symbol
        unsigned long long s = 0;
        for (uint32_t x = 0; x < kCodes; ++x) s += dict_rank<kB, K>(blocks, super, x, k);
        out[i] = k - s;
    }
}

// FM-index backward search (Lemma 1 applied to a pattern instead of a new
// read): the rows of the suffixes that start with P[k..] are [lo, hi); one
// step per symbol, right to left, from [0, n).  hi - lo counts P.  A byte
// outside the alphabet (code table in shared memory) counts zero.
template <int kB, int K>
__global__ void __launch_bounds__(kThreads) count_kernel(const typename DictLayout<kB, K>::Block* blocks,
                                                         const unsigned long long* __restrict__ super,
                                                         const unsigned long long* __restrict__ d_C,
                                                         unsigned long long n, Alphabet16 alpha, int sigma,
                                                         const uint8_t* __restrict__ pats,
                                                         const unsigned long long* __restrict__ offs,
                                                         unsigned long long q, unsigned long long* __restrict__ out) {
    constexpr uint32_t kNot = 0xFFu;
    __shared__ uint8_t code_of[256];
    code_of[threadIdx.x] = kNot;
    __syncthreads();
    if ((int)threadIdx.x < sigma) code_of[alpha.a[threadIdx.x]] = (uint8_t)threadIdx.x;
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= q) return;
    unsigned long long lo = 0, hi = n;
    for (uint64_t k = offs[i + 1]; k > offs[i] && lo < hi; --k) {
        const uint32_t c = code_of[pats[k - 1]];
        if (c == kNot) {  // not in the alphabet: no occurrence
            lo = hi = 0;
            break;
        }
        const unsigned long long Cc = __ldg(d_C + c);
        lo = Cc + dict_rank<kB, K>(blocks, super, c, lo);
        hi = Cc + dict_rank<kB, K>(blocks, super, c, hi);
    }
    out[i] = hi > lo ? hi - lo : 0ull;
}

// The read-back of the 2-bit dictionary: one 64-row part per thread, 64
// output bytes written as four 16-byte stores when the part is whole; rows
// [r0, r1), r0 a multiple of 64.
template <int K>
__global__ void __launch_bounds__(kThreads) unpack_kernel(const unsigned long long* __restrict__ words,
                                                          unsigned long long r0, unsigned long long r1,
                                                          uint32_t alpha4, uint8_t* __restrict__ out) {
    const uint64_t part = (r0 >> kOccShift) + (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t row0 = part << kOccShift;
    if (row0 >= r1) return;
    const unsigned long long* p = words + (part / K) * Occ<K>::kWords + 3 * (part % K);
    const unsigned long long lo = p[0], hi = p[1], dm = p[2];
    uint32_t wd[16];
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        uint32_t x = 0;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            const uint32_t q = 4 * w + q4;
            const uint32_t c = (uint32_t)((lo >> q) & 1ull) | ((uint32_t)((hi >> q) & 1ull) << 1);
            const uint32_t byte = ((dm >> q) & 1ull) ? (uint32_t)'$' : ((alpha4 >> (8 * c)) & 0xFFu);
            x |= byte << (8 * q4);
        }
        wd[w] = x;
    }
    if (row0 + kOccSpan <= r1) {
        uint4* dst = reinterpret_cast<uint4*>(out + row0);
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = make_uint4(wd[4 * v], wd[4 * v + 1], wd[4 * v + 2], wd[4 * v + 3]);
    } else {
        for (uint32_t q = 0; q < (uint32_t)(r1 - row0); ++q) out[row0 + q] = (uint8_t)(wd[q >> 2] >> (8 * (q & 3)));
    }
}

// The read-back for the 4-bit dictionary (5 to 16 symbols).
__global__ void __launch_bounds__(kThreads) unpack_w_kernel(const OccBlockW* __restrict__ blocks,
                                                            unsigned long long r0, unsigned long long r1,
                                                            Alphabet16 alpha, uint8_t* __restrict__ out) {
    // one occurrence block (64 rows) per thread, as for unpack_kernel; the
    // alphabet is looked up from shared memory
    __shared__ uint8_t sym_byte[kSigmaW];
    if (threadIdx.x < kSigmaW) sym_byte[threadIdx.x] = alpha.a[threadIdx.x];
    __syncthreads();
    const uint64_t b = (r0 >> kOccShift) + (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t row0 = b << kOccShift;
    if (row0 >= r1) return;
    const OccBlockW blk = blocks[b];
    uint32_t words[16];
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        uint32_t x = 0;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            const uint32_t q = 4 * w + q4;
            const uint32_t c = (uint32_t)(blk.sym[q >> 4] >> (4 * (q & 15))) & 15u;
            const uint32_t byte = ((blk.dmask >> q) & 1ull) ? (uint32_t)'$' : (uint32_t)sym_byte[c];
            x |= byte << (8 * q4);
        }
        words[w] = x;
    }
    if (row0 + kOccSpan <= r1) {
        uint4* dst = reinterpret_cast<uint4*>(out + row0);
#pragma unroll
        for (int v = 0; v < 4; ++v)
            dst[v] = make_uint4(words[4 * v], words[4 * v + 1], words[4 * v + 2], words[4 * v + 3]);
    } else {
        for (uint32_t q = 0; q < (uint32_t)(r1 - row0); ++q) out[row0 + q] = (uint8_t)(words[q >> 2] >> (8 * (q & 3)));
    }
}

uint32_t alpha4_of(const Alphabet16& alpha) {
    uint32_t a4 = 0;
    for (int a = 0; a < 4; ++a) a4 |= (uint32_t)alpha.a[a] << (8 * a);
    return a4;
}

template <class IdxT, int kB, int K>
void compute_ranks_launch(Launcher& L, const uint32_t* text, const uint64_t* d_offsets, uint64_t j_begin,
                          uint64_t nreads, uint64_t max_len, uint32_t seg_rows, double bytes, const void* blocks,
                          const unsigned long long* super, const unsigned long long* d_C, uint64_t n_ext,
                          uint64_t m_ext, IdxT* g, uint32_t* d_err) {
    using D = DictLayout<kB, K>;
    using Block = typename D::Block;
    const size_t stage = ((n_ext >> D::kSuperShift) + 1) * D::kCodes * sizeof(IdxT);
    const bool staged = stage <= kSuperStageBytes;
    const auto* offs = reinterpret_cast<const unsigned long long*>(d_offsets);
    if (max_len > 2ull * seg_rows) {  // long reads: one thread per segment
        const uint32_t segs = (uint32_t)(max_len / seg_rows + 1);
        auto* const kern = staged ? compute_ranks_seg_kernel<IdxT, true, kB, K>
                                  : compute_ranks_seg_kernel<IdxT, false, kB, K>;
        SBWT_LAUNCH(L, "compute_ranks", bytes, 0, nullptr, kern, ceil_div_u(nreads * segs, kThreads), kThreads,
                    staged ? stage : 0, text, offs, (unsigned long long)j_begin, (unsigned long long)nreads, segs,
                    seg_rows, static_cast<const Block*>(blocks), super, d_C, (unsigned long long)n_ext,
                    (unsigned long long)m_ext, g, d_err);
        return;
    }
    auto* const kern = staged ? compute_ranks_kernel<IdxT, true, kB, K> : compute_ranks_kernel<IdxT, false, kB, K>;
    SBWT_LAUNCH(L, "compute_ranks", bytes, 0, nullptr, kern, ceil_div_u(nreads, kThreads), kThreads,
                staged ? stage : 0, text, offs, (unsigned long long)j_begin, (unsigned long long)nreads,
                static_cast<const Block*>(blocks), super, d_C, (unsigned long long)n_ext, (unsigned long long)m_ext,
                g, d_err);
}

// Sectors a rank query of the 2-bit dictionary reads: one for sampling 64,
// the counts plus the parts before the row for 128 and 256 (on average half
// of them, rounded up to whole sectors).
double rank_query_bytes(int code_bits, int occ_k) {
    if (code_bits == 4) return 64.0;
    return occ_k == 1 ? 32.0 : (occ_k == 2 ? 64.0 : 96.0);
}

}  // namespace

void launch_bint(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, const uint32_t* sa,
                 uint32_t n, uint8_t* bint) {
    if (n == 0) return;
    SBWT_LAUNCH(L, "extract_bint", (double)n * (4 + 1 + 4 + 4), 0, nullptr, bint_kernel, ceil_div_u(n, kThreads),
                kThreads, 0, text, term, (unsigned long long)base, sa, n, bint);
}

template <class IdxT>
void launch_compute_ranks(Launcher& L, const uint32_t* text, const uint64_t* d_offsets, uint64_t j_begin,
                          uint64_t nreads, uint64_t n_int, uint64_t max_len, const void* blocks,
                          const unsigned long long* super, const unsigned long long* d_C, uint64_t n_ext,
                          uint64_t m_ext, IdxT* g, uint32_t* d_err, int code_bits, int occ_k, uint32_t seg_rows) {
    if (nreads == 0) return;
    // per suffix: one rank query's sectors, a g write, the text codes
    const double bytes = (double)(n_int - nreads) * rank_query_bytes(code_bits, occ_k) +
                         (double)n_int * sizeof(IdxT) + n_int * code_bits / 8.0 + 16.0 * nreads;
    if (code_bits == 4) {
        compute_ranks_launch<IdxT, 4, 1>(L, text, d_offsets, j_begin, nreads, max_len, seg_rows, bytes, blocks, super, d_C,
                                         n_ext, m_ext, g, d_err);
    } else if (occ_k == 4) {
        compute_ranks_launch<IdxT, 2, 4>(L, text, d_offsets, j_begin, nreads, max_len, seg_rows, bytes, blocks, super, d_C,
                                         n_ext, m_ext, g, d_err);
    } else if (occ_k == 2) {
        compute_ranks_launch<IdxT, 2, 2>(L, text, d_offsets, j_begin, nreads, max_len, seg_rows, bytes, blocks, super, d_C,
                                         n_ext, m_ext, g, d_err);
    } else {
        compute_ranks_launch<IdxT, 2, 1>(L, text, d_offsets, j_begin, nreads, max_len, seg_rows, bytes, blocks, super, d_C,
                                         n_ext, m_ext, g, d_err);
    }
}

template <class IdxT>
void launch_bint_gather(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, const uint32_t* sa,
                        const IdxT* g, uint32_t n, uint8_t* bint, IdxT* gsa, int code_bits, uint32_t* ins_i0,
                        uint64_t nsb, int super_shift) {
    if (n == 0) return;
    // per suffix: SA_int read, one text word and one bitmap word (random), a
    // random g sector, B_int and g_sa writes; 4 bytes per plan entry
    auto* const kern = code_bits == 4 ? bint_gather_kernel<IdxT, 4> : bint_gather_kernel<IdxT, 2>;
    SBWT_LAUNCH(L, "bint_gather", (double)n * (4 + 4 + 4 + 32 + 1 + sizeof(IdxT)) + (ins_i0 ? 4.0 * (nsb + 1) : 0.0),
                0, nullptr, kern, ceil_div_u(n, (uint64_t)kThreads * kGather), kThreads, 0, text, term,
                (unsigned long long)base, sa, g,
                n, bint, gsa, ins_i0, (unsigned long long)nsb, super_shift);
}

namespace {
template <int K>
void rank_batch_k(Launcher& L, const void* blocks, const unsigned long long* super, const uint8_t* codes,
                  const unsigned long long* ks, uint64_t q, unsigned long long* out) {
    SBWT_LAUNCH(L, "rank_query", (double)q * (1 + 8 + rank_query_bytes(2, K) + 8 + 8), 0, nullptr,
                (rank_batch_kernel<2, K>), ceil_div_u(q, kThreads), kThreads, 0,
                static_cast<const unsigned long long*>(blocks), super, codes, ks, (unsigned long long)q, out);
}
template <int K>
void count_k(Launcher& L, const void* blocks, const unsigned long long* super, const unsigned long long* d_C,
             uint64_t n, const Alphabet16& alpha, int sigma, const uint8_t* pats, const uint64_t* offs, uint64_t q,
             uint64_t total_len, unsigned long long* out) {
    SBWT_LAUNCH(L, "count_query", (double)total_len * (1 + 2 * (rank_query_bytes(2, K) + 8)) + 16.0 * q, 0,
                nullptr, (count_kernel<2, K>), ceil_div_u(q, kThreads), kThreads, 0,
                static_cast<const unsigned long long*>(blocks), super, d_C, (unsigned long long)n, alpha, sigma, pats,
                reinterpret_cast<const unsigned long long*>(offs), (unsigned long long)q, out);
}
template <int K>
void unpack_k(Launcher& L, const void* blocks, uint64_t r0, uint64_t r1, const Alphabet16& alpha, uint8_t* out,
              uint64_t nparts) {
    SBWT_LAUNCH(L, "unpack_bwt", (double)(r1 - r0) * (1 + 0.375 + 0.125 / K), 0, nullptr, unpack_kernel<K>,
                ceil_div_u(nparts, kThreads), kThreads, 0, static_cast<const unsigned long long*>(blocks),
                (unsigned long long)r0, (unsigned long long)r1, alpha4_of(alpha), out);
}
}  // namespace

void launch_rank_batch(Launcher& L, const void* blocks, const unsigned long long* super, const uint8_t* codes,
                       const unsigned long long* ks, uint64_t q, unsigned long long* out, int code_bits, int occ_k) {
    if (q == 0) return;
    if (code_bits == 4) {
        SBWT_LAUNCH(L, "rank_query", (double)q * (1 + 8 + 64 + 8 + 8), 0, nullptr, (rank_batch_kernel<4, 1>),
                    ceil_div_u(q, kThreads), kThreads, 0, static_cast<const OccBlockW*>(blocks), super, codes, ks,
                    (unsigned long long)q, out);
    } else if (occ_k == 4) {
        rank_batch_k<4>(L, blocks, super, codes, ks, q, out);
    } else if (occ_k == 2) {
        rank_batch_k<2>(L, blocks, super, codes, ks, q, out);
    } else {
        rank_batch_k<1>(L, blocks, super, codes, ks, q, out);
    }
}

void launch_count(Launcher& L, const void* blocks, const unsigned long long* super, const unsigned long long* d_C,
                  uint64_t n, const Alphabet16& alpha, int sigma, const uint8_t* pats, const uint64_t* offs,
                  uint64_t q, uint64_t total_len, unsigned long long* out, int code_bits, int occ_k) {
    if (q == 0) return;
    if (code_bits == 4) {
        SBWT_LAUNCH(L, "count_query", (double)total_len * (1 + 2 * 72) + 16.0 * q, 0, nullptr, (count_kernel<4, 1>),
                    ceil_div_u(q, kThreads), kThreads, 0, static_cast<const OccBlockW*>(blocks), super, d_C,
                    (unsigned long long)n, alpha, sigma, pats, reinterpret_cast<const unsigned long long*>(offs),
                    (unsigned long long)q, out);
    } else if (occ_k == 4) {
        count_k<4>(L, blocks, super, d_C, n, alpha, sigma, pats, offs, q, total_len, out);
    } else if (occ_k == 2) {
        count_k<2>(L, blocks, super, d_C, n, alpha, sigma, pats, offs, q, total_len, out);
    } else {
        count_k<1>(L, blocks, super, d_C, n, alpha, sigma, pats, offs, q, total_len, out);
    }
}

void launch_unpack(Launcher& L, const void* blocks, uint64_t r0, uint64_t r1, const Alphabet16& alpha, uint8_t* out,
                   int code_bits, int occ_k) {
    if (r1 <= r0) return;
    const uint64_t nparts = ((r1 - 1) >> kOccShift) - (r0 >> kOccShift) + 1;
    if (code_bits == 4) {
        SBWT_LAUNCH(L, "unpack_bwt", (double)(r1 - r0) * (1 + 1.0), 0, nullptr, unpack_w_kernel,
                    ceil_div_u(nparts, kThreads), kThreads, 0, static_cast<const OccBlockW*>(blocks),
                    (unsigned long long)r0, (unsigned long long)r1, alpha, out);
    } else if (occ_k == 4) {
        unpack_k<4>(L, blocks, r0, r1, alpha, out, nparts);
    } else if (occ_k == 2) {
        unpack_k<2>(L, blocks, r0, r1, alpha, out, nparts);
    } else {
        unpack_k<1>(L, blocks, r0, r1, alpha, out, nparts);
    }
}

template void launch_compute_ranks<uint32_t>(Launcher&, const uint32_t*, const uint64_t*, uint64_t, uint64_t,
                                             uint64_t, uint64_t, const void*, const unsigned long long*,
                                             const unsigned long long*, uint64_t, uint64_t, uint32_t*, uint32_t*, int,
                                             int, uint32_t);
template void launch_compute_ranks<unsigned long long>(Launcher&, const uint32_t*, const uint64_t*, uint64_t,
                                                       uint64_t, uint64_t, uint64_t, const void*,
                                                       const unsigned long long*, const unsigned long long*, uint64_t,
                                                       uint64_t, unsigned long long*, uint32_t*, int, int, uint32_t);
template void launch_bint_gather<uint32_t>(Launcher&, const uint32_t*, const uint32_t*, uint64_t, const uint32_t*,
                                           const uint32_t*, uint32_t, uint8_t*, uint32_t*, int, uint32_t*, uint64_t,
                                           int);
template void launch_bint_gather<unsigned long long>(Launcher&, const uint32_t*, const uint32_t*, uint64_t,
                                                     const uint32_t*, const unsigned long long*, uint32_t, uint8_t*,
                                                     unsigned long long*, int, uint32_t*, uint64_t, int);

}  // namespace sbwt
