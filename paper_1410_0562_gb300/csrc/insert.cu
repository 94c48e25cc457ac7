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
// One CTA builds one superblock (1024 occurrence blocks of 64 rows), four
// consecutive blocks per thread (or one per thread, 1024 threads, when the
// new rows are at least a quarter of the result: the splicing then needs the
// parallelism more than the binary searches need sharing).  For output
// block b (rows [o, o+64)) a binary search finds i0 = |{i : g_sa[i] + i <
// o}|; the block then holds the old rows
// starting at o - i0, into which the new symbols with final rows in [o, o+64)
// are spliced in ascending order.  Per-block counts are scanned across the
// CTA for the 16-bit block counters; a one-CTA pass scans the superblock
// totals into the 64-bit superblock counters and C[] (Lemma 1's C[c] counts
// every smaller symbol, the terminators included).
#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;

struct Window {
    unsigned long long w0, w1, dm;
};

// 64 old rows starting at row s (rows past the old end read as zero).
__device__ __forceinline__ Window old_window(const OccBlock* __restrict__ old_blocks, uint64_t nb_old, uint64_t s) {
    const uint64_t bs = s >> kOccShift;
    const uint32_t off = (uint32_t)(s & (kOccSpan - 1));
    const OccBlock& A = old_blocks[bs];
    const unsigned long long a0 = A.sym[0], a1 = A.sym[1], da = A.dmask;
    unsigned long long a2 = 0, a3 = 0, db = 0;
    if (bs + 1 < nb_old) {
        const OccBlock& B = old_blocks[bs + 1];
        a2 = B.sym[0];
        a3 = B.sym[1];
        db = B.dmask;
    }
    Window w;
    const uint32_t sh = 2 * off;  // 0 .. 126 bits
    if (sh == 0) {
        w.w0 = a0;
        w.w1 = a1;
    } else if (sh < 64) {
        w.w0 = (a0 >> sh) | (a1 << (64 - sh));
        w.w1 = (a1 >> sh) | (a2 << (64 - sh));
    } else if (sh == 64) {
        w.w0 = a1;
        w.w1 = a2;
    } else {
        const uint32_t s2 = sh - 64;
        w.w0 = (a1 >> s2) | (a2 << (64 - s2));
        w.w1 = (a2 >> s2) | (a3 << (64 - s2));
    }
    w.dm = off == 0 ? da : ((da >> off) | (db << (64 - off)));
    return w;
}

// Splice one row holding `code` (terminator when dollar) in at position p of
// the 64-row window; rows p.. move up by one and row 63 falls off.
__device__ __forceinline__ void splice(Window& w, uint32_t p, uint32_t code, uint32_t dollar) {
    if (p < 32) {
        w.w1 = (w.w1 << 2) | (w.w0 >> 62);
        const unsigned long long keep = low_bits(2 * p);
        w.w0 = (w.w0 & keep) | ((unsigned long long)code << (2 * p)) | ((w.w0 & ~keep) << 2);
    } else {
        const uint32_t q = p - 32;
        const unsigned long long keep = low_bits(2 * q);
        w.w1 = (w.w1 & keep) | ((unsigned long long)code << (2 * q)) | ((w.w1 & ~keep) << 2);
    }
    const unsigned long long keepd = low_bits(p);
    w.dm = (w.dm & keepd) | ((unsigned long long)dollar << p) | ((w.dm & ~keepd) << 1);
}

// kPer output blocks per thread (kBlocksPerSuper / kPer threads): 4 for a
// block of sparse new rows (one binary search serves four blocks), 1 when
// new rows are dense (four times the threads for the splicing).
template <class IdxT, int kPer>
__global__ void __launch_bounds__(kBlocksPerSuper / kPer) insert_kernel(const OccBlock* __restrict__ old_blocks,
                                                          unsigned long long n_ext, const uint8_t* __restrict__ bint,
                                                          const IdxT* __restrict__ gsa, unsigned long long n_int,
                                                          OccBlock* __restrict__ new_blocks,
                                                          unsigned long long n_new, uint32_t* __restrict__ sb_tot) {
    const uint64_t nb_new = (n_new >> kOccShift) + 1;
    const uint64_t nb_old = (n_ext >> kOccShift) + 1;
    constexpr int kPerThread = kPer, kT = kBlocksPerSuper / kPer;
    const uint64_t b0 = (uint64_t)blockIdx.x * kBlocksPerSuper + (uint64_t)threadIdx.x * kPerThread;
    Window win[kPerThread];
    uint32_t cnt[kPerThread][4];
#pragma unroll
    for (int bb = 0; bb < kPerThread; ++bb) {
        win[bb].w0 = win[bb].w1 = win[bb].dm = 0;
        cnt[bb][0] = cnt[bb][1] = cnt[bb][2] = cnt[bb][3] = 0;
    }
    if (b0 < nb_new) {
        uint64_t lo = 0, hi = n_int;  // first i with g_sa[i] + i >= o
        const uint64_t o0 = b0 << kOccShift;
        while (lo < hi) {
            const uint64_t mid = lo + ((hi - lo) >> 1);
            if ((uint64_t)gsa[mid] + mid < o0) lo = mid + 1; else hi = mid;
        }
        uint64_t i = lo;
#pragma unroll
        for (int bb = 0; bb < kPerThread; ++bb) {
            const uint64_t b = b0 + bb;
            if (b >= nb_new) break;
            const uint64_t o = b << kOccShift;
            // o - i old rows precede this block; clamped so a bad g_sa can
            // never send the window past the old dictionary
            const uint64_t s_old = o >= i ? min((unsigned long long)(o - i), n_ext) : 0ull;
            Window w = old_window(old_blocks, nb_old, s_old);
            while (i < n_int) {
                const uint64_t row = (uint64_t)gsa[i] + i;
                if (row >= o + kOccSpan) break;
                const uint8_t x = bint[i];
                splice(w, (uint32_t)(row - o), x == kBintDollar ? 0u : x, x == kBintDollar ? 1u : 0u);
                ++i;
            }
            const uint32_t valid = n_new > o ? (uint32_t)min((unsigned long long)kOccSpan, n_new - o) : 0u;
            const unsigned long long v0 = low_bits(2 * min(valid, 32u));
            const unsigned long long v1 = valid > 32 ? low_bits(2 * (valid - 32)) : 0ull;
            w.w0 &= v0;
            w.w1 &= v1;
            w.dm &= low_bits(valid);
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c)
                cnt[bb][c] = __popcll(match_code(w.w0, c) & v0) + __popcll(match_code(w.w1, c) & v1);
            cnt[bb][0] -= __popcll(w.dm);
            win[bb] = w;
        }
    }
    // 16-bit block counters: exclusive scan of the per-thread totals.
    unsigned long long t01 = 0, t23 = 0;
#pragma unroll
    for (int bb = 0; bb < kPerThread; ++bb) {
        t01 += (unsigned long long)cnt[bb][0] | ((unsigned long long)cnt[bb][1] << 32);
        t23 += (unsigned long long)cnt[bb][2] | ((unsigned long long)cnt[bb][3] << 32);
    }
    unsigned long long tot01, tot23;
    const unsigned long long e01 = cta_exclusive_scan<SumOp, kT>(t01, tot01);
    const unsigned long long e23 = cta_exclusive_scan<SumOp, kT>(t23, tot23);
    uint32_t pref[4] = {(uint32_t)e01, (uint32_t)(e01 >> 32), (uint32_t)e23, (uint32_t)(e23 >> 32)};
#pragma unroll
    for (int bb = 0; bb < kPerThread; ++bb) {
        const uint64_t b = b0 + bb;
        if (b >= nb_new) break;
        OccBlock out;
        out.sym[0] = win[bb].w0;
        out.sym[1] = win[bb].w1;
        out.dmask = win[bb].dm;
        out.cnt = (unsigned long long)pref[0] | ((unsigned long long)pref[1] << 16) |
                  ((unsigned long long)pref[2] << 32) | ((unsigned long long)pref[3] << 48);
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(new_blocks + b);
        dst[0] = make_ulonglong2(out.sym[0], out.sym[1]);
        dst[1] = make_ulonglong2(out.dmask, out.cnt);
#pragma unroll
        for (int c = 0; c < 4; ++c) pref[c] += cnt[bb][c];
    }
    if (threadIdx.x == 0) {
        uint32_t* t = sb_tot + 4ull * blockIdx.x;
        t[0] = (uint32_t)tot01;
        t[1] = (uint32_t)(tot01 >> 32);
        t[2] = (uint32_t)tot23;
        t[3] = (uint32_t)(tot23 >> 32);
    }
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
__device__ __forceinline__ WindowW old_window_w(const OccBlockW* __restrict__ old_blocks, uint64_t nb_old, uint64_t s) {
    const uint64_t bs = s >> kOccShift;
    const uint32_t off = (uint32_t)(s & (kOccSpan - 1));
    const OccBlockW& A = old_blocks[bs];
    unsigned long long x[9];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = A.sym[k];
    unsigned long long da = A.dmask, db = 0;
#pragma unroll
    for (int k = 4; k < 9; ++k) x[k] = 0;
    if (bs + 1 < nb_old) {
        const OccBlockW& B = old_blocks[bs + 1];
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

template <class IdxT>
__global__ void __launch_bounds__(kThreads) insert_w_kernel(const OccBlockW* __restrict__ old_blocks,
                                                            unsigned long long n_ext, const uint8_t* __restrict__ bint,
                                                            const IdxT* __restrict__ gsa, unsigned long long n_int,
                                                            OccBlockW* __restrict__ new_blocks,
                                                            unsigned long long n_new, unsigned long long nsb,
                                                            uint32_t* __restrict__ sb_tot) {
    __shared__ uint32_t warp_tot[kThreads / 32][kSigmaW];
    const uint64_t nb_new = (n_new >> kOccShift) + 1;
    const uint64_t nb_old = (n_ext >> kOccShift) + 1;
    const uint64_t b = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
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
        w = old_window_w(old_blocks, nb_old, s_old);
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

template <class IdxT>
void launch_insert(Launcher& L, const void* old_blocks, uint64_t n_ext, const uint8_t* bint, const IdxT* gsa,
                   uint64_t n_int, void* new_blocks, unsigned long long* new_super, unsigned long long* new_C,
                   uint64_t m_new, uint32_t* sb_tot, int code_bits) {
    const uint64_t n_new = n_ext + n_int;
    // the superblock scan's per-chunk totals live after the superblock totals
    const uint64_t nsb_all = dict_supers_of(n_new, code_bits);
    unsigned long long* chunk_tot =
        reinterpret_cast<unsigned long long*>(sb_tot + ((nsb_all * dict_codes(code_bits) + 3) & ~3ull));
    if (code_bits == 4) {
        const uint64_t nsb = dict_supers_w(n_new);
        const double bytes = 64.0 * dict_blocks(n_ext) + (1.0 + sizeof(IdxT)) * n_int + 64.0 * dict_blocks(n_new);
        SBWT_LAUNCH(L, "insert_merge", bytes, 0, nullptr, insert_w_kernel<IdxT>,
                    ceil_div_u(nsb * kBlocksPerSuperW, kThreads), kThreads, 0,
                    static_cast<const OccBlockW*>(old_blocks), (unsigned long long)n_ext, bint, gsa,
                    (unsigned long long)n_int, static_cast<OccBlockW*>(new_blocks), (unsigned long long)n_new,
                    (unsigned long long)nsb, sb_tot);
        super_scan<kSigmaW>(L, sb_tot, nsb, new_super, new_C, m_new, chunk_tot);
        return;
    }
    const uint64_t nsb = dict_supers(n_new);
    const double bytes = 32.0 * dict_blocks(n_ext) + (1.0 + sizeof(IdxT)) * n_int + 32.0 * dict_blocks(n_new);
    // dense new rows (at least a quarter of the result): one block per thread
    const bool dense = 4 * n_int >= n_new;
    auto* const kern = dense ? insert_kernel<IdxT, 1> : insert_kernel<IdxT, 4>;
    SBWT_LAUNCH(L, "insert_merge", bytes, 0, nullptr, kern, (unsigned)nsb, dense ? kBlocksPerSuper : kThreads, 0,
                static_cast<const OccBlock*>(old_blocks), (unsigned long long)n_ext, bint, gsa,
                (unsigned long long)n_int, static_cast<OccBlock*>(new_blocks), (unsigned long long)n_new, sb_tot);
    super_scan<4>(L, sb_tot, nsb, new_super, new_C, m_new, chunk_tot);
}

template void launch_insert<uint32_t>(Launcher&, const void*, uint64_t, const uint8_t*, const uint32_t*, uint64_t,
                                      void*, unsigned long long*, unsigned long long*, uint64_t, uint32_t*, int);
template void launch_insert<unsigned long long>(Launcher&, const void*, uint64_t, const uint8_t*,
                                                const unsigned long long*, uint64_t, void*, unsigned long long*,
                                                unsigned long long*, uint64_t, uint32_t*, int);

}  // namespace sbwt
