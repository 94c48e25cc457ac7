// suffix_sort.cu -- ConstructSA of one block (Algorithm 1; Section 3 of
// arXiv 1410.0562 asks for any suffix sort and uses an MSD radix sort over
// packed symbols that sieves out finished suffixes).  Here: prefix doubling
// over the hand-written radix sort, with the sieve.
//
// Suffix order (Section 2): symbols compare by code; a suffix that reaches
// its terminator first is smaller; two suffixes that reach their terminators
// at the same offset compare by read index ($_j order), which inside a block
// is the order of their text positions.
//
// 1. Initial key of the suffix at block position t: its first 29 codes,
//    MSB first, with codes at and past its terminator zeroed, then
//    min(len, 29) in the low 5 bits, len = distance to the terminator.
//    Equal keys with len < 29 end at the same offset, so the stable sort
//    (values = t in increasing order) already puts them in read order: each
//    is a finished singleton.  Keys with len >= 29 that are equal form the
//    unsorted groups.
// 2. rank[t] = index of the first row of t's group (the Larsson-Sadakane
//    convention), so ranks stay valid while groups split in later rounds.
// 3. Round with offset h (29, 58, ...): only members of unsorted groups
//    (the sieve) are re-sorted, by (rank[t], rank[t + h]); t + h never leaves
//    the read because an unsorted member has len >= h.  Sorting them as one
//    list by that composite key keeps groups in place, so the k-th sorted
//    element goes to the k-th active row.  Rounds continue until the
//    resolved prefix exceeds the longest read of the block.
// At the end rank[] is the inverse suffix array of the block.
//
// After each sort one single-pass kernel does the bookkeeping: group heads,
// the running max of head rows (each element's group head), the active
// flags and their running count (the compaction offsets), with both scans
// carried across tiles by decoupled look-back; it writes SA, rank and the
// compacted list of unsorted members.  The key kernels also build the digit
// histograms of the sort that follows.
#include <algorithm>

#include "sbwt_internal.cuh"
#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kH0 = 29;
constexpr int kGItems = 16;
constexpr int kGTile = kThreads * kGItems;  // elements per group-kernel tile

// Counter slots (one tile counter per group launch).
constexpr int kSlotInit = 0;

__device__ __forceinline__ unsigned long long initial_key(const uint32_t* __restrict__ text,
                                                          const uint32_t* __restrict__ term, uint64_t P) {
    // distance to the terminator, capped at kH0 (terminator bitmap window)
    const uint64_t tw = P >> 5;
    const unsigned long long tb = (((unsigned long long)term[tw + 1] << 32) | term[tw]) >> (P & 31);
    const unsigned long long near = tb & ((1ull << kH0) - 1);
    const uint32_t len = near ? (uint32_t)(__ffsll((long long)near) - 1) : kH0;
    // 32 codes from P, MSB first
    const uint64_t wi = P >> 4;
    const uint32_t s = 2u * (uint32_t)(P & 15);
    const unsigned long long hi = ((unsigned long long)text[wi] << 32) | text[wi + 1];
    const unsigned long long lo = text[wi + 2];
    const unsigned long long v = (hi << s) | ((lo << s) >> 32);
    unsigned long long k58 = v >> 6;  // codes P .. P+28
    if (len < kH0) k58 &= ~((1ull << (2 * (kH0 - len))) - 1ull);
    return (k58 << 5) | len;
}

__global__ void __launch_bounds__(kThreads) sa_init_keys_kernel(const uint32_t* __restrict__ text,
                                                                const uint32_t* __restrict__ term,
                                                                unsigned long long base, uint32_t n,
                                                                unsigned long long* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ d_n,
                                                                uint32_t* __restrict__ ghist, int passes) {
    __shared__ uint32_t h[kRadixMaxPasses * kRadixBins];
    for (int i = threadIdx.x; i < passes * kRadixBins; i += kThreads) h[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = n;
    __syncthreads();
    for (uint32_t t = blockIdx.x * kThreads + threadIdx.x; t < n; t += gridDim.x * kThreads) {
        const unsigned long long key = initial_key(text, term, base + t);
        keys[t] = key;
        vals[t] = t;
        radix_hist_add(h, key, 0, passes);
    }
    __syncthreads();
    radix_hist_flush<kThreads>(h, ghist, passes);
}

__global__ void __launch_bounds__(kThreads) sa_round_keys_kernel(const uint32_t* __restrict__ act_suf,
                                                                 const uint32_t* __restrict__ d_cnt,
                                                                 const uint32_t* __restrict__ rank, uint32_t h,
                                                                 uint32_t n, int bits,
                                                                 unsigned long long* __restrict__ keys,
                                                                 uint32_t* __restrict__ vals,
                                                                 uint32_t* __restrict__ ghist, int passes,
                                                                 uint32_t* __restrict__ d_err) {
    __shared__ uint32_t hs[kRadixMaxPasses * kRadixBins];
    for (int i = threadIdx.x; i < passes * kRadixBins; i += kThreads) hs[i] = 0;
    __syncthreads();
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
        const unsigned long long key = ((unsigned long long)here << bits) | next;
        keys[k] = key;
        vals[k] = t;
        radix_hist_add(hs, key, 0, passes);
    }
    __syncthreads();
    radix_hist_flush<kThreads>(hs, ghist, passes);
}

// Group bookkeeping after a sort, one tile of kGTile elements per step.
// Element i of the sorted list (keys, vals) sits on row pos(i) of the block
// SA: pos(i) = i after the initial sort, act_pos[i] after a round.  Writes
// SA[pos] = t, rank[t] = row of t's group head, and appends the members of
// groups with two or more elements to (act_pos_out, act_suf_out); the
// number appended goes to *d_cnt_out.
template <bool kRound>
__global__ void __launch_bounds__(kThreads) sa_groups_kernel(
    const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ act_pos_in, const uint32_t* __restrict__ d_cnt, uint32_t n_block,
    uint32_t* __restrict__ sa, uint32_t* __restrict__ rank, uint32_t* __restrict__ act_pos_out,
    uint32_t* __restrict__ act_suf_out, uint32_t* __restrict__ d_cnt_out, unsigned long long* __restrict__ lookback,
    uint32_t* __restrict__ tile_counter, unsigned long long epoch, uint32_t* __restrict__ d_err) {
    __shared__ uint32_t s_tile, s_pmax, s_psum;
    const uint32_t n = kRound ? *d_cnt : n_block;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kGTile - 1) / kGTile);
    const unsigned long long tag = lb_tag(epoch);
    if (ntiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *d_cnt_out = 0;
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t i0 = tile * kGTile + threadIdx.x * kGItems;

        unsigned long long k[kGItems];
        uint32_t pos[kGItems];
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            const uint32_t i = i0 + q;
            k[q] = i < n ? keys[i] : 0ull;
            pos[q] = kRound ? (i < n ? act_pos_in[i] : 0u) : i;
        }
        const unsigned long long kprev = (i0 > 0 && i0 - 1 < n) ? keys[i0 - 1] : 0ull;
        // is the element after this thread's last one a group head?
        bool next_head = true;
        if ((uint64_t)i0 + kGItems < n) {
            const unsigned long long kn = keys[i0 + kGItems];
            next_head = kn != k[kGItems - 1] || (!kRound && (uint32_t)(kn & 31) < kH0);
        }
        // head flags: a new key, or (initial sort) a key that contains its terminator
        uint32_t heads = 0;
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            const uint32_t i = i0 + q;
            const unsigned long long prev = q == 0 ? kprev : k[q - 1];
            const bool h = i < n && (i == 0 || k[q] != prev || (!kRound && (uint32_t)(k[q] & 31) < kH0));
            heads |= (uint32_t)h << q;
        }
        uint32_t tmax = 0, tsum = 0;
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            const uint32_t i = i0 + q;
            if (i >= n) continue;
            const bool h = (heads >> q) & 1u;
            const bool hn = q + 1 < kGItems ? (((heads >> (q + 1)) & 1u) || i + 1 >= n) : next_head;
            if (h) tmax = pos[q];
            tsum += (h && hn) ? 0u : 1u;
        }
        uint32_t totmax, totsum;
        const uint32_t exmax = cta_exclusive_scan<MaxOp, kThreads>(tmax, totmax);
        const uint32_t exsum = cta_exclusive_scan<SumOp, kThreads>(tsum, totsum);
        if (threadIdx.x == 0) {
            unsigned long long* w = lookback + 2ull * tile;
            uint32_t pmax = 0, psum = 0;
            if (tile == 0) {
                lb_store(w, tag | kLbPrefix | totmax);
                lb_store(w + 1, tag | kLbPrefix | totsum);
            } else {
                lb_store(w, tag | kLbAggregate | totmax);
                lb_store(w + 1, tag | kLbAggregate | totsum);
                pmax = lb_lookback<MaxOp>(lookback, 2, tile, tag, d_err, 128u);
                psum = lb_lookback<SumOp>(lookback + 1, 2, tile, tag, d_err, 128u);
                lb_store(w, tag | kLbPrefix | (pmax > totmax ? pmax : totmax));
                lb_store(w + 1, tag | kLbPrefix | (psum + totsum));
            }
            s_pmax = pmax;
            s_psum = psum;
            if (tile == ntiles - 1) *d_cnt_out = psum + totsum;
        }
        __syncthreads();
        uint32_t cur = s_pmax > exmax ? s_pmax : exmax;
        uint32_t out = s_psum + exsum;
#pragma unroll
        for (int q = 0; q < kGItems; ++q) {
            const uint32_t i = i0 + q;
            if (i >= n) continue;
            const bool h = (heads >> q) & 1u;
            const bool hn = q + 1 < kGItems ? (((heads >> (q + 1)) & 1u) || i + 1 >= n) : next_head;
            if (h) cur = pos[q];
            const uint32_t t = vals[i];
            if (t < n_block && pos[q] < n_block) {
                sa[pos[q]] = t;
                rank[t] = cur;
            } else {
                atomicOr(d_err, 32u);
            }
            if (!(h && hn)) {
                if (out < n_block) {
                    act_pos_out[out] = pos[q];
                    act_suf_out[out] = t;
                } else {
                    atomicOr(d_err, 32u);
                }
                ++out;
            }
        }
        __syncthreads();
    }
}

unsigned g_keys_ctas[64] = {0};
unsigned g_round_keys_ctas[64] = {0};
unsigned g_groups_ctas[64] = {0};
unsigned g_round_groups_ctas[64] = {0};

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

}  // namespace

void suffix_sort_init() {
    radix_init();
    const int dev = current_device();
    g_keys_ctas[dev] = persistent_ctas((const void*)sa_init_keys_kernel, kThreads, 0);
    g_round_keys_ctas[dev] = persistent_ctas((const void*)sa_round_keys_kernel, kThreads, 0);
    g_groups_ctas[dev] = persistent_ctas((const void*)sa_groups_kernel<false>, kThreads, 0);
    g_round_groups_ctas[dev] = persistent_ctas((const void*)sa_groups_kernel<true>, kThreads, 0);
}

uint32_t suffix_sort_rounds(uint32_t max_len) {
    uint32_t r = 0;
    uint64_t resolved = kH0;
    while (resolved <= max_len) {
        resolved *= 2;
        ++r;
    }
    return r;
}

size_t suffix_sort_log_slots(uint32_t max_len) { return suffix_sort_rounds(max_len) + 2; }

size_t suffix_sort_lookback_words(uint64_t cap) { return 2 * (size_t)(cap / kGTile + 2); }

void suffix_sort_block(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, uint32_t n,
                       uint32_t max_len, const SuffixSortBuffers& b) {
    if (n == 0) return;
    const int dev = current_device();
    const uint64_t gtiles = (uint64_t)n / kGTile + 1;
    auto grid_of = [](unsigned ctas, uint64_t need) {
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(std::max(1u, ctas), need));
    };
    const uint32_t rounds = suffix_sort_rounds(max_len);
    cudaMemsetAsync(b.counters, 0, (rounds + 2) * sizeof(uint32_t), L.stream);

    uint32_t* d_n = b.count_log;  // slot 0: n; slot r + 1: unsorted members after round r (r = 0: initial)
    const int passes0 = radix_passes(0, 63);
    radix_hist_clear(L, b.radix_temp);
    SBWT_LAUNCH(L, "sa_init_keys", (double)n * 12 + n / 4.0 + n / 8.0, 0, nullptr, sa_init_keys_kernel,
                grid_of(g_keys_ctas[dev], (uint64_t)n / kThreads + 1), kThreads, 0, text, term,
                (unsigned long long)base, n, b.keys, b.vals, d_n, radix_histograms(b.radix_temp), passes0);
    bool alt = radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, d_n, n, 0, 63, b.radix_temp, b.err, true);
    SBWT_LAUNCH(L, "sa_groups", (double)n * (8 + 4 + 4 + 4), 8, b.count_log + 1, sa_groups_kernel<false>,
                grid_of(g_groups_ctas[dev], gtiles), kThreads, 0, alt ? b.keys_alt : b.keys,
                alt ? b.vals_alt : b.vals, nullptr, d_n, n, b.sa, b.rank, b.act_pos[0], b.act_suf[0],
                b.count_log + 1, b.lookback, b.counters + kSlotInit, lb_next_epoch(), b.err);

    const int bits = n > 1 ? 32 - __builtin_clz(n - 1) : 1;
    const int passes = radix_passes(0, 2 * bits);
    uint32_t h = kH0;
    int cur = 0;
    for (uint32_t r = 1; r <= rounds; ++r, h *= 2) {
        const uint32_t* cnt = b.count_log + r;
        uint32_t* next_cnt = b.count_log + r + 1;
        radix_hist_clear(L, b.radix_temp);
        SBWT_LAUNCH(L, "sa_round_keys", 0, 24, cnt, sa_round_keys_kernel,
                    grid_of(g_round_keys_ctas[dev], (uint64_t)n / kThreads + 1), kThreads, 0, b.act_suf[cur], cnt,
                    b.rank, h, n, bits, b.keys, b.vals, radix_histograms(b.radix_temp), passes, b.err);
        const bool a =
            radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, cnt, n, 0, 2 * bits, b.radix_temp, b.err, true);
        SBWT_LAUNCH(L, "sa_round_groups", 0, 28, cnt, sa_groups_kernel<true>, grid_of(g_round_groups_ctas[dev], gtiles),
                    kThreads, 0, a ? b.keys_alt : b.keys, a ? b.vals_alt : b.vals, b.act_pos[cur], cnt, n, b.sa,
                    b.rank, b.act_pos[cur ^ 1], b.act_suf[cur ^ 1], next_cnt, b.lookback, b.counters + r,
                    lb_next_epoch(), b.err);
        cur ^= 1;
    }
}

}  // namespace sbwt
