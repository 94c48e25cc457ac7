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
// After each sort the bookkeeping (group heads, the running max of head rows
// = each element's group head, the unsorted flags and their running count =
// the compaction offsets) is reduce-then-scan over chunks of tiles; it writes
// SA, rank and the compacted list of unsorted members.
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
                                                                uint32_t* __restrict__ d_n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = n;
    for (uint32_t t = blockIdx.x * kThreads + threadIdx.x; t < n; t += gridDim.x * kThreads) {
        keys[t] = initial_key(text, term, base + t);
        vals[t] = t;
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

// Group bookkeeping after a sort.  Element i of the sorted list (keys, vals)
// sits on row pos(i) of the block SA: pos(i) = i after the initial sort,
// act_pos[i] after a round.  It writes SA[pos] = t, rank[t] = row of t's
// group head, and appends the members of groups with two or more elements to
// (act_pos_out, act_suf_out).  Like the radix passes it is reduce-then-scan
// over chunks of whole tiles: groups_reduce gives each chunk's last head row
// and member count, groups_scan turns them into per-chunk prefixes (and the
// total into *d_cnt_out), groups_apply walks each chunk with running values.
struct ElemInfo {
    unsigned long long k[kGItems];
    uint32_t pos[kGItems];
    uint32_t heads;  // bit q: element q starts a group
    uint32_t ends;   // bit q: element q is the last of its group
};

template <bool kRound>
__device__ __forceinline__ void load_tile_info(const unsigned long long* __restrict__ keys,
                                               const uint32_t* __restrict__ act_pos_in, uint32_t n, uint32_t i0,
                                               ElemInfo& e) {
#pragma unroll
    for (int q = 0; q < kGItems; ++q) {
        const uint32_t i = i0 + q;
        e.k[q] = i < n ? keys[i] : 0ull;
        e.pos[q] = kRound ? (i < n ? act_pos_in[i] : 0u) : i;
    }
    const unsigned long long kprev = (i0 > 0 && i0 - 1 < n) ? keys[i0 - 1] : 0ull;
    // is the element after this thread's last one a group head?
    bool next_head = true;
    if ((uint64_t)i0 + kGItems < n) {
        const unsigned long long kn = keys[i0 + kGItems];
        next_head = kn != e.k[kGItems - 1] || (!kRound && (uint32_t)(kn & 31) < kH0);
    }
    // head: a new key, or (initial sort) a key that contains its terminator
    e.heads = 0;
#pragma unroll
    for (int q = 0; q < kGItems; ++q) {
        const uint32_t i = i0 + q;
        const unsigned long long prev = q == 0 ? kprev : e.k[q - 1];
        const bool h = i < n && (i == 0 || e.k[q] != prev || (!kRound && (uint32_t)(e.k[q] & 31) < kH0));
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

template <bool kRound>
__global__ void __launch_bounds__(kThreads) sa_groups_reduce_kernel(const unsigned long long* __restrict__ keys,
                                                                    const uint32_t* __restrict__ act_pos_in,
                                                                    const uint32_t* __restrict__ d_cnt,
                                                                    uint32_t n_block, uint2* __restrict__ chunk_agg) {
    const uint32_t n = kRound ? *d_cnt : n_block;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kGTile - 1) / kGTile);
    uint32_t t0, t1;
    chunk_tiles(ntiles, t0, t1);
    uint32_t tmax = 0, tsum = 0;
    for (uint32_t tile = t0; tile < t1; ++tile) {
        ElemInfo e;
        const uint32_t i0 = tile * kGTile + threadIdx.x * kGItems;
        load_tile_info<kRound>(keys, act_pos_in, n, i0, e);
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

template <bool kRound>
__global__ void __launch_bounds__(kThreads) sa_groups_apply_kernel(
    const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ act_pos_in, const uint32_t* __restrict__ d_cnt, uint32_t n_block,
    const uint2* __restrict__ chunk_prefix, uint32_t* __restrict__ sa, uint32_t* __restrict__ rank,
    uint32_t* __restrict__ act_pos_out, uint32_t* __restrict__ act_suf_out, uint32_t* __restrict__ d_err) {
    const uint32_t n = kRound ? *d_cnt : n_block;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kGTile - 1) / kGTile);
    uint32_t t0, t1;
    chunk_tiles(ntiles, t0, t1);
    uint32_t run_max = chunk_prefix[blockIdx.x].x, run_sum = chunk_prefix[blockIdx.x].y;
    for (uint32_t tile = t0; tile < t1; ++tile) {
        ElemInfo e;
        const uint32_t i0 = tile * kGTile + threadIdx.x * kGItems;
        load_tile_info<kRound>(keys, act_pos_in, n, i0, e);
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

unsigned g_keys_ctas[64] = {0};
unsigned g_round_keys_ctas[64] = {0};
unsigned g_groups_ctas[64] = {0};

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
    g_groups_ctas[dev] = std::min<unsigned>(kMaxGroupChunks,
                                            persistent_ctas((const void*)sa_groups_apply_kernel<true>, kThreads, 0));
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

size_t suffix_sort_chunk_words(uint64_t cap) {
    (void)cap;
    return kMaxGroupChunks;  // one (max, count) pair per chunk, 8 bytes each
}

namespace {

template <bool kRound>
void run_groups(Launcher& L, const SuffixSortBuffers& b, const unsigned long long* keys, const uint32_t* vals,
                const uint32_t* act_pos_in, const uint32_t* d_cnt, uint32_t n_block, uint32_t* act_pos_out,
                uint32_t* act_suf_out, uint32_t* d_cnt_out, unsigned grid) {
    uint2* agg = reinterpret_cast<uint2*>(b.chunks);
    const char* names[3] = {kRound ? "sa_round_groups_reduce" : "sa_groups_reduce", "sa_groups_scan",
                            kRound ? "sa_round_groups_apply" : "sa_groups_apply"};
    const double fixed = kRound ? 0.0 : (double)n_block;
    const double per = kRound ? 1.0 : 0.0;
    SBWT_LAUNCH(L, names[0], fixed * (kRound ? 0 : 8), per * 12, kRound ? d_cnt : nullptr,
                sa_groups_reduce_kernel<kRound>, grid, kThreads, 0, keys, act_pos_in, d_cnt, n_block, agg);
    SBWT_LAUNCH(L, names[1], 16.0 * grid, 0, nullptr, sa_groups_scan_kernel, 1, kThreads, 0, agg, (int)grid,
                d_cnt_out);
    // per element: key (+ neighbours), value, position, SA and rank writes,
    // and the compacted pair of an unsorted member
    SBWT_LAUNCH(L, names[2], fixed * 28, per * 36, kRound ? d_cnt : nullptr, sa_groups_apply_kernel<kRound>, grid,
                kThreads, 0, keys, vals, act_pos_in, d_cnt, n_block, agg, b.sa, b.rank, act_pos_out, act_suf_out,
                b.err);
}

}  // namespace

void suffix_sort_block(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, uint32_t n,
                       uint32_t max_len, const SuffixSortBuffers& b) {
    if (n == 0) return;
    const int dev = current_device();
    const uint64_t gtiles = (uint64_t)n / kGTile + 1;
    auto grid_of = [](unsigned ctas, uint64_t need) {
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(std::max(1u, ctas), need));
    };
    const uint32_t rounds = suffix_sort_rounds(max_len);

    uint32_t* d_n = b.count_log;  // slot 0: n; slot r + 1: unsorted members after round r (r = 0: initial)
    SBWT_LAUNCH(L, "sa_init_keys", (double)n * 12 + n / 4.0 + n / 8.0, 0, nullptr, sa_init_keys_kernel,
                grid_of(g_keys_ctas[dev], (uint64_t)n / kThreads + 1), kThreads, 0, text, term,
                (unsigned long long)base, n, b.keys, b.vals, d_n);
    bool alt = radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, d_n, n, 0, 63, b.radix_temp, b.err);
    run_groups<false>(L, b, alt ? b.keys_alt : b.keys, alt ? b.vals_alt : b.vals, nullptr, d_n, n, b.act_pos[0],
                      b.act_suf[0], b.count_log + 1, grid_of(g_groups_ctas[dev], gtiles));

    const int bits = n > 1 ? 32 - __builtin_clz(n - 1) : 1;
    uint32_t h = kH0;
    int cur = 0;
    for (uint32_t r = 1; r <= rounds; ++r, h *= 2) {
        const uint32_t* cnt = b.count_log + r;
        uint32_t* next_cnt = b.count_log + r + 1;
        SBWT_LAUNCH(L, "sa_round_keys", 0, 24, cnt, sa_round_keys_kernel,
                    grid_of(g_round_keys_ctas[dev], (uint64_t)n / kThreads + 1), kThreads, 0, b.act_suf[cur], cnt,
                    b.rank, h, n, bits, b.keys, b.vals, b.err);
        const bool a =
            radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, cnt, n, 0, 2 * bits, b.radix_temp, b.err);
        run_groups<true>(L, b, a ? b.keys_alt : b.keys, a ? b.vals_alt : b.vals, b.act_pos[cur], cnt, n,
                         b.act_pos[cur ^ 1], b.act_suf[cur ^ 1], next_cnt, grid_of(g_groups_ctas[dev], gtiles));
        cur ^= 1;
    }
}

}  // namespace sbwt
