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
#include "sbwt_internal.cuh"
#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kH0 = 29;

__global__ void __launch_bounds__(kThreads) sa_init_keys_kernel(const uint32_t* __restrict__ text,
                                                                const uint32_t* __restrict__ term,
                                                                unsigned long long base, uint32_t n,
                                                                unsigned long long* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ d_n) {
    const uint32_t t = blockIdx.x * kThreads + threadIdx.x;
    if (t == 0) *d_n = n;
    if (t >= n) return;
    const uint64_t P = base + t;
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
    keys[t] = (k58 << 5) | len;
    vals[t] = t;
}

// After the initial sort: SA, group-head candidates for the max-scan.
__global__ void __launch_bounds__(kThreads) sa_heads_kernel(const unsigned long long* __restrict__ keys,
                                                            const uint32_t* __restrict__ vals, uint32_t n,
                                                            uint32_t* __restrict__ sa,
                                                            uint32_t* __restrict__ headval) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    const bool head = i == 0 || k != keys[i - 1] || (uint32_t)(k & 31) < kH0;
    sa[i] = vals[i];
    headval[i] = head ? i : 0u;
}

// rank[SA[i]] = group head; active[i] = 1 iff i's group has >= 2 members.
__global__ void __launch_bounds__(kThreads) sa_rank_kernel(const uint32_t* __restrict__ sa,
                                                           const uint32_t* __restrict__ headidx, uint32_t n,
                                                           uint32_t* __restrict__ rank,
                                                           uint32_t* __restrict__ active,
                                                           uint32_t* __restrict__ d_err) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t h = headidx[i];
    const uint32_t t = sa[i];
    if (t < n) rank[t] = h; else atomicOr(d_err, 32u);
    const bool head = h == i;
    const bool next_head = i + 1 == n || headidx[i + 1] == i + 1;
    active[i] = (head && next_head) ? 0u : 1u;
}

__global__ void __launch_bounds__(kThreads) sa_compact_kernel(const uint32_t* __restrict__ active,
                                                              const uint32_t* __restrict__ idx,
                                                              const uint32_t* __restrict__ sa, uint32_t n,
                                                              uint32_t* __restrict__ act_pos,
                                                              uint32_t* __restrict__ act_suf,
                                                              uint32_t* __restrict__ d_err) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n || !active[i]) return;
    const uint32_t k = idx[i];
    if (k >= n) {
        atomicOr(d_err, 32u);
        return;
    }
    act_pos[k] = i;
    act_suf[k] = sa[i];
}

__global__ void __launch_bounds__(kThreads) sa_round_keys_kernel(const uint32_t* __restrict__ act_suf,
                                                                 const uint32_t* __restrict__ d_cnt,
                                                                 const uint32_t* __restrict__ rank, uint32_t h,
                                                                 uint32_t n, int bits,
                                                                 unsigned long long* __restrict__ keys,
                                                                 uint32_t* __restrict__ vals,
                                                                 uint32_t* __restrict__ d_err) {
    const uint32_t k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= *d_cnt) return;
    const uint32_t t = act_suf[k];
    // an unsorted member has at least h symbols before its terminator, so
    // t + h stays inside the block; anything else is a fault of the caller
    uint32_t next = 0;
    if ((uint64_t)t + h < n) next = rank[t + h]; else atomicOr(d_err, 4u);
    keys[k] = ((unsigned long long)rank[t] << bits) | next;
    vals[k] = t;
}

__global__ void __launch_bounds__(kThreads) sa_round_heads_kernel(const unsigned long long* __restrict__ keys,
                                                                  const uint32_t* __restrict__ vals,
                                                                  const uint32_t* __restrict__ act_pos,
                                                                  const uint32_t* __restrict__ d_cnt, uint32_t n,
                                                                  uint32_t* __restrict__ sa,
                                                                  uint32_t* __restrict__ headval,
                                                                  uint32_t* __restrict__ d_err) {
    const uint32_t k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= *d_cnt) return;
    const uint32_t p = act_pos[k];
    if (p < n) sa[p] = vals[k]; else atomicOr(d_err, 32u);
    const bool head = k == 0 || keys[k] != keys[k - 1];
    headval[k] = head ? p : 0u;
}

__global__ void __launch_bounds__(kThreads) sa_round_rank_kernel(const uint32_t* __restrict__ vals,
                                                                 const uint32_t* __restrict__ act_pos,
                                                                 const uint32_t* __restrict__ headidx,
                                                                 const uint32_t* __restrict__ d_cnt, uint32_t n,
                                                                 uint32_t* __restrict__ rank,
                                                                 uint32_t* __restrict__ active,
                                                                 uint32_t* __restrict__ d_err) {
    const uint32_t cnt = *d_cnt;
    const uint32_t k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= cnt) return;
    const uint32_t h = headidx[k];
    const uint32_t t = vals[k];
    if (t < n) rank[t] = h; else atomicOr(d_err, 32u);
    const bool head = h == act_pos[k];
    const bool next_head = k + 1 == cnt || headidx[k + 1] == act_pos[k + 1];
    active[k] = (head && next_head) ? 0u : 1u;
}

__global__ void __launch_bounds__(kThreads) sa_round_compact_kernel(const uint32_t* __restrict__ active,
                                                                    const uint32_t* __restrict__ idx,
                                                                    const uint32_t* __restrict__ act_pos,
                                                                    const uint32_t* __restrict__ vals,
                                                                    const uint32_t* __restrict__ d_cnt, uint32_t n,
                                                                    uint32_t* __restrict__ act_pos2,
                                                                    uint32_t* __restrict__ act_suf2,
                                                                    uint32_t* __restrict__ d_err) {
    const uint32_t k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= *d_cnt || !active[k]) return;
    const uint32_t j = idx[k];
    if (j >= n) {
        atomicOr(d_err, 32u);
        return;
    }
    act_pos2[j] = act_pos[k];
    act_suf2[j] = vals[k];
}

}  // namespace

uint32_t suffix_sort_rounds(uint32_t max_len) {
    uint32_t r = 0;
    uint64_t resolved = kH0;
    while (resolved <= max_len) {
        resolved *= 2;
        ++r;
    }
    return r;
}

void suffix_sort_block(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, uint32_t n,
                       uint32_t max_len, const SuffixSortBuffers& b) {
    if (n == 0) return;
    const unsigned grid = ceil_div_u(n, kThreads);
    uint32_t* d_n = b.count_log;  // slot 0: n; slot r: active count after round r-1 (slot 1 = after init)
    SBWT_LAUNCH(L, "sa_init_keys", (double)n * 12 + n / 4.0 + n / 8.0, 0, nullptr, sa_init_keys_kernel, grid,
                kThreads, 0, text, term, (unsigned long long)base, n, b.keys, b.vals, d_n);
    bool alt = radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, d_n, n, 0, 63, b.radix_temp, b.err);
    const unsigned long long* sk = alt ? b.keys_alt : b.keys;
    const uint32_t* sv = alt ? b.vals_alt : b.vals;
    SBWT_LAUNCH(L, "sa_heads", (double)n * 20, 0, nullptr, sa_heads_kernel, grid, kThreads, 0, sk, sv, n, b.sa,
                b.tmp_a);
    scan_inclusive_max(L, b.tmp_a, b.tmp_a, d_n, n, b.scan_temp);
    SBWT_LAUNCH(L, "sa_rank", (double)n * 16, 0, nullptr, sa_rank_kernel, grid, kThreads, 0, b.sa, b.tmp_a, n,
                b.rank, b.tmp_b, b.err);
    uint32_t* d_cnt = b.count_log + 1;
    scan_exclusive_sum(L, b.tmp_b, b.tmp_a, d_n, n, b.scan_temp, d_cnt);
    SBWT_LAUNCH(L, "sa_compact", (double)n * 12, 0, nullptr, sa_compact_kernel, grid, kThreads, 0, b.tmp_b,
                b.tmp_a, b.sa, n, b.act_pos[0], b.act_suf[0], b.err);

    const uint32_t rounds = suffix_sort_rounds(max_len);
    const int bits = n > 1 ? 32 - __builtin_clz(n - 1) : 1;
    uint32_t h = kH0;
    int cur = 0;
    for (uint32_t r = 1; r <= rounds; ++r, h *= 2) {
        const uint32_t* cnt = b.count_log + r;
        uint32_t* next_cnt = b.count_log + r + 1;
        SBWT_LAUNCH(L, "sa_round_keys", 0, 24, cnt, sa_round_keys_kernel, grid, kThreads, 0, b.act_suf[cur], cnt,
                    b.rank, h, n, bits, b.keys, b.vals, b.err);
        bool a = radix_sort_pairs(L, b.keys, b.vals, b.keys_alt, b.vals_alt, cnt, n, 0, 2 * bits, b.radix_temp,
                                  b.err);
        const unsigned long long* rk = a ? b.keys_alt : b.keys;
        const uint32_t* rv = a ? b.vals_alt : b.vals;
        SBWT_LAUNCH(L, "sa_round_heads", 0, 24, cnt, sa_round_heads_kernel, grid, kThreads, 0, rk, rv,
                    b.act_pos[cur], cnt, n, b.sa, b.tmp_a, b.err);
        scan_inclusive_max(L, b.tmp_a, b.tmp_a, cnt, n, b.scan_temp);
        SBWT_LAUNCH(L, "sa_round_rank", 0, 20, cnt, sa_round_rank_kernel, grid, kThreads, 0, rv, b.act_pos[cur],
                    b.tmp_a, cnt, n, b.rank, b.tmp_b, b.err);
        scan_exclusive_sum(L, b.tmp_b, b.tmp_a, cnt, n, b.scan_temp, next_cnt);
        SBWT_LAUNCH(L, "sa_round_compact", 0, 20, cnt, sa_round_compact_kernel, grid, kThreads, 0, b.tmp_b,
                    b.tmp_a, b.act_pos[cur], rv, cnt, n, b.act_pos[cur ^ 1], b.act_suf[cur ^ 1], b.err);
        cur ^= 1;
    }
}

size_t suffix_sort_log_slots(uint32_t max_len) { return suffix_sort_rounds(max_len) + 2; }

}  // namespace sbwt
