// sbwt_internal.cuh -- device data layouts and helpers shared by the kernels
// of the GB300 set-bwte library (arXiv 1410.0562).  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace sbwt {

// ---------------------------------------------------------------------------
// Text of an append (all its blocks): one 2-bit code per position, terminator
// positions hold code 0 and are flagged in a separate bitmap.  Position of
// read j's symbol k is offsets[j] + j + k; its terminator sits at
// offsets[j+1] + j (the block-local form of the same rule is the reading of
// Algorithm 2's text index: the exclusive prefix sum of |P_l|+1, plus k).
//   text[t >> 4] holds positions 16w .. 16w+15, MSB first: the code of t is
//   at bits 30 - 2*(t & 15), so concatenated words compare like strings.
//   term[t >> 5] bit (t & 31) is set iff t is a terminator.
// Both arrays start on a 16-byte boundary and carry zeroed padding words past
// the end (kTextPadWords, kTermPadWords) so fixed-width windows, read as
// aligned vectors, never leave them.
// ---------------------------------------------------------------------------
constexpr int kTextPadWords = 4;
constexpr int kTermPadWords = 2;

__device__ __forceinline__ uint32_t text_code(const uint32_t* __restrict__ text, uint64_t t) {
    return (text[t >> 4] >> (30u - 2u * (uint32_t)(t & 15))) & 3u;
}
// The same text with 4-bit codes (alphabets of 5 to 16 symbols):
// text[t >> 3] holds positions 8w .. 8w+7, MSB first, the code of t at bits
// 28 - 4*(t & 7).
template <int kB>
__device__ __forceinline__ uint32_t text_code_b(const uint32_t* __restrict__ text, uint64_t t) {
    constexpr uint32_t kPer = 32 / kB;
    return (text[t / kPer] >> (32u - kB - kB * (uint32_t)(t % kPer))) & ((1u << kB) - 1u);
}
// text words of an append of npos positions (without the padding)
inline uint64_t text_words(uint64_t npos, int code_bits) { return (npos + 31) / 32 * (uint64_t)code_bits; }
__device__ __forceinline__ uint32_t is_term(const uint32_t* __restrict__ term, uint64_t t) {
    return (term[t >> 5] >> (t & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Rank dictionary over B (Section 5's occurrence counters), the 2-bit codes
// held as bit planes.  Occurrence sampling S = 64 K rows (K = 1, 2 or 4:
// counters every 64, 128 or 256 rows).  Occurrence block b covers rows
// [S b, S (b+1)) in 3K + 1 64-bit words:
//   part q (rows S b + 64 q ... + 63, q < K): lo, hi, dm at words 3q, 3q+1,
//     3q+2 -- bit p of lo / hi is bit 0 / bit 1 of the code of the part's
//     row p (a terminator is stored as code 0), bit p of dm is set iff that
//     row holds a terminator;
//   word 3K: four 16-bit counts, count of code c (terminators excluded) in
//     [superblock start, block start), at bits 16c.
// With K = 1 a block is one 32-byte sector, so a rank query reads one
// sector; K = 2 and 4 hold 3.5 and 3.25 bits per row instead of 4 and a
// query reads two to four sectors.  Superblocks span 2^16 rows;
// super[4*s + c] counts code c in [0, 2^16 s).  A dictionary of n rows has
// n / S + 1 blocks and (n >> 16) + 1 superblocks, so rank(c, n) needs no
// special case; rows >= n are zero.
//   rank(c, i) = super[4*(i>>16)+c] + count_c(block of i) + the rows of
//   that block before i whose planes spell c and that hold no terminator.
// ---------------------------------------------------------------------------
constexpr int kOccShift = 6;  // rows of a part
constexpr int kOccSpan = 1 << kOccShift;
constexpr int kSuperShift = 16;
constexpr int kBlocksPerSuper = 1 << (kSuperShift - kOccShift);  // 1024 parts of 64 rows
constexpr uint8_t kBintDollar = 255;                              // B_int code of a terminator

template <int K>
struct Occ {
    static_assert(K == 1 || K == 2 || K == 4, "occurrence sampling of 64, 128 or 256 rows");
    static constexpr int kWords = 3 * K + 1;                                       // words per block
    static constexpr int kShift = kOccShift + (K == 1 ? 0 : (K == 2 ? 1 : 2));     // log2 rows per block
};

// 64-row parts of a dictionary of n rows with blocks of 64 k rows: every
// part of every block, the last block included.
__host__ __device__ __forceinline__ unsigned long long dict_parts(unsigned long long n, int k) {
    return (n / (64ull * (unsigned long long)k) + 1) * (unsigned long long)k;
}

__device__ __forceinline__ unsigned long long low_bits(uint32_t nbits) {
    return nbits >= 64 ? ~0ull : ((1ull << nbits) - 1ull);
}

// The rows of a part that hold code c (bit p for its row p); terminator rows
// never match.
__device__ __forceinline__ unsigned long long plane_match(unsigned long long lo, unsigned long long hi,
                                                          unsigned long long dm, uint32_t c) {
    return ((c & 1u) ? lo : ~lo) & ((c & 2u) ? hi : ~hi) & ~dm;
}

// rank(c, i) within i's superblock: the block counter plus the rows of the
// block before i that hold c.
template <int K>
__device__ __forceinline__ unsigned long long occ_rank_in_super(const unsigned long long* __restrict__ words,
                                                                uint32_t c, unsigned long long i) {
    const unsigned long long* p = words + (i >> Occ<K>::kShift) * Occ<K>::kWords;
    if constexpr (K == 1) {
        const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(p));
        const ulonglong2 d = __ldg(reinterpret_cast<const ulonglong2*>(p) + 1);
        const uint32_t r = (uint32_t)i & 63u;
        return ((uint32_t)(d.y >> (16 * c)) & 0xFFFFu) + __popcll(plane_match(a.x, a.y, d.x, c) & ((1ull << r) - 1ull));
    } else {
        const uint32_t r = (uint32_t)i & (64u * K - 1u), q = r >> 6;
        uint32_t in_block = 0;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if ((uint32_t)s <= q) {
                const unsigned long long m = plane_match(__ldg(p + 3 * s), __ldg(p + 3 * s + 1), __ldg(p + 3 * s + 2), c);
                in_block += __popcll((uint32_t)s < q ? m : (m & ((1ull << (r & 63u)) - 1ull)));
            }
        }
        return ((uint32_t)(__ldg(p + 3 * K) >> (16 * c)) & 0xFFFFu) + in_block;
    }
}

// ---------------------------------------------------------------------------
// The dictionary for 4-bit codes (alphabets of 5 to 16 symbols), one 64-byte
// block per 64 rows:
//   sym[4]  : row q at bits 4*(q & 15) of sym[q >> 4] (LSB first); a
//             terminator is stored as code 0
//   dmask   : bit q set iff row q holds a terminator
//   cnt[3]  : sixteen 12-bit counts, code c at bits 12c of the 192-bit field
//             cnt[0] | cnt[1] << 64 | cnt[2] << 128: code c (terminators
//             excluded) in [superblock start, block start)
// Superblocks span 2^12 rows (64 blocks, so the counts fit 12 bits);
// super[16*s + c] counts code c in [0, 2^12 s).  A dictionary of n rows has
// (n >> 6) + 1 blocks and ceil(blocks / 64) superblocks.
// ---------------------------------------------------------------------------
constexpr int kSuperShiftW = 12;
constexpr int kBlocksPerSuperW = 1 << (kSuperShiftW - kOccShift);  // 64
constexpr int kSigmaW = 16;

struct __align__(64) OccBlockW {
    unsigned long long sym[4];
    unsigned long long dmask;
    unsigned long long cnt[3];
};
static_assert(sizeof(OccBlockW) == 64, "two sectors per wide occurrence block");

// Mask with bit 4q set for every 4-bit field q of x equal to code c.
__device__ __forceinline__ unsigned long long match_code4(unsigned long long x, uint32_t c) {
    unsigned long long y = x ^ (0x1111111111111111ull * c);
    y |= y >> 1;
    y |= y >> 2;
    return ~y & 0x1111111111111111ull;
}

// 12-bit count of code c from the three counter words (selects, no
// indexing by c, so the words stay in registers).
__device__ __forceinline__ uint32_t cnt12(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                          uint32_t c) {
    const uint32_t o = 12u * c;
    const uint32_t w = o >> 6, sh = o & 63u;
    const unsigned long long lo = w == 0 ? c0 : (w == 1 ? c1 : c2);
    const unsigned long long hi = w == 0 ? c1 : c2;
    unsigned long long v = lo >> sh;
    if (sh > 52) v |= hi << (64 - sh);
    return (uint32_t)v & 0xFFFu;
}

// rank(c, i) within i's superblock for the wide dictionary.
__device__ __forceinline__ unsigned long long occ_rank_in_super_w(const OccBlockW* __restrict__ blocks, uint32_t c,
                                                                  unsigned long long i) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(blocks + (i >> kOccShift));
    const ulonglong2 s01 = __ldg(p), s23 = __ldg(p + 1), dc = __ldg(p + 2), c12 = __ldg(p + 3);
    const unsigned long long sym[4] = {s01.x, s01.y, s23.x, s23.y};
    const uint32_t r = (uint32_t)(i & (kOccSpan - 1));
    uint32_t in_block = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t rows = r > 16u * w ? min(r - 16u * w, 16u) : 0u;
        in_block += __popcll(match_code4(sym[w], c) & low_bits(4 * rows));
    }
    if (c == 0) in_block -= __popcll(dc.x & low_bits(r));
    return cnt12(dc.y, c12.x, c12.y, c) + in_block;
}

__device__ __forceinline__ unsigned long long occ_rank_w(const OccBlockW* __restrict__ blocks,
                                                         const unsigned long long* __restrict__ super, uint32_t c,
                                                         unsigned long long i) {
    return __ldg(super + ((i >> kSuperShiftW) << 4) + c) + occ_rank_in_super_w(blocks, c, i);
}

// The dictionary layouts behind one interface, by code width kB and (2-bit
// codes) occurrence sampling 64 K rows.
template <int kB, int K>
struct DictLayout;
template <int K>
struct DictLayout<2, K> {
    using Block = unsigned long long;  // the dictionary as an array of 64-bit words
    static constexpr int kSuperShift = sbwt::kSuperShift;
    static constexpr int kCodes = 4;
    __device__ __forceinline__ static unsigned long long in_super(const Block* __restrict__ b, uint32_t c,
                                                                  unsigned long long i) {
        return occ_rank_in_super<K>(b, c, i);
    }
};
template <>
struct DictLayout<4, 1> {
    using Block = OccBlockW;
    static constexpr int kSuperShift = kSuperShiftW;
    static constexpr int kCodes = kSigmaW;
    __device__ __forceinline__ static unsigned long long in_super(const Block* __restrict__ b, uint32_t c,
                                                                  unsigned long long i) {
        return occ_rank_in_super_w(b, c, i);
    }
};
template <int kB, int K>
__device__ __forceinline__ unsigned long long dict_rank(const typename DictLayout<kB, K>::Block* __restrict__ blocks,
                                                        const unsigned long long* __restrict__ super, uint32_t c,
                                                        unsigned long long i) {
    using D = DictLayout<kB, K>;
    return __ldg(super + (i >> D::kSuperShift) * D::kCodes + c) + D::in_super(blocks, c, i);
}

// ---------------------------------------------------------------------------
// CTA-wide scans (warp shuffles + one shared array of warp totals).
// ---------------------------------------------------------------------------
struct SumOp {
    template <class T>
    __device__ __forceinline__ static T id() { return T(0); }
    template <class T>
    __device__ __forceinline__ static T f(T a, T b) { return a + b; }
};
struct MaxOp {  // identity 0: every scanned value is unsigned
    template <class T>
    __device__ __forceinline__ static T id() { return T(0); }
    template <class T>
    __device__ __forceinline__ static T f(T a, T b) { return a > b ? a : b; }
};
struct MinOp {  // identity: all bits set (unsigned values)
    template <class T>
    __device__ __forceinline__ static T id() { return ~T(0); }
    template <class T>
    __device__ __forceinline__ static T f(T a, T b) { return a < b ? a : b; }
};

// Exclusive scan of one value per thread over a CTA of NT threads (NT a
// multiple of 32, at most 1024).  Every thread must call it.  Returns the
// exclusive prefix and sets `total` to the CTA-wide result.
template <class Op, int NT, class T>
__device__ __forceinline__ T cta_exclusive_scan(T v, T& total) {
    constexpr int kW = NT / 32;
    __shared__ T warp_tot[kW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = Op::f(y, x);
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kW ? warp_tot[lane] : Op::template id<T>();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = Op::f(y, w);
        }
        if (lane < kW) warp_tot[lane] = w;
    }
    __syncthreads();
    T excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = Op::template id<T>();
    T before = warp > 0 ? warp_tot[warp - 1] : Op::template id<T>();
    total = warp_tot[kW - 1];
    __syncthreads();
    return Op::f(before, excl);
}

// ---------------------------------------------------------------------------
// Launch bookkeeping: every kernel launch goes through a Launcher, which
// counts it and (with profiling on) brackets it with CUDA events.  The
// algorithmic bytes of a launch are `fixed` plus `per_unit` times a count
// that may live in device memory (the number of elements a launch with a
// device-side count actually processed); such counts must sit in the
// Launcher's unit log so one copy resolves them all after the stream drains.
// ---------------------------------------------------------------------------
struct KernelStat {
    std::string name;
    uint64_t launches = 0;
    double ms = 0;
    double bytes = 0;
};

class Launcher {
  public:
    struct Pending {
        int stat;
        cudaEvent_t a, b;
        double fixed, per_unit;
        const uint32_t* units;
        bool settled;
    };
    // What a captured CUDA graph launches: the stat of every kernel, and
    // (when captured with profiling on) the event pairs recorded by the graph.
    struct GraphLog {
        std::vector<int> launches;
        std::vector<Pending> timed;
    };

    cudaStream_t stream = nullptr;
    bool profiling = false;
    std::string only;  // with profiling: time only launches of this name (empty = all)
    std::vector<KernelStat> stats;
    const uint32_t* unit_log = nullptr;  // device array of element counts
    size_t unit_log_len = 0;
    GraphLog* capture = nullptr;  // non-null while a graph is being captured

    // After a replay of a captured graph (stream idle): counts its launches
    // and, if it was captured with profiling, folds in its event times.
    cudaError_t account_replay(const GraphLog& g);
    // Returns the events of a graph log that no graph uses any more.
    void recycle(GraphLog& g);

    int before(const char* name, double fixed, double per_unit = 0, const uint32_t* d_units = nullptr);
    void after(int token);
    // Reads the device-side element counts of the pending launches (one copy
    // of the unit log); call with the stream idle, before the log is reused.
    cudaError_t settle_units();
    // Folds pending event pairs into stats; call with the stream idle.
    cudaError_t resolve();
    // Host-side time of a named phase (stats entries named "host:...").
    void add_host(const char* name, double ms);
    void reset();
    void release();

  private:
    std::vector<Pending> pending_;
    std::vector<cudaEvent_t> free_events_;
    cudaEvent_t take_event();
    int stat_index(const char* name);
};

// SBWT_LAUNCH(L, "name", fixed_bytes, per_unit_bytes, d_units, kernel, grid, block, smem, args...)
#define SBWT_LAUNCH(L, NAME, FIXED, PER_UNIT, UNITS, KERNEL, GRID, BLOCK, SMEM, ...)            \
    do {                                                                                       \
        int _tok = (L).before(NAME, (double)(FIXED), (double)(PER_UNIT), (UNITS));             \
        KERNEL<<<(GRID), (BLOCK), (SMEM), (L).stream>>>(__VA_ARGS__);                          \
        (L).after(_tok);                                                                       \
    } while (0)

inline unsigned int ceil_div_u(uint64_t a, uint64_t b) { return (unsigned int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, global -> shared) completed on an
// mbarrier.  Addresses and sizes must be multiples of 16 bytes.  Every wait
// is bounded: mbar_wait returns false when it gave up.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}
constexpr uint32_t kMbarSpinLimit = 1u << 20;

// CTAs per launch for a persistent kernel: SMs x resident CTAs per SM.
unsigned persistent_ctas(const void* kernel, int threads, size_t smem);

// ---------------------------------------------------------------------------
// Radix sort (radix.cu).  Every count is read from device memory so a
// sequence of launches needs no host round trip; `cap` bounds the count.
// ---------------------------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;

constexpr uint32_t kRadixTile = 2048;  // keys per tile of a pass

inline int radix_passes(int begin_bit, int end_bit) { return (end_bit - begin_bit + kRadixBits - 1) / kRadixBits; }

// A pass over n keys with a grid of `grid` CTAs splits them into chunks of
// whole tiles, one per CTA: chunk c holds tiles [t0, t1) (empty for the
// chunks past the last tile).
__host__ __device__ inline void radix_chunk_tiles(uint32_t n, uint32_t grid, uint32_t c, uint32_t& t0, uint32_t& t1) {
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kRadixTile - 1) / kRadixTile);
    const uint32_t per = (ntiles + grid - 1) / grid;
    const uint64_t a = (uint64_t)c * per;
    t0 = a < ntiles ? (uint32_t)a : ntiles;
    t1 = t0 + per < ntiles ? t0 + per : ntiles;
}

size_t radix_temp_words(uint64_t cap);
void radix_init();  // once per device, before the first sort

// The first pass of a keys-only sort may be counted by the kernel that
// writes the keys, saving one read of them.  That kernel runs with
// radix_keys_grid(cap) CTAs; CTA c writes the digit counts of its chunk
// (radix_chunk_tiles with that grid) to radix_first_counts(temp)[c * 256 +
// d] and adds them to radix_first_totals(temp)[d], which radix_clear(temp)
// zeroed before it; a chunk without tiles writes nothing.  Then
// radix_sort_keys(..., first_counted = true).
unsigned radix_keys_grid(uint64_t cap);
uint32_t* radix_first_counts(uint32_t* temp);
uint32_t* radix_first_totals(uint32_t* temp);
void radix_clear(Launcher& L, uint32_t* temp);

// Stable LSD radix sort of (*d_n) 64-bit keys on bits [begin_bit, end_bit);
// key bits outside that range are carried along but do not take part in the
// order (a value can ride in them).  Sorts between keys and keys_alt; returns
// true when the result ended in keys_alt.  A scatter index out of range is
// skipped and flagged in *d_err (bit 4).  Both arrays must start on a 16-byte
// boundary (whole tiles arrive by TMA bulk copies).
bool radix_sort_keys(Launcher& L, unsigned long long* keys, unsigned long long* keys_alt, const uint32_t* d_n,
                     uint64_t cap, int begin_bit, int end_bit, uint32_t* temp, uint32_t* d_err,
                     bool first_counted = false);
// A sort of (64-bit key, 32-bit value) pairs, keyed like radix_sort_keys,
// in one cooperative launch (all passes, the CTAs meeting at bounded grid
// barriers; a barrier that times out flags *d_err bit 9); the values move in
// (vals, vals_alt) alongside.  Meant for lists that are often empty: an
// empty list costs one launch that returns at once.
bool radix_sort_pairs_fused(Launcher& L, unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                            uint32_t* vals_alt, const uint32_t* d_n, uint64_t cap, int begin_bit, int end_bit,
                            uint32_t* temp, uint32_t* d_err);

}  // namespace sbwt
