// Host emulation of the radix sort's count and scan phases (radix.cu), for
// CPU tests: the upsweep that counts each chunk's digits and the chunk scan
// that turns the counts into output offsets.
//
// The kernel text is compiled here unchanged apart from the one inline PTX
// load, done as two plain loads (the test cuts it out of the CUDA sources
// into the .inc files below), on the emulation in cuda_emu.h: one
// std::thread per GPU thread, warp intrinsics and CTA barriers emulated,
// every array between inaccessible pages.
#include "cuda_emu.h"

// Host stand-ins for the mbarrier and bulk-copy helpers of
// sbwt_internal.cuh, whose device versions are inline PTX: a bulk copy is
// done at once and completes its bytes on the barrier.  The barrier word
// holds the pending bytes (bits 0..31), the arrivals still expected
// (32..43), the arrival count (44..55) and the phase (bit 56); a phase
// completes when both pending counts reach zero.  A copy whose addresses or
// size are not multiples of 16 bytes (the bulk copy's rule) is recorded in
// g_tma_misaligned.
static std::atomic<int> g_tma_misaligned{0};
static void mbar_update(unsigned long long* bar, uint32_t arrive, uint32_t add_tx, uint32_t sub_tx) {
    std::atomic_ref<unsigned long long> r(*bar);
    unsigned long long cur = r.load(), nxt;
    do {
        uint32_t tx = (uint32_t)cur + add_tx - sub_tx;
        uint32_t arr = (uint32_t)((cur >> 32) & 0xFFFu) - arrive;
        const uint32_t count = (uint32_t)((cur >> 44) & 0xFFFu);
        unsigned long long phase = (cur >> 56) & 1ull;
        if (arr == 0 && tx == 0) {
            phase ^= 1ull;
            arr = count;
        }
        nxt = tx | ((unsigned long long)arr << 32) | ((unsigned long long)count << 44) | (phase << 56);
    } while (!r.compare_exchange_weak(cur, nxt));
}
static void mbar_init(unsigned long long* bar, uint32_t count) {
    std::atomic_ref<unsigned long long>(*bar).store(((unsigned long long)count << 32) |
                                                    ((unsigned long long)count << 44));
}
static void fence_proxy_async_smem() {}
static void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) { mbar_update(bar, 1, bytes, 0); }
static void tma_bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    if ((((uintptr_t)dst) | ((uintptr_t)src) | bytes) & 15u) g_tma_misaligned = 1;
    memcpy(dst, src, bytes);
    mbar_update(bar, 0, 0, bytes);
}
static bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    return ((std::atomic_ref<unsigned long long>(*bar).load() >> 56) & 1ull) != parity;
}
static bool mbar_wait(unsigned long long* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        std::this_thread::yield();
    }
    return false;
}
constexpr uint32_t kMbarSpinLimit = 1u << 20;
alignas(128) static unsigned char g_dyn_smem[80 * 1024];  // the downsweep's dynamic shared memory

namespace sbwt {
#include "radix_hdr.inc"
#include "scan.inc"
#include "radix_consts.inc"
#include "radix_count.inc"
#include "radix_down.inc"
#include "radix_fused_scan.inc"
}  // namespace sbwt
using namespace sbwt;

// One pass's counting: the upsweep over n keys (digit bits [shift, shift +
// 8)) with a grid of `grid` CTAs, then the chunk scan.  temp holds
// radix_temp-style words: totals at kTotals (both arrays, zeroed here),
// chunk counts (then offsets) at kChunkOffsets.  Returns the chunk offsets
// (grid x 256) in `offsets` and the next pass's totals (must come back
// zeroed) in `next_totals`.
extern "C" int emu_radix_count(const unsigned long long* keys, uint32_t n, int shift, uint32_t grid,
                               uint32_t* offsets, uint32_t* next_totals) {
    std::vector<std::pair<void*, size_t>> maps;
    const size_t words = kChunkOffsets + (size_t)grid * kBins + 64;
    std::vector<uint32_t> temp(words, 0u);
    for (int d = 0; d < kBins; ++d) temp[kTotals + kBins + d] = 7u;  // stale next totals the scan must clear
    const unsigned long long* g_keys = guarded(keys, n ? n : 1, maps);
    uint32_t* g_temp = guarded(temp.data(), words, maps);
    const uint32_t* g_n = guarded(&n, 1, maps);
    run_grid(grid, kThreads, [&] {
        radix_upsweep_kernel<unsigned long long>(g_keys, g_n, shift, g_temp + kChunkOffsets, g_temp + kTotals);
    });
    run_grid(kBins / kScanWarps, kScanThreads, [&] {
        radix_chunk_scan_kernel(g_temp + kChunkOffsets, (int)grid, g_temp + kTotals, g_temp + kTotals + kBins, g_n);
    });
    memcpy(offsets, g_temp + kChunkOffsets, (size_t)grid * kBins * 4);
    memcpy(next_totals, g_temp + kTotals + kBins, kBins * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// One whole pass: the upsweep, the chunk scan and the downsweep (keys alone,
// or with 32-bit values) with a grid of `grid` CTAs.  The input arrays are
// placed on 16-byte boundaries as device allocations are.  Returns 0, or 1
// when a bulk copy broke its alignment rule; *d_err as the kernels left it.
extern "C" int emu_radix_pass(const unsigned long long* keys, const uint32_t* vals, uint32_t n, int shift,
                              uint32_t grid, int pairs, unsigned long long* out_keys, uint32_t* out_vals,
                              uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    static_assert(down_smem<unsigned long long, true>() <= sizeof(g_dyn_smem), "the stand-in shared memory");
    const size_t words = kChunkOffsets + (size_t)grid * kBins + 64;
    std::vector<uint32_t> temp(words, 0u);
    const size_t nk = ((size_t)n + 1) & ~(size_t)1, nv = ((size_t)n + 3) & ~(size_t)3;  // whole 16-byte ends
    std::vector<unsigned long long> k(nk ? nk : 2, 0ull);
    std::vector<uint32_t> v(nv ? nv : 4, 0u);
    if (n) memcpy(k.data(), keys, n * 8ull);
    if (n && pairs) memcpy(v.data(), vals, n * 4ull);
    const unsigned long long* g_keys = guarded(k.data(), k.size(), maps);
    const uint32_t* g_vals = guarded(v.data(), v.size(), maps);
    unsigned long long* g_out = guarded(out_keys, n ? n : 1, maps);
    uint32_t* g_outv = guarded(out_vals, n ? n : 1, maps);
    uint32_t* g_temp = guarded(temp.data(), words, maps);
    const uint32_t* g_n = guarded(&n, 1, maps);
    g_tma_misaligned = 0;
    run_grid(grid, kThreads, [&] {
        radix_upsweep_kernel<unsigned long long>(g_keys, g_n, shift, g_temp + kChunkOffsets, g_temp + kTotals);
    });
    run_grid(kBins / kScanWarps, kScanThreads, [&] {
        radix_chunk_scan_kernel(g_temp + kChunkOffsets, (int)grid, g_temp + kTotals, g_temp + kTotals + kBins, g_n);
    });
    run_grid(grid, kThreads, [&] {
        if (pairs)
            radix_downsweep_kernel<unsigned long long, true>(g_keys, g_vals, g_out, g_outv, g_n, shift,
                                                             g_temp + kChunkOffsets, d_err);
        else
            radix_downsweep_kernel<unsigned long long, false>(g_keys, nullptr, g_out, nullptr, g_n, shift,
                                                              g_temp + kChunkOffsets, d_err);
    });
    memcpy(out_keys, g_out, n * 8ull);
    if (pairs) memcpy(out_vals, g_outv, n * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return g_tma_misaligned ? 1 : 0;
}

// The fused sort's passes (radix_sort_fused_kernel) with its phases run as
// consecutive grids in the kernel's order: a grid barrier of the kernel is
// the end of one grid here, since the emulation runs one CTA at a time.
// Each downsweep grid starts its tile barrier afresh (the kernel carries
// one across passes).  Keys with values; the result is in out_keys /
// out_vals.  Returns 0, or 1 when a bulk copy broke its alignment rule.
extern "C" int emu_fused_sort(const unsigned long long* keys, const uint32_t* vals, uint32_t n, int begin_bit,
                              int passes, uint32_t grid, unsigned long long* out_keys, uint32_t* out_vals,
                              uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const size_t words = kChunkOffsets + (size_t)grid * kBins + 64;
    std::vector<uint32_t> temp(words, 0u);
    const size_t nk = ((size_t)n + 1) & ~(size_t)1, nv = ((size_t)n + 3) & ~(size_t)3;
    std::vector<unsigned long long> k0(nk ? nk : 2, 0ull), k1(nk ? nk : 2, 0ull);
    std::vector<uint32_t> v0(nv ? nv : 4, 0u), v1(nv ? nv : 4, 0u);
    if (n) {
        memcpy(k0.data(), keys, n * 8ull);
        memcpy(v0.data(), vals, n * 4ull);
    }
    unsigned long long* g_k[2] = {guarded(k0.data(), k0.size(), maps), guarded(k1.data(), k1.size(), maps)};
    uint32_t* g_v[2] = {guarded(v0.data(), v0.size(), maps), guarded(v1.data(), v1.size(), maps)};
    uint32_t* g_temp = guarded(temp.data(), words, maps);
    g_tma_misaligned = 0;
    uint32_t ntiles = 0;
    const uint32_t tpc = tiles_per_chunk(n, grid, ntiles);
    const uint32_t nchunks = tpc ? (ntiles + tpc - 1) / tpc : 0;
    uint32_t* chunk = g_temp + kChunkOffsets;
    uint32_t* partials = g_temp + kPartials;
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(g_dyn_smem + down_smem<unsigned long long, true>() - 16);
    for (int p = 0; p < passes && n > 0; ++p) {
        const int a = p & 1;
        const int shift = begin_bit + kRadixBits * p;
        uint32_t* totals = g_temp + kTotals + (size_t)kBins * (p & 1);
        uint32_t* next_totals = g_temp + kTotals + (size_t)kBins * ((p + 1) & 1);
        run_grid(grid, kThreads, [&] {
            up_phase(g_k[a], n, shift, chunk, totals, reinterpret_cast<uint32_t*>(g_dyn_smem));
        });
        run_grid(grid, kThreads, [&] {
            scan_a_phase(chunk, nchunks, partials);
            if (blockIdx.x == 0) next_totals[threadIdx.x] = 0;
        });
        run_grid(grid, kThreads, [&] { scan_b_phase(chunk, nchunks, partials, totals); });
        run_grid(grid, kThreads, [&] {
            if (threadIdx.x == 0) mbar_init(bar, 1);
            uint32_t parity = 0;
            down_phase<unsigned long long, true>(g_k[a], g_v[a], g_k[a ^ 1], g_v[a ^ 1], n, shift, chunk, d_err,
                                                 g_dyn_smem, parity);
        });
    }
    const int fin = passes & 1;
    memcpy(out_keys, g_k[fin], n * 8ull);
    memcpy(out_vals, g_v[fin], n * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return g_tma_misaligned ? 1 : 0;
}
