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

namespace sbwt {
#include "radix_hdr.inc"
#include "scan.inc"
#include "radix_consts.inc"
#include "radix_count.inc"
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
