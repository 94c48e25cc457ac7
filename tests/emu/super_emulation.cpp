// Host emulation of Insert's superblock-counter scan (insert.cu), for CPU
// tests: the 64-bit counters before each superblock and C[] from the
// per-superblock code totals, by the one-CTA form or the three-kernel form.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h:
// one std::thread per GPU thread, CTA barriers emulated, every array
// between inaccessible pages.
#include "cuda_emu.h"

#include "scan.inc"
#include "super.inc"

namespace {
template <int kCodes>
int run_scan(const uint32_t* sb_tot, uint64_t nsb, uint64_t m, int force_chunks, unsigned long long* super,
             unsigned long long* C) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_tot = guarded(sb_tot, (size_t)kCodes * (nsb ? nsb : 1), maps);
    unsigned long long* g_super = guarded(super, (size_t)kCodes * (nsb ? nsb : 1), maps);
    unsigned long long* g_C = guarded(C, (size_t)kCodes, maps);
    if (!force_chunks && nsb <= kSmallScan) {
        run_grid(1, kScanThreads, [&] { super_scan_small_kernel<kCodes>(g_tot, nsb, g_super, g_C, m); });
    } else {
        const unsigned nchunks = (unsigned)((nsb + kScanThreads - 1) / kScanThreads);
        std::vector<unsigned long long> chunk(kCodes * (size_t)(nchunks ? nchunks : 1), 0ull);
        unsigned long long* g_chunk = guarded(chunk.data(), chunk.size(), maps);
        run_grid(nchunks, kScanThreads, [&] { super_local_kernel<kCodes>(g_tot, nsb, g_super, g_chunk); });
        run_grid(1, kScanThreads, [&] { super_chunks_kernel<kCodes>(g_chunk, nchunks, g_C, m); });
        run_grid(nchunks, kScanThreads, [&] { super_add_kernel<kCodes>(g_super, nsb, g_chunk); });
    }
    memcpy(super, g_super, (size_t)kCodes * nsb * 8);
    memcpy(C, g_C, (size_t)kCodes * 8);
    for (auto& mp : maps) munmap(mp.first, mp.second);
    return 0;
}
}  // namespace

// codes: 4 (2-bit dictionary) or 16 (4-bit); force_chunks: take the
// three-kernel form even for few superblocks.
extern "C" int emu_super_scan(int codes, const uint32_t* sb_tot, uint64_t nsb, uint64_t m, int force_chunks,
                              unsigned long long* super, unsigned long long* C) {
    if (codes == 4) return run_scan<4>(sb_tot, nsb, m, force_chunks, super, C);
    if (codes == 16) return run_scan<16>(sb_tot, nsb, m, force_chunks, super, C);
    return 1;
}
