// Host emulation of the 2-bit Insert kernel of insert.cu, for CPU tests.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h: one
// std::thread per GPU thread, warp intrinsics and CTA barriers emulated,
// every array between inaccessible pages.
#include "cuda_emu.h"

#include "dict.inc"
#include "scan.inc"
#include "insert.inc"

// One Insert launch: nsb CTAs of kInsertThreads threads over the old dictionary (n_ext
// rows), the new symbols (bint, gsa; n_int of them) and the plan ins_i0
// (nsb + 1 entries); writes the new dictionary's blocks and the superblock
// totals.  gsa_bytes is 4 or 8 (the index width).
extern "C" int emu_insert(const void* old_blocks, unsigned long long n_ext, const uint8_t* bint, const void* gsa,
                          int gsa_bytes, unsigned long long n_int, const uint32_t* ins_i0, void* new_blocks,
                          unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nb_old = (n_ext >> kOccShift) + 1, nb_new = (n_new >> kOccShift) + 1;
    const uint64_t nsb = (nb_new + kBlocksPerSuper - 1) / kBlocksPerSuper;
    const OccBlock* g_old = guarded(static_cast<const OccBlock*>(old_blocks), nb_old, maps);
    const uint8_t* g_bint = guarded(bint, n_int, maps);
    const uint32_t* g_plan = guarded(ins_i0, nsb + 1, maps);
    OccBlock* g_new = guarded(static_cast<OccBlock*>(new_blocks), nb_new, maps);
    uint32_t* g_tot = guarded(sb_tot, 4 * nsb, maps);
    if (gsa_bytes == 4) {
        const uint32_t* g_gsa = guarded(static_cast<const uint32_t*>(gsa), n_int, maps);
        run_grid((unsigned)nsb, kInsertThreads, [&] {
            insert_kernel<uint32_t, kInsertThreads>(g_old, n_ext, g_bint, g_gsa, n_int, g_plan, g_new, n_new, g_tot, d_err);
        });
    } else {
        const unsigned long long* g_gsa = guarded(static_cast<const unsigned long long*>(gsa), n_int, maps);
        run_grid((unsigned)nsb, kInsertThreads, [&] {
            insert_kernel<unsigned long long, kInsertThreads>(g_old, n_ext, g_bint, g_gsa, n_int, g_plan, g_new, n_new, g_tot,
                                                   d_err);
        });
    }
    memcpy(new_blocks, g_new, nb_new * sizeof(OccBlock));
    memcpy(sb_tot, g_tot, 4 * nsb * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
