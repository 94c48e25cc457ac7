// Host emulation of the 4-bit Insert kernel of insert.cu (alphabets of 5 to
// 16 symbols), for CPU tests.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h: one
// std::thread per GPU thread, warp intrinsics and CTA barriers emulated,
// every array between inaccessible pages.
#include "cuda_emu.h"

#include "dict.inc"
#include "dictw.inc"
#include "threads.inc"
#include "insert_w.inc"

namespace {
template <class IdxT>
int run_insert_w(const OccBlockW* old_blocks, unsigned long long n_ext, const uint8_t* bint, const IdxT* gsa,
                 unsigned long long n_int, OccBlockW* new_blocks, unsigned long long n_new, uint32_t* sb_tot,
                 uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nb_old = (n_ext >> kOccShift) + 1, nb_new = (n_new >> kOccShift) + 1;
    const uint64_t nsb = (nb_new + kBlocksPerSuperW - 1) / kBlocksPerSuperW;
    const uint64_t nb_all = nsb * kBlocksPerSuperW;  // output blocks the grid covers
    const OccBlockW* g_old = guarded(old_blocks, nb_old, maps);
    const uint8_t* g_bint = guarded(bint, n_int ? n_int : 1, maps);
    const IdxT* g_gsa = guarded(gsa, n_int ? n_int : 1, maps);
    OccBlockW* g_new = guarded(new_blocks, nb_new, maps);
    uint32_t* g_tot = guarded(sb_tot, (size_t)kSigmaW * nsb, maps);
    run_grid((unsigned)((nb_all + kThreads - 1) / kThreads), kThreads, [&] {
        insert_w_kernel<IdxT>(g_old, n_ext, g_bint, g_gsa, n_int, g_new, n_new, nsb, g_tot, d_err, 0ull, 0, 0ull);
    });
    memcpy(new_blocks, g_new, nb_new * sizeof(OccBlockW));
    memcpy(sb_tot, g_tot, (size_t)kSigmaW * nsb * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
}  // namespace

// One 4-bit Insert over the old dictionary (n_ext rows, (n_ext >> 6) + 1
// blocks), the new symbols (bint codes, 255 for a terminator; g_sa of 4- or
// 8-byte entries) into (n_new >> 6) + 1 new blocks and the per-superblock
// code totals (16 per superblock of 4096 rows).
extern "C" int emu_insert_w(const OccBlockW* old_blocks, unsigned long long n_ext, const uint8_t* bint,
                            const void* gsa, int gsa_bytes, unsigned long long n_int, OccBlockW* new_blocks,
                            unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err) {
    if (gsa_bytes == 4)
        return run_insert_w(old_blocks, n_ext, bint, static_cast<const uint32_t*>(gsa), n_int, new_blocks, n_new,
                            sb_tot, d_err);
    return run_insert_w(old_blocks, n_ext, bint, static_cast<const unsigned long long*>(gsa), n_int, new_blocks,
                        n_new, sb_tot, d_err);
}
