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

// One Insert launch: nsb CTAs of kInsertThreads threads over the old
// dictionary (n_ext rows, blocks of 64 k rows as 64-bit words), the new
// symbols (bint, gsa; n_int of them) and the plan ins_i0 (nsb + 1 entries);
// writes the new dictionary's words and the superblock totals.  gsa_bytes is
// 4 or 8 (the index width).
template <int K, int kT, class IdxT>
static void run_insert(const unsigned long long* old_words, unsigned long long n_ext, const uint8_t* bint,
                       const IdxT* gsa, unsigned long long n_int, const uint32_t* ins_i0, unsigned long long* new_words,
                       unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t w_old = (n_ext / (64ull * K) + 1) * Occ<K>::kWords, w_new = (n_new / (64ull * K) + 1) * Occ<K>::kWords;
    const uint64_t nsb = (n_new >> kSuperShift) + 1;
    const unsigned long long* g_old = guarded(old_words, w_old, maps);
    const uint8_t* g_bint = guarded(bint, n_int, maps);
    const uint32_t* g_plan = guarded(ins_i0, nsb + 1, maps);
    unsigned long long* g_new = guarded(new_words, w_new, maps);
    uint32_t* g_tot = guarded(sb_tot, 4 * nsb, maps);
    const IdxT* g_gsa = guarded(gsa, n_int, maps);
    run_grid((unsigned)nsb, kT, [&] {
        insert_kernel<IdxT, kT, K>(g_old, n_ext, g_bint, g_gsa, n_int, g_plan, g_new, n_new, g_tot, d_err, 0ull, 0,
                                   0ull);
    });
    memcpy(new_words, g_new, w_new * 8);
    memcpy(sb_tot, g_tot, 4 * nsb * 4);
    for (auto& m : maps) munmap(m.first, m.second);
}

template <int K, int kT>
static void run_width(const void* old_words, unsigned long long n_ext, const uint8_t* bint, const void* gsa,
                      int gsa_bytes, unsigned long long n_int, const uint32_t* ins_i0, void* new_words,
                      unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err) {
    const auto* o = static_cast<const unsigned long long*>(old_words);
    auto* w = static_cast<unsigned long long*>(new_words);
    if (gsa_bytes == 4)
        run_insert<K, kT>(o, n_ext, bint, static_cast<const uint32_t*>(gsa), n_int, ins_i0, w, n_new, sb_tot, d_err);
    else
        run_insert<K, kT>(o, n_ext, bint, static_cast<const unsigned long long*>(gsa), n_int, ins_i0, w, n_new,
                          sb_tot, d_err);
}

// the CTA size the launcher picks: 512 threads for dense new rows, 256 else
template <int K>
static void run_density(const void* old_words, unsigned long long n_ext, const uint8_t* bint, const void* gsa,
                        int gsa_bytes, unsigned long long n_int, const uint32_t* ins_i0, void* new_words,
                        unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err) {
    if (4 * n_int >= n_new)
        run_width<K, kInsertThreads>(old_words, n_ext, bint, gsa, gsa_bytes, n_int, ins_i0, new_words, n_new, sb_tot,
                                     d_err);
    else
        run_width<K, kInsertThreadsSparse>(old_words, n_ext, bint, gsa, gsa_bytes, n_int, ins_i0, new_words, n_new,
                                           sb_tot, d_err);
}

extern "C" int emu_insert(const void* old_words, unsigned long long n_ext, const uint8_t* bint, const void* gsa,
                          int gsa_bytes, unsigned long long n_int, const uint32_t* ins_i0, void* new_words,
                          unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err, int occ_k) {
    if (occ_k == 4)
        run_density<4>(old_words, n_ext, bint, gsa, gsa_bytes, n_int, ins_i0, new_words, n_new, sb_tot, d_err);
    else if (occ_k == 2)
        run_density<2>(old_words, n_ext, bint, gsa, gsa_bytes, n_int, ins_i0, new_words, n_new, sb_tot, d_err);
    else
        run_density<1>(old_words, n_ext, bint, gsa, gsa_bytes, n_int, ins_i0, new_words, n_new, sb_tot, d_err);
    return 0;
}

// The in-place Insert of the host tier: the dictionary in `words` (sized for
// n_new rows, holding the n_ext old rows) is rewritten from the top
// superblock down in chunks of `chunk` superblocks, each chunk's old blocks
// first copied to a staging buffer, as launch_insert does with
// kStageSupers-superblock chunks.
template <int K, int kT, class IdxT>
static void run_in_place(unsigned long long* words, unsigned long long n_ext, const uint8_t* bint, const IdxT* gsa,
                         unsigned long long n_int, const uint32_t* ins_i0, unsigned long long n_new, uint32_t* sb_tot,
                         uint32_t* d_err, uint64_t chunk) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t w_new = (n_new / (64ull * K) + 1) * Occ<K>::kWords;
    const uint64_t nsb = (n_new >> kSuperShift) + 1;
    const uint64_t stage_blocks = chunk * kBlocksPerSuper / K + 8;
    std::vector<unsigned long long> zero(stage_blocks * Occ<K>::kWords, 0ull);
    unsigned long long* g_words = guarded(words, w_new, maps);
    unsigned long long* g_stage = guarded(zero.data(), zero.size(), maps);
    const uint8_t* g_bint = guarded(bint, n_int, maps);
    const uint32_t* g_plan = guarded(ins_i0, nsb + 1, maps);
    uint32_t* g_tot = guarded(sb_tot, 4 * nsb, maps);
    const IdxT* g_gsa = guarded(gsa, n_int, maps);
    for (uint64_t s1 = nsb; s1 > 0;) {
        const uint64_t s0 = s1 > chunk ? s1 - chunk : 0;
        run_grid(4, kThreads, [&] {
            stage_old_kernel<K>(g_words, n_ext, g_plan, s0, s1, g_stage, stage_blocks, d_err);
        });
        run_grid((unsigned)(s1 - s0), kT, [&] {
            insert_kernel<IdxT, kT, K>(g_stage, n_ext, g_bint, g_gsa, n_int, g_plan, g_words, n_new, g_tot, d_err, s0,
                                       1, stage_blocks);
        });
        s1 = s0;
    }
    memcpy(words, g_words, w_new * 8);
    memcpy(sb_tot, g_tot, 4 * nsb * 4);
    for (auto& m : maps) munmap(m.first, m.second);
}

extern "C" int emu_insert_in_place(void* words, unsigned long long n_ext, const uint8_t* bint, const void* gsa,
                                   int gsa_bytes, unsigned long long n_int, const uint32_t* ins_i0,
                                   unsigned long long n_new, uint32_t* sb_tot, uint32_t* d_err, int occ_k,
                                   unsigned long long chunk) {
    auto* w = static_cast<unsigned long long*>(words);
    const bool dense = 4 * n_int >= n_new;
#define SBWT_EMU_IN_PLACE(K, T)                                                                                      \
    (gsa_bytes == 4 ? run_in_place<K, T>(w, n_ext, bint, static_cast<const uint32_t*>(gsa), n_int, ins_i0, n_new,    \
                                         sb_tot, d_err, chunk)                                                      \
                    : run_in_place<K, T>(w, n_ext, bint, static_cast<const unsigned long long*>(gsa), n_int, ins_i0, \
                                         n_new, sb_tot, d_err, chunk))
    if (occ_k == 4) {
        if (dense) SBWT_EMU_IN_PLACE(4, kInsertThreads); else SBWT_EMU_IN_PLACE(4, kInsertThreadsSparse);
    } else if (occ_k == 2) {
        if (dense) SBWT_EMU_IN_PLACE(2, kInsertThreads); else SBWT_EMU_IN_PLACE(2, kInsertThreadsSparse);
    } else {
        if (dense) SBWT_EMU_IN_PLACE(1, kInsertThreads); else SBWT_EMU_IN_PLACE(1, kInsertThreadsSparse);
    }
#undef SBWT_EMU_IN_PLACE
    return 0;
}

// spread_old of one output part: the window's three planes and the part's
// new-row mask in, the spread planes out
extern "C" void emu_spread_old(const unsigned long long* in, unsigned long long F, unsigned long long* out) {
    const Window w = spread_old(Window{in[0], in[1], in[2]}, F);
    out[0] = w.lo;
    out[1] = w.hi;
    out[2] = w.dm;
}
