// Host emulation of the ComputeRanks kernels of ranks.cu (Algorithm 2 with
// Lemma 1), for CPU tests.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h: one
// std::thread per GPU thread, every array between inaccessible pages.
#include "cuda_emu.h"

alignas(16) static unsigned long long g_dyn_smem[48 * 1024 / 8];  // the superblock counters' stage

namespace sbwt {
#include "text.inc"
#include "dict.inc"
#include "ranks.inc"
#include "gather.inc"
}  // namespace sbwt
using namespace sbwt;

// One block's ComputeRanks: the per-read kernel (seg = 0) or the segmented
// one (seg = 1, `segs` segments of seg_rows positions per read) over the 2-bit dictionary of
// sampling 64 k rows (n_ext rows, as 64-bit words), its superblock counters
// and C[]; text, offsets as in an append of the block's reads alone;
// writes g (32-bit).
template <int K>
static void run_k(int seg, uint32_t segs, uint32_t seg_rows, const uint32_t* text, uint64_t text_words, const unsigned long long* offsets,
                  unsigned long long nreads, const unsigned long long* words, const unsigned long long* super,
                  const unsigned long long* C, unsigned long long n_ext, unsigned long long m_start, uint32_t* g,
                  uint64_t n_int, uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nw = (n_ext / (64ull * K) + 1) * Occ<K>::kWords, nsb = (n_ext >> 16) + 1;
    const uint32_t* g_text = guarded(text, text_words, maps);
    const unsigned long long* g_off = guarded(offsets, nreads + 1, maps);
    const unsigned long long* g_words = guarded(words, nw, maps);
    const unsigned long long* g_super = guarded(super, 4 * nsb, maps);
    const unsigned long long* g_C = guarded(C, 4, maps);
    uint32_t* g_g = guarded(g, n_int, maps);
    const uint64_t threads = seg ? nreads * segs : nreads;
    run_grid((unsigned)((threads + kThreads - 1) / kThreads), kThreads, [&] {
        if (seg)
            compute_ranks_seg_kernel<uint32_t, true, 2, K>(g_text, g_off, 0, nreads, segs, seg_rows, g_words, g_super,
                                                           g_C, n_ext, m_start, g_g, d_err);
        else
            compute_ranks_kernel<uint32_t, true, 2, K>(g_text, g_off, 0, nreads, g_words, g_super, g_C, n_ext, m_start,
                                                       g_g, d_err);
    });
    memcpy(g, g_g, n_int * 4);
    for (auto& m : maps) munmap(m.first, m.second);
}

extern "C" int emu_compute_ranks(int k, int seg, uint32_t segs, uint32_t seg_rows, const uint32_t* text, uint64_t text_words,
                                 const unsigned long long* offsets, unsigned long long nreads,
                                 const unsigned long long* words, const unsigned long long* super,
                                 const unsigned long long* C, unsigned long long n_ext, unsigned long long m_start,
                                 uint32_t* g, uint64_t n_int, uint32_t* d_err) {
    if (k == 4)
        run_k<4>(seg, segs, seg_rows, text, text_words, offsets, nreads, words, super, C, n_ext, m_start, g, n_int, d_err);
    else if (k == 2)
        run_k<2>(seg, segs, seg_rows, text, text_words, offsets, nreads, words, super, C, n_ext, m_start, g, n_int, d_err);
    else
        run_k<1>(seg, segs, seg_rows, text, text_words, offsets, nreads, words, super, C, n_ext, m_start, g, n_int, d_err);
    return 0;
}

// One gather of B_int, g_sa and Insert's plan over a block's SA_int (2-bit
// text, 32-bit index), as the library launches it: kGather elements per
// thread, CTAs of kThreads threads.
extern "C" int emu_bint_gather(const uint32_t* text, uint64_t text_words, const uint32_t* term, uint64_t term_words,
                               unsigned long long base, const uint32_t* sa, const uint32_t* g, uint64_t g_len,
                               uint32_t n, uint8_t* bint, uint32_t* gsa, uint32_t* ins_i0, unsigned long long nsb,
                               int super_shift) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_text = guarded(text, text_words, maps);
    const uint32_t* g_term = guarded(term, term_words, maps);
    const uint32_t* g_sa = guarded(sa, n, maps);
    const uint32_t* g_g = guarded(g, g_len, maps);
    uint8_t* g_bint = guarded(bint, n, maps);
    uint32_t* g_gsa = guarded(gsa, n, maps);
    uint32_t* g_plan = guarded(ins_i0, nsb + 1, maps);
    const uint64_t per_cta = (uint64_t)kThreads * kGather;
    run_grid((unsigned)((n + per_cta - 1) / per_cta), kThreads, [&] {
        bint_gather_kernel<uint32_t, 2>(g_text, g_term, base, g_sa, g_g, n, g_bint, g_gsa, g_plan, nsb, super_shift);
    });
    memcpy(bint, g_bint, n);
    memcpy(gsa, g_gsa, n * 4ull);
    memcpy(ins_i0, g_plan, (nsb + 1) * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
