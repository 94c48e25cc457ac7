// Host emulation of the ComputeRanks kernels of ranks.cu (Algorithm 2 with
// Lemma 1), for CPU tests.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h: one
// std::thread per GPU thread, every array between inaccessible pages.
#include "cuda_emu.h"

alignas(16) static unsigned long long g_dyn_smem[48 * 1024 / 8];  // the superblock counters' stage

namespace sbwt {
#include "dict.inc"
#include "ranks.inc"
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
