// Host emulation of the ComputeRanks kernels of ranks.cu (Algorithm 2 with
// Lemma 1), for CPU tests.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h: one
// std::thread per GPU thread, every array between inaccessible pages.
#include "cuda_emu.h"

alignas(16) static unsigned long long g_dyn_smem[48 * 1024 / 8];  // the superblock counters' stage

namespace sbwt {
#include "alphabet.inc"
#include "text.inc"
#include "dict.inc"
#include "bint.inc"
#include "ranks.inc"
#include "gather.inc"
#include "queries.inc"
#include "unpack.inc"
#include "unpack_w.inc"
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

// rank(c, k) queries (c = 4: the terminator) and FM-index counts of
// patterns over the 2-bit dictionary of sampling 64 K rows (n rows), and
// the read-back of rows [r0, r1) (r0 a multiple of 64) as bytes.
template <int K>
static void run_queries(const unsigned long long* words, const unsigned long long* super, const unsigned long long* C,
                        unsigned long long n, const uint8_t* codes, const unsigned long long* ks, uint64_t q,
                        unsigned long long* rank_out, const uint8_t* pats, uint64_t pat_bytes,
                        const unsigned long long* offs, uint64_t npat, unsigned long long* count_out,
                        unsigned long long r0, unsigned long long r1, uint8_t* bytes) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nw = (n / (64ull * K) + 1) * Occ<K>::kWords, nsb = (n >> 16) + 1;
    const unsigned long long* g_words = guarded(words, nw, maps);
    const unsigned long long* g_super = guarded(super, 4 * nsb, maps);
    const unsigned long long* g_C = guarded(C, 4, maps);
    const uint8_t* g_codes = guarded(codes, q ? q : 1, maps);
    const unsigned long long* g_ks = guarded(ks, q ? q : 1, maps);
    unsigned long long* g_rank = guarded(rank_out, q ? q : 1, maps);
    const uint8_t* g_pats = guarded(pats, pat_bytes ? pat_bytes : 1, maps);
    const unsigned long long* g_offs = guarded(offs, npat + 1, maps);
    unsigned long long* g_count = guarded(count_out, npat ? npat : 1, maps);
    // the read-back's output: whole 16-byte rows of the parts it writes
    const size_t out_bytes = (size_t)((n + 63) / 64 * 64);
    uint8_t* g_bytes = guarded(bytes, out_bytes, maps);
    Alphabet16 alpha{};
    const char* acgt = "ACGT";
    for (int a = 0; a < 4; ++a) alpha.a[a] = (uint8_t)acgt[a];
    const uint32_t alpha4 = 'A' | ('C' << 8) | ('G' << 16) | ((uint32_t)'T' << 24);
    run_grid((unsigned)((q + kThreads - 1) / kThreads), kThreads,
             [&] { rank_batch_kernel<2, K>(g_words, g_super, g_codes, g_ks, q, g_rank); });
    run_grid((unsigned)((npat + kThreads - 1) / kThreads), kThreads,
             [&] { count_kernel<2, K>(g_words, g_super, g_C, n, alpha, 4, g_pats, g_offs, npat, g_count); });
    const uint64_t parts = (r1 + 63) / 64 - r0 / 64;
    run_grid((unsigned)((parts + kThreads - 1) / kThreads), kThreads,
             [&] { unpack_kernel<K>(g_words, r0, r1, alpha4, g_bytes); });
    memcpy(rank_out, g_rank, q * 8);
    memcpy(count_out, g_count, npat * 8);
    memcpy(bytes, g_bytes, out_bytes);
    for (auto& m : maps) munmap(m.first, m.second);
}

extern "C" int emu_queries(int k, const unsigned long long* words, const unsigned long long* super,
                           const unsigned long long* C, unsigned long long n, const uint8_t* codes,
                           const unsigned long long* ks, uint64_t q, unsigned long long* rank_out, const uint8_t* pats,
                           uint64_t pat_bytes, const unsigned long long* offs, uint64_t npat,
                           unsigned long long* count_out, unsigned long long r0, unsigned long long r1,
                           uint8_t* bytes) {
    if (k == 4)
        run_queries<4>(words, super, C, n, codes, ks, q, rank_out, pats, pat_bytes, offs, npat, count_out, r0, r1, bytes);
    else if (k == 2)
        run_queries<2>(words, super, C, n, codes, ks, q, rank_out, pats, pat_bytes, offs, npat, count_out, r0, r1, bytes);
    else
        run_queries<1>(words, super, C, n, codes, ks, q, rank_out, pats, pat_bytes, offs, npat, count_out, r0, r1, bytes);
    return 0;
}

// The same over the 4-bit dictionary (blocks of 64 rows, superblocks of
// 4096 rows, 16 codes; c = 16: the terminator), alphabet of sigma symbols.
extern "C" int emu_queries_w(const OccBlockW* blocks, const unsigned long long* super, const unsigned long long* C,
                             unsigned long long n, const uint8_t* alpha_bytes, int sigma, const uint8_t* codes,
                             const unsigned long long* ks, uint64_t q, unsigned long long* rank_out,
                             const uint8_t* pats, uint64_t pat_bytes, const unsigned long long* offs, uint64_t npat,
                             unsigned long long* count_out, unsigned long long r0, unsigned long long r1,
                             uint8_t* bytes) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nb = (n >> kOccShift) + 1, nsb = (nb + kBlocksPerSuperW - 1) / kBlocksPerSuperW;
    const OccBlockW* g_blocks = guarded(blocks, nb, maps);
    const unsigned long long* g_super = guarded(super, (size_t)kSigmaW * nsb, maps);
    const unsigned long long* g_C = guarded(C, kSigmaW, maps);
    const uint8_t* g_codes = guarded(codes, q ? q : 1, maps);
    const unsigned long long* g_ks = guarded(ks, q ? q : 1, maps);
    unsigned long long* g_rank = guarded(rank_out, q ? q : 1, maps);
    const uint8_t* g_pats = guarded(pats, pat_bytes ? pat_bytes : 1, maps);
    const unsigned long long* g_offs = guarded(offs, npat + 1, maps);
    unsigned long long* g_count = guarded(count_out, npat ? npat : 1, maps);
    const size_t out_bytes = (size_t)((n + 63) / 64 * 64);
    uint8_t* g_bytes = guarded(bytes, out_bytes, maps);
    Alphabet16 alpha{};
    for (int a = 0; a < sigma && a < 16; ++a) alpha.a[a] = alpha_bytes[a];
    run_grid((unsigned)((q + kThreads - 1) / kThreads), kThreads,
             [&] { rank_batch_kernel<4, 1>(g_blocks, g_super, g_codes, g_ks, q, g_rank); });
    run_grid((unsigned)((npat + kThreads - 1) / kThreads), kThreads,
             [&] { count_kernel<4, 1>(g_blocks, g_super, g_C, n, alpha, sigma, g_pats, g_offs, npat, g_count); });
    const uint64_t parts = (r1 + 63) / 64 - r0 / 64;
    run_grid((unsigned)((parts + kThreads - 1) / kThreads), kThreads,
             [&] { unpack_w_kernel(g_blocks, r0, r1, alpha, g_bytes); });
    memcpy(rank_out, g_rank, q * 8);
    memcpy(count_out, g_count, npat * 8);
    memcpy(bytes, g_bytes, out_bytes);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// ComputeRanks over the 4-bit dictionary (text of 4-bit codes, 8 per word),
// the per-read (seg = 0) or segmented kernel, with the superblock counters
// staged in shared memory or read from global memory.
template <bool kStage>
static void run_w(int seg, uint32_t segs, uint32_t seg_rows, const uint32_t* text, uint64_t text_words,
                  const unsigned long long* offsets, unsigned long long nreads, const OccBlockW* blocks,
                  const unsigned long long* super, const unsigned long long* C, unsigned long long n_ext,
                  unsigned long long m_start, uint32_t* g, uint64_t n_int, uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t nb = (n_ext >> kOccShift) + 1, nsb = (n_ext >> kSuperShiftW) + 1;
    const uint32_t* g_text = guarded(text, text_words, maps);
    const unsigned long long* g_off = guarded(offsets, nreads + 1, maps);
    const OccBlockW* g_blocks = guarded(blocks, nb, maps);
    const unsigned long long* g_super = guarded(super, (size_t)kSigmaW * nsb, maps);
    const unsigned long long* g_C = guarded(C, kSigmaW, maps);
    uint32_t* g_g = guarded(g, n_int, maps);
    const uint64_t threads = seg ? nreads * segs : nreads;
    run_grid((unsigned)((threads + kThreads - 1) / kThreads), kThreads, [&] {
        if (seg)
            compute_ranks_seg_kernel<uint32_t, kStage, 4, 1>(g_text, g_off, 0, nreads, segs, seg_rows, g_blocks,
                                                            g_super, g_C, n_ext, m_start, g_g, d_err);
        else
            compute_ranks_kernel<uint32_t, kStage, 4, 1>(g_text, g_off, 0, nreads, g_blocks, g_super, g_C, n_ext,
                                                        m_start, g_g, d_err);
    });
    memcpy(g, g_g, n_int * 4);
    for (auto& m : maps) munmap(m.first, m.second);
}

extern "C" int emu_compute_ranks_w(int staged, int seg, uint32_t segs, uint32_t seg_rows, const uint32_t* text,
                                   uint64_t text_words, const unsigned long long* offsets, unsigned long long nreads,
                                   const OccBlockW* blocks, const unsigned long long* super,
                                   const unsigned long long* C, unsigned long long n_ext, unsigned long long m_start,
                                   uint32_t* g, uint64_t n_int, uint32_t* d_err) {
    if (staged)
        run_w<true>(seg, segs, seg_rows, text, text_words, offsets, nreads, blocks, super, C, n_ext, m_start, g,
                    n_int, d_err);
    else
        run_w<false>(seg, segs, seg_rows, text, text_words, offsets, nreads, blocks, super, C, n_ext, m_start, g,
                     n_int, d_err);
    return 0;
}

// B_int by the one-block kernel (a block into an empty index): one thread
// per suffix, SA of n entries.
extern "C" int emu_bint_plain(const uint32_t* text, uint64_t text_words, const uint32_t* term, uint64_t term_words,
                              unsigned long long base, const uint32_t* sa, uint32_t n, uint8_t* bint) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_text = guarded(text, text_words, maps);
    const uint32_t* g_term = guarded(term, term_words, maps);
    const uint32_t* g_sa = guarded(sa, n ? n : 1, maps);
    uint8_t* g_bint = guarded(bint, n ? n : 1, maps);
    run_grid((n + kThreads - 1) / kThreads, kThreads, [&] { bint_kernel(g_text, g_term, base, g_sa, n, g_bint); });
    memcpy(bint, g_bint, n);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
