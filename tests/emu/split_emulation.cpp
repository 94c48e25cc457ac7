// Host emulation of the front of the bucket split (suffix_sort.cu), for CPU
// tests: sa_digit_keys (each suffix's element and the first radix pass's
// per-chunk digit counts) and sa_unit_begin (per window of the
// bucket-sorted elements: the first bucket start and the long-suffix counts;
// SA and rank of the short suffixes; the list of long rows with their keys),
// then the unit scan and the global-path gather of units too large for a CTA.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h:
// one std::thread per GPU thread, warp intrinsics and CTA barriers emulated,
// every array between inaccessible pages.
#include "cuda_emu.h"

#include "radix_hdr.inc"
#include "scan.inc"
#include "constants.inc"
#include "keys.inc"
#include "digit_keys.inc"
#include "unit_begin.inc"
#include "unit_scan.inc"
#include "large_gather.inc"

namespace {
// the packed text with the padding the kernels read past its end, its size
// a multiple of 16 bytes (guarded() then places it on a 16-byte boundary)
uint64_t text_alloc_words(uint64_t text_words) { return (text_words + 4 + 3) & ~3ull; }
}  // namespace

// sa_digit_keys over positions 0 .. n-1 with a grid of `grid` CTAs.  counts
// (grid x 256) and totals (256) are read and written as the kernel leaves
// them.
extern "C" int emu_digit_keys(int kb, const uint32_t* text, uint64_t text_words, const uint32_t* term,
                              uint64_t term_words, uint32_t n, uint32_t sigma, uint32_t pw, uint32_t grid,
                              unsigned long long* elems, uint32_t* counts, uint32_t* totals, uint32_t* n_out) {
    std::vector<std::pair<void*, size_t>> maps;
    std::vector<uint32_t> t(text_alloc_words(text_words), 0u), b(term_words + 2, 0u);
    memcpy(t.data(), text, text_words * 4);
    memcpy(b.data(), term, term_words * 4);
    const uint32_t* g_text = guarded(t.data(), t.size(), maps);
    const uint32_t* g_term = guarded(b.data(), b.size(), maps);
    unsigned long long* g_elems = guarded(elems, n ? n : 1, maps);
    uint32_t* g_counts = guarded(counts, (size_t)grid * kRadixBins, maps);
    uint32_t* g_totals = guarded(totals, kRadixBins, maps);
    uint32_t* g_n = guarded(n_out, 1, maps);
    run_grid(grid, kKeyThreads, [&] {
        if (kb == 2)
            sa_digit_keys_kernel<2>(g_text, g_term, 0ull, n, sigma, pw, g_elems, g_n, g_counts, g_totals);
        else
            sa_digit_keys_kernel<4>(g_text, g_term, 0ull, n, sigma, pw, g_elems, g_n, g_counts, g_totals);
    });
    memcpy(elems, g_elems, n * 8ull);
    memcpy(counts, g_counts, (size_t)grid * kRadixBins * 4);
    memcpy(totals, g_totals, kRadixBins * 4);
    *n_out = *g_n;
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// sa_unit_begin over the bucket-sorted elements (nwin windows) with a grid
// of `grid` CTAs.  ll_* hold nwin * kWindow entries.
extern "C" int emu_unit_begin(int kb, const uint32_t* text, uint64_t text_words, const unsigned long long* elems,
                              uint32_t n, uint32_t nwin, uint32_t* beg, uint32_t* lcb, uint32_t* lct, uint32_t* sa,
                              uint32_t* rank, uint32_t* ll_t, uint32_t* ll_row, unsigned long long* ll_key,
                              uint32_t* d_err, unsigned grid) {
    std::vector<std::pair<void*, size_t>> maps;
    std::vector<uint32_t> t(text_alloc_words(text_words), 0u);
    memcpy(t.data(), text, text_words * 4);
    const uint32_t* g_text = guarded(t.data(), t.size(), maps);
    const unsigned long long* g_elems = guarded(elems, n, maps);
    uint32_t* g_beg = guarded(beg, nwin, maps);
    uint32_t* g_lcb = guarded(lcb, nwin, maps);
    uint32_t* g_lct = guarded(lct, nwin, maps);
    uint32_t* g_sa = guarded(sa, n, maps);
    uint32_t* g_rank = guarded(rank, n, maps);
    const size_t slots = (size_t)nwin * kWindow;
    uint32_t* g_ll_t = guarded(ll_t, slots, maps);
    uint32_t* g_ll_row = guarded(ll_row, slots, maps);
    unsigned long long* g_ll_key = guarded(ll_key, slots, maps);
    Units u{g_beg, g_lcb, g_lct, nullptr, nullptr, nullptr, nullptr, nullptr};
    run_grid(grid, kThreads, [&] {
        if (kb == 2)
            sa_unit_begin_kernel<2>(g_text, 0ull, g_elems, n, nwin, u, g_sa, g_rank, g_ll_t, g_ll_row, g_ll_key,
                                    d_err);
        else
            sa_unit_begin_kernel<4>(g_text, 0ull, g_elems, n, nwin, u, g_sa, g_rank, g_ll_t, g_ll_row, g_ll_key,
                                    d_err);
    });
    memcpy(beg, g_beg, nwin * 4ull);
    memcpy(lcb, g_lcb, nwin * 4ull);
    memcpy(lct, g_lct, nwin * 4ull);
    memcpy(sa, g_sa, n * 4ull);
    memcpy(rank, g_rank, n * 4ull);
    memcpy(ll_t, g_ll_t, slots * 4);
    memcpy(ll_row, g_ll_row, slots * 4);
    memcpy(ll_key, g_ll_key, slots * 8);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// The chain after the bucket sort for one block: sa_unit_begin, the unit
// scan (one CTA) and the global-path gather, over the bucket-sorted
// elements.  fields: the unit table, 8 fields of `stride` words (the device
// layout); lkeys/lvals/lpos hold n entries; *d_large the list's size.
extern "C" int emu_large_chain(int kb, const uint32_t* text, uint64_t text_words, const unsigned long long* elems,
                               uint32_t n, uint32_t nwin, uint64_t stride, uint32_t* fields, uint32_t* sa,
                               uint32_t* rank, unsigned long long* lkeys, uint32_t* lvals, uint32_t* lpos,
                               uint32_t* d_large, uint32_t* d_err) {
    std::vector<std::pair<void*, size_t>> maps;
    std::vector<uint32_t> t(text_alloc_words(text_words), 0u);
    memcpy(t.data(), text, text_words * 4);
    const uint32_t* g_text = guarded(t.data(), t.size(), maps);
    const unsigned long long* g_elems = guarded(elems, n, maps);
    uint32_t* g = guarded(fields, stride * 8, maps);
    Units u{g, g + stride, g + 2 * stride, g + 3 * stride, g + 4 * stride, g + 5 * stride, g + 6 * stride,
            g + 7 * stride};
    uint32_t* g_sa = guarded(sa, n, maps);
    uint32_t* g_rank = guarded(rank, n, maps);
    const size_t slots = (size_t)nwin * kWindow;
    std::vector<uint32_t> ll_t(slots), ll_row(slots);
    std::vector<unsigned long long> ll_key(slots);
    uint32_t* g_ll_t = guarded(ll_t.data(), slots, maps);
    uint32_t* g_ll_row = guarded(ll_row.data(), slots, maps);
    unsigned long long* g_ll_key = guarded(ll_key.data(), slots, maps);
    unsigned long long* g_lkeys = guarded(lkeys, n, maps);
    uint32_t* g_lvals = guarded(lvals, n, maps);
    uint32_t* g_lpos = guarded(lpos, n, maps);
    uint32_t* g_large = guarded(d_large, 1, maps);
    std::vector<uint32_t> zero(4, 0u);
    uint32_t* g_zero = guarded(zero.data(), zero.size(), maps);
    run_grid(3, kThreads, [&] {
        if (kb == 2)
            sa_unit_begin_kernel<2>(g_text, 0ull, g_elems, n, nwin, u, g_sa, g_rank, g_ll_t, g_ll_row, g_ll_key,
                                    d_err);
        else
            sa_unit_begin_kernel<4>(g_text, 0ull, g_elems, n, nwin, u, g_sa, g_rank, g_ll_t, g_ll_row, g_ll_key,
                                    d_err);
    });
    run_grid(1, kScanThreads, [&] { sa_unit_scan_kernel(u, nwin, n, g_large, g_zero, 1, 1, g_zero + 2, 1); });
    run_grid(5, kThreads, [&] {
        if (kb == 2)
            sa_large_gather_kernel<2>(g_text, 0ull, n, g_elems, u, nwin, g_lkeys, g_lvals, g_lpos, g_large);
        else
            sa_large_gather_kernel<4>(g_text, 0ull, n, g_elems, u, nwin, g_lkeys, g_lvals, g_lpos, g_large);
    });
    memcpy(fields, g, stride * 8 * 4);
    memcpy(sa, g_sa, n * 4ull);
    memcpy(rank, g_rank, n * 4ull);
    memcpy(lkeys, g_lkeys, n * 8ull);
    memcpy(lvals, g_lvals, n * 4ull);
    memcpy(lpos, g_lpos, n * 4ull);
    *d_large = *g_large;
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
