// Host emulation of the read packing (pack.cu), for CPU tests: the 2-bit
// and 4-bit text words and the terminator bitmap of an append's reads.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA source into the .inc files below) on the emulation in cuda_emu.h:
// one std::thread per GPU thread, CTA barriers emulated, every array
// between inaccessible pages.
#include "cuda_emu.h"

#include "alphabet.inc"
constexpr int kThreads = 256;
#include "pack.inc"

// Packs words [w_begin, w_end) of npos positions.  text holds 2 (4) words
// and term 1 word per 32 positions; alpha holds sigma bytes.
extern "C" int emu_pack(int code_bits, const uint8_t* reads, uint64_t nbytes, const uint64_t* offsets, uint64_t m,
                        uint64_t npos, const uint8_t* alpha, int sigma, uint32_t* text, uint32_t* term,
                        uint32_t* d_err, uint64_t w_begin, uint64_t w_end) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint64_t words = (npos + 31) / 32;
    const int per = code_bits == 2 ? 2 : 4;
    const uint8_t* g_reads = guarded(reads, nbytes ? nbytes : 1, maps);
    const unsigned long long* g_off =
        guarded(reinterpret_cast<const unsigned long long*>(offsets), (size_t)m + 1, maps);
    uint32_t* g_text = guarded(text, (size_t)words * per, maps);
    uint32_t* g_term = guarded(term, (size_t)words, maps);
    const unsigned grid = (unsigned)((w_end - w_begin + kThreads - 1) / kThreads);
    if (code_bits == 2) {
        uint32_t alpha4 = 0;
        for (int i = 0; i < sigma && i < 4; ++i) alpha4 |= (uint32_t)alpha[i] << (8 * i);
        run_grid(grid, kThreads, [&] {
            pack_kernel(g_reads, g_off, m, npos, alpha4, sigma, g_text, g_term, d_err, w_begin, w_end);
        });
    } else {
        Alphabet16 a{};
        for (int i = 0; i < sigma && i < 16; ++i) a.a[i] = alpha[i];
        run_grid(grid, kThreads, [&] {
            pack_w_kernel(g_reads, g_off, m, npos, a, sigma, g_text, g_term, d_err, w_begin, w_end);
        });
    }
    memcpy(text, g_text, (size_t)words * per * 4);
    memcpy(term, g_term, (size_t)words * 4);
    for (auto& mp : maps) munmap(mp.first, mp.second);
    return 0;
}
