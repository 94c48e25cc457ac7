// pack.cu -- validates an append's reads against the alphabet and packs them
// into the text (2-bit codes, or 4-bit codes for 5 to 16 symbols) and the
// terminator bitmap every later kernel reads.
//
// Position rule: read j's symbol k sits at offsets[j] + j + k and its
// terminator at offsets[j+1] + j, i.e. every read is followed by one
// terminator slot (T = S_0 $_0 S_1 $_1 ..., Section 2 of arXiv 1410.0562).
// The byte behind position t of read j is therefore reads[t - j].
#include <algorithm>

#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;

// One thread per 32 positions: two MSB-first text words and one bitmap word.
__global__ void __launch_bounds__(kThreads) pack_kernel(const uint8_t* __restrict__ reads,
                                                        const unsigned long long* __restrict__ offsets,
                                                        unsigned long long m, unsigned long long npos,
                                                        uint32_t alpha4, int sigma, uint32_t* __restrict__ text,
                                                        uint32_t* __restrict__ term,
                                                        uint32_t* __restrict__ d_err, unsigned long long w_begin,
                                                        unsigned long long w_end) {
    const uint64_t w = w_begin + (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t t0 = w * 32;
    if (w >= w_end || t0 >= npos) return;
    // read holding t0: the last j with offsets[j] + j <= t0
    uint64_t lo = 0, hi = m;  // invariant: offsets[lo] + lo <= t0 < offsets[hi] + hi
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (offsets[mid] + mid <= t0) lo = mid; else hi = mid;
    }
    uint64_t j = lo;
    uint64_t end_j = offsets[j + 1] + j;  // terminator position of read j
    uint32_t tw[2] = {0u, 0u}, bw = 0u;
    bool bad = false;
    const uint32_t a0 = alpha4 & 0xFF, a1 = (alpha4 >> 8) & 0xFF, a2 = (alpha4 >> 16) & 0xFF, a3 = alpha4 >> 24;
    for (int q = 0; q < 32; ++q) {
        const uint64_t t = t0 + q;
        if (t >= npos) break;
        uint32_t code = 0;
        if (t == end_j) {
            bw |= 1u << q;
            ++j;
            if (j < m) end_j = offsets[j + 1] + j;
        } else {
            const uint32_t b = reads[t - j];
            if (b == a0) code = 0;
            else if (sigma > 1 && b == a1) code = 1;
            else if (sigma > 2 && b == a2) code = 2;
            else if (sigma > 3 && b == a3) code = 3;
            else bad = true;
        }
        tw[q >> 4] |= code << (30 - 2 * (q & 15));
    }
    text[2 * w] = tw[0];
    text[2 * w + 1] = tw[1];
    term[w] = bw;
    if (bad) atomicOr(d_err, 1u);
}

// The same for 4-bit codes (alphabets of 5 to 16 symbols): four text words
// per 32 positions; a byte's code comes from a 256-entry table in shared
// memory (0xFF: not in the alphabet).
__global__ void __launch_bounds__(kThreads) pack_w_kernel(const uint8_t* __restrict__ reads,
                                                          const unsigned long long* __restrict__ offsets,
                                                          unsigned long long m, unsigned long long npos,
                                                          Alphabet16 alpha, int sigma, uint32_t* __restrict__ text,
                                                          uint32_t* __restrict__ term,
                                                          uint32_t* __restrict__ d_err, unsigned long long w_begin,
                                                          unsigned long long w_end) {
    __shared__ uint8_t code_of[256];
    code_of[threadIdx.x] = 0xFF;
    __syncthreads();
    if ((int)threadIdx.x < sigma) code_of[alpha.a[threadIdx.x]] = (uint8_t)threadIdx.x;
    __syncthreads();
    const uint64_t w = w_begin + (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t t0 = w * 32;
    if (w >= w_end || t0 >= npos) return;
    uint64_t lo = 0, hi = m;  // invariant: offsets[lo] + lo <= t0 < offsets[hi] + hi
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (offsets[mid] + mid <= t0) lo = mid; else hi = mid;
    }
    uint64_t j = lo;
    uint64_t end_j = offsets[j + 1] + j;
    uint32_t tw[4] = {0u, 0u, 0u, 0u}, bw = 0u;
    bool bad = false;
    for (int q = 0; q < 32; ++q) {
        const uint64_t t = t0 + q;
        if (t >= npos) break;
        uint32_t code = 0;
        if (t == end_j) {
            bw |= 1u << q;
            ++j;
            if (j < m) end_j = offsets[j + 1] + j;
        } else {
            code = code_of[reads[t - j]];
            if (code == 0xFF) {
                bad = true;
                code = 0;
            }
        }
        tw[q >> 3] |= code << (28 - 4 * (q & 7));
    }
    *reinterpret_cast<uint4*>(text + 4 * w) = make_uint4(tw[0], tw[1], tw[2], tw[3]);
    term[w] = bw;
    if (bad) atomicOr(d_err, 1u);
}

}  // namespace

void launch_pack_w(Launcher& L, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m, uint64_t npos,
                   const Alphabet16& alpha, int sigma, uint32_t* text, uint32_t* term, uint32_t* d_err,
                   uint64_t w_begin, uint64_t w_end) {
    w_end = std::min<uint64_t>(w_end, (npos + 31) / 32);
    if (w_end <= w_begin) return;
    const double pos = (double)std::min<uint64_t>(npos, w_end * 32) - (double)(w_begin * 32);
    const unsigned grid = ceil_div_u(w_end - w_begin, kThreads);
    SBWT_LAUNCH(L, "pack_reads", pos + 8.0 * (m + 1) * pos / npos + pos / 2.0 + pos / 8.0, 0, nullptr,
                pack_w_kernel, grid, kThreads, 0, d_reads, reinterpret_cast<const unsigned long long*>(d_offsets),
                (unsigned long long)m, (unsigned long long)npos, alpha, sigma, text, term, d_err,
                (unsigned long long)w_begin, (unsigned long long)w_end);
}

void launch_pack(Launcher& L, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m, uint64_t npos,
                 uint32_t alpha4, int sigma, uint32_t* text, uint32_t* term, uint32_t* d_err, uint64_t w_begin,
                 uint64_t w_end) {
    w_end = std::min<uint64_t>(w_end, (npos + 31) / 32);
    if (w_end <= w_begin) return;
    // per position: its byte (about one per position), the text and bitmap
    // writes; the offsets read by the binary searches
    const double pos = (double)std::min<uint64_t>(npos, w_end * 32) - (double)(w_begin * 32);
    const unsigned grid = ceil_div_u(w_end - w_begin, kThreads);
    SBWT_LAUNCH(L, "pack_reads", pos + 8.0 * (m + 1) * pos / npos + pos / 4.0 + pos / 8.0, 0, nullptr,
                pack_kernel, grid, kThreads, 0, d_reads, reinterpret_cast<const unsigned long long*>(d_offsets),
                (unsigned long long)m, (unsigned long long)npos, alpha4, sigma, text, term, d_err,
                (unsigned long long)w_begin, (unsigned long long)w_end);
}

}  // namespace sbwt
