// Host emulation of the suffix sort's key arithmetic (suffix_sort.cu), for
// CPU tests: the 63-bit key of a suffix (its first H codes, zeroed at and
// past its terminator, and its length field) and the dense bucket numbers
// of the bucket split, for 2-bit codes and for 4-bit codes in base sigma.
//
// The device functions are compiled here unchanged (the test cuts them out
// of the CUDA source into the .inc files below) on cuda_emu.h; they run on
// one host thread, as they are per-element functions.
#include <cstdlib>

#include "cuda_emu.h"

#include "constants.inc"
#include "keys.inc"

// bucket_digit (2-bit codes) of each key.
extern "C" int emu_bucket_digit(uint64_t count, const unsigned long long* keys, uint32_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = bucket_digit(keys[i]);
    return 0;
}

// bucket_digit_sigma (4-bit codes, buckets of pw codes in base sigma).
extern "C" int emu_bucket_digit_sigma(uint64_t count, const unsigned long long* keys, uint32_t sigma, uint32_t pw,
                                      uint32_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = bucket_digit_sigma(keys[i], sigma, pw);
    return 0;
}

// initial_key and key_with_len (the latter given the length field the
// former found) at each position, code width kb.  text and term are copied
// into 16-byte aligned buffers with the padding the kernels read past the
// end.
extern "C" int emu_keys(int kb, const uint32_t* text, uint64_t text_words, const uint32_t* term, uint64_t term_words,
                        uint64_t count, const uint64_t* pos, unsigned long long* init_out,
                        unsigned long long* with_len_out) {
    const uint64_t tw = (text_words + 8 + 3) & ~3ull;
    uint32_t* t = static_cast<uint32_t*>(std::aligned_alloc(16, tw * 4));
    uint32_t* b = static_cast<uint32_t*>(std::aligned_alloc(16, ((term_words + 4 + 3) & ~3ull) * 4));
    if (!t || !b) return 1;
    memset(t, 0, tw * 4);
    memset(b, 0, ((term_words + 4 + 3) & ~3ull) * 4);
    memcpy(t, text, text_words * 4);
    memcpy(b, term, term_words * 4);
    for (uint64_t i = 0; i < count; ++i) {
        if (kb == 2) {
            init_out[i] = initial_key<2>(t, b, pos[i]);
            with_len_out[i] = key_with_len<2>(t, pos[i], (uint32_t)(init_out[i] & 31));
        } else {
            init_out[i] = initial_key<4>(t, b, pos[i]);
            with_len_out[i] = key_with_len<4>(t, pos[i], (uint32_t)(init_out[i] & 31));
        }
    }
    std::free(t);
    std::free(b);
    return 0;
}
