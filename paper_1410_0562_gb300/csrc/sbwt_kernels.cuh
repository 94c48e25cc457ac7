// sbwt_kernels.cuh -- host-side launchers of the set-bwte kernels (one .cu
// file each); the runtime in capi.cu strings them together per block.
#pragma once

#include "sbwt_internal.cuh"

namespace sbwt {

// The alphabet of an index, by value (a kernel parameter).
struct Alphabet16 {
    uint8_t a[16];
};

// pack.cu: reads + offsets (device) -> 2-bit text and terminator bitmap of
// the whole append; sets *d_err != 0 when a byte is outside the alphabet.
// [w_begin, w_end) limits the launch to those 32-position words (the bytes
// of their positions must be in d_reads already).
void launch_pack(Launcher& L, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m, uint64_t npos,
                 uint32_t alpha4, int sigma, uint32_t* text, uint32_t* term, uint32_t* d_err, uint64_t w_begin = 0,
                 uint64_t w_end = ~0ull);
// The same with 4-bit codes (5 to 16 symbols); text starts on a 16-byte boundary.
void launch_pack_w(Launcher& L, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m, uint64_t npos,
                   const Alphabet16& alpha, int sigma, uint32_t* text, uint32_t* term, uint32_t* d_err,
                   uint64_t w_begin = 0, uint64_t w_end = ~0ull);

// suffix_sort.cu: ConstructSA of one block of n suffixes starting at text
// position `base`.  Results: sa (SA_int), rank (its inverse).
struct SuffixSortBuffers {
    unsigned long long *keys, *keys_alt;  // n each
    uint32_t *vals, *vals_alt;            // n each
    uint32_t *sa, *rank;                  // n each
    uint32_t *act_pos[2], *act_suf[2];    // n each: unsorted members of the device-wide path
    uint32_t *loc_act, *loc_next;         // n each: unsorted members of the CTA-local units, their next ranks
    void* units;                          // suffix_sort_unit_bytes(n): one record per window of rows
    uint32_t* radix_temp;                 // radix_temp_words(n)
    unsigned long long* chunks;           // suffix_sort_chunk_words(n): per-chunk (max, count) pairs
    uint32_t* count_log;                  // suffix_sort_log_slots(max_len) words, 8-byte aligned
    uint32_t* err;                        // error flags (bits 2..7)
};
void suffix_sort_init();  // once per device (includes radix_init)
// code_bits: 2 (alphabets of up to 4 symbols) or 4 (5 to 16 symbols)
uint32_t suffix_sort_rounds(uint32_t max_len, int code_bits);
size_t suffix_sort_log_slots(uint32_t max_len, int code_bits);
size_t suffix_sort_chunk_words(uint64_t cap);
size_t suffix_sort_unit_bytes(uint64_t cap);
void suffix_sort_block(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, uint32_t n,
                       uint32_t max_len, int code_bits, int sigma, const SuffixSortBuffers& b);

// ranks.cu
// B_int[i] = code of the symbol before block suffix SA[i], kBintDollar at a
// read start (Algorithm 1, B(S_jk, SA_int)).
void launch_bint(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, const uint32_t* sa,
                 uint32_t n, uint8_t* bint);
// ComputeRanks (Algorithm 2 with Lemma 1): g[t] for every block position.
// A row index past n_ext (impossible for a consistent dictionary) is clamped
// and flagged in *d_err (bit 3) instead of being dereferenced.  blocks is the
// bit-plane dictionary of sampling 64 occ_k rows for code_bits == 2 (occ_k
// 1, 2 or 4), an OccBlockW array for code_bits == 4 (occ_k 1); g starts on a
// 16-byte boundary.
// max_len bounds the block's read lengths: reads longer than 2 seg_rows
// symbols are ranked in segments of seg_rows positions, each started exactly
// by a backward search (see ranks.cu).
template <class IdxT>
void launch_compute_ranks(Launcher& L, const uint32_t* text, const uint64_t* d_offsets, uint64_t j_begin,
                          uint64_t nreads, uint64_t n_int, uint64_t max_len, const void* blocks,
                          const unsigned long long* super, const unsigned long long* d_C, uint64_t n_ext,
                          uint64_t m_ext, IdxT* g, uint32_t* d_err, int code_bits, int occ_k, uint32_t seg_rows = 256);
// B_int and g_sa fused: one pass over SA_int after ComputeRanks.  With
// ins_i0 non-null it also writes Insert's plan (nsb + 1 entries: the first
// new symbol of each superblock of 2^super_shift rows of the next dictionary).
template <class IdxT>
void launch_bint_gather(Launcher& L, const uint32_t* text, const uint32_t* term, uint64_t base, const uint32_t* sa,
                        const IdxT* g, uint32_t n, uint8_t* bint, IdxT* gsa, int code_bits, uint32_t* ins_i0 = nullptr,
                        uint64_t nsb = 0, int super_shift = 0);
// rank queries: codes 0..sigma-1, or 4 (16 for code_bits == 4) for the terminator.
void launch_rank_batch(Launcher& L, const void* blocks, const unsigned long long* super, const uint8_t* codes,
                       const unsigned long long* ks, uint64_t q, unsigned long long* out, int code_bits, int occ_k);
// Backward-search counts of q patterns (pattern i = pats[offs[i] .. offs[i+1])).
void launch_count(Launcher& L, const void* blocks, const unsigned long long* super, const unsigned long long* d_C,
                  uint64_t n, const Alphabet16& alpha, int sigma, const uint8_t* pats, const uint64_t* offs,
                  uint64_t q, uint64_t total_len, unsigned long long* out, int code_bits, int occ_k);
// B as bytes, rows [r0, r1) (r0 a multiple of 64): alphabet byte per code,
// '$' for a terminator row; out[r] for row r.
void launch_unpack(Launcher& L, const void* blocks, uint64_t r0, uint64_t r1, const Alphabet16& alpha, uint8_t* out,
                   int code_bits, int occ_k);

// insert.cu: Insert (Section 5) as a stable merge of the old dictionary
// (n_ext rows) with n_int new symbols at rows g_sa[i] + i; writes the new
// dictionary's symbols, terminator masks and block counters, then the
// superblock counters and C[] (m = terminators in the new dictionary).
// Blocks are the bit-plane dictionary of sampling 64 occ_k rows (code_bits
// 2) or OccBlockW (code_bits 4, occ_k 1); sb_tot holds 4 (16) words per
// superblock, rounded up to 4 words, then 4 (16) 64-bit words per 256
// superblocks.  ins_i0 is the plan bint_gather wrote (2-bit dictionary;
// unused for 4-bit codes); an inconsistent plan sets *d_err bit 10.
// With `stage`, new_blocks is old_blocks: the dictionary is rewritten in
// place, from the top superblock down in chunks, each chunk's old blocks
// first copied to `stage` (stage_blocks dictionary blocks, in HBM, at least
// insert_stage_blocks(code_bits, occ_k, n_new)).  insert_threads: 256 or
// 512 threads per CTA of the 2-bit Insert, 0 = 512 while a quarter or more
// of the result's rows are new, else 256.
template <class IdxT>
void launch_insert(Launcher& L, const void* old_blocks, uint64_t n_ext, const uint8_t* bint, const IdxT* gsa,
                   uint64_t n_int, const uint32_t* ins_i0, void* new_blocks, unsigned long long* new_super,
                   unsigned long long* new_C, uint64_t m_new, uint32_t* sb_tot, uint32_t* d_err, int code_bits,
                   int occ_k, unsigned long long* stage = nullptr, uint64_t stage_blocks = 0,
                   int insert_threads = 0);
uint64_t insert_stage_blocks(int code_bits, int occ_k, uint64_t n_final);

// plan.cu: checks device-resident offsets (offsets[0] = 0, non-decreasing,
// every read shorter than max_block suffixes; summary->bad != 0 otherwise),
// finds the longest read and writes the greedy block partition (Algorithm 1:
// whole reads, at most M suffixes per block unless one read is longer) into
// table[0 .. min(blocks, cap)); summary->blocks is the number of blocks.
struct PlanBlock {
    unsigned long long j0, j1;  // reads [j0, j1)
    unsigned long long base;    // text position of the block's first suffix
    unsigned long long n_int;   // suffixes in the block
};
struct PlanSummary {
    unsigned int bad;
    unsigned int blocks;
    unsigned long long max_len;
    unsigned long long npos;  // suffixes in the whole append
};
void launch_plan(Launcher& L, const uint64_t* d_offsets, uint64_t m, uint64_t M, uint64_t max_block,
                 PlanBlock* table, unsigned cap, PlanSummary* summary);

// Sizes of a dictionary of n rows: occurrence blocks of 64 k rows (k = 1, 2
// or 4 for the 2-bit layout, 1 for the 4-bit one).
inline uint64_t dict_blocks(uint64_t n, int k = 1) { return n / (64ull * (uint64_t)k) + 1; }
inline uint64_t dict_supers(uint64_t n) { return (n >> kSuperShift) + 1; }
inline uint64_t dict_supers_w(uint64_t n) { return (dict_blocks(n) + kBlocksPerSuperW - 1) / kBlocksPerSuperW; }
// Bytes per occurrence block, superblock counters and C of each layout.
inline size_t dict_block_bytes(int code_bits, int k = 1) {
    return code_bits == 4 ? sizeof(OccBlockW) : (size_t)8 * (3 * k + 1);
}
inline uint64_t dict_supers_of(uint64_t n, int code_bits) { return code_bits == 4 ? dict_supers_w(n) : dict_supers(n); }
inline size_t dict_codes(int code_bits) { return code_bits == 4 ? (size_t)kSigmaW : 4; }

}  // namespace sbwt
