// Host emulation of the device-wide path's bookkeeping (suffix_sort.cu), for
// CPU tests: the keys of a doubling round's unsorted members
// (sa_round_keys) and the group pass over a sorted list (sa_groups_reduce,
// sa_groups_scan, sa_groups_apply: SA, ranks and the next member list).
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h:
// one std::thread per GPU thread, CTA barriers emulated, every array
// between inaccessible pages.
#include "cuda_emu.h"

#include "scan.inc"
#include "constants.inc"
#include "groups.inc"

extern "C" int emu_round_keys(const uint32_t* act_suf, uint32_t cnt, const uint32_t* rank, uint32_t h, uint32_t n,
                              int bits, unsigned long long* keys, uint32_t* vals, uint32_t* d_err, unsigned grid) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_act = guarded(act_suf, cnt ? cnt : 1, maps);
    const uint32_t* g_rank = guarded(rank, n, maps);
    const uint32_t* g_cnt = guarded(&cnt, 1, maps);
    unsigned long long* g_keys = guarded(keys, cnt ? cnt : 1, maps);
    uint32_t* g_vals = guarded(vals, cnt ? cnt : 1, maps);
    run_grid(grid, kThreads, [&] { sa_round_keys_kernel(g_act, g_cnt, g_rank, h, n, bits, g_keys, g_vals, d_err); });
    memcpy(keys, g_keys, cnt * 8ull);
    memcpy(vals, g_vals, cnt * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// The group pass over cnt sorted elements with a grid of `grid` CTAs;
// init: the list of the initial keys.  Returns the next list's size in
// *cnt_out.
extern "C" int emu_groups(int init, const unsigned long long* keys, const uint32_t* vals, const uint32_t* act_pos_in,
                          uint32_t cnt, uint32_t n_block, uint32_t* sa, uint32_t* rank, uint32_t* act_pos_out,
                          uint32_t* act_suf_out, uint32_t* cnt_out, uint32_t* d_err, unsigned grid) {
    std::vector<std::pair<void*, size_t>> maps;
    const unsigned long long* g_keys = guarded(keys, cnt ? cnt : 1, maps);
    const uint32_t* g_vals = guarded(vals, cnt ? cnt : 1, maps);
    const uint32_t* g_pos = guarded(act_pos_in, cnt ? cnt : 1, maps);
    const uint32_t* g_cnt = guarded(&cnt, 1, maps);
    uint32_t* g_sa = guarded(sa, n_block, maps);
    uint32_t* g_rank = guarded(rank, n_block, maps);
    uint32_t* g_pos_out = guarded(act_pos_out, n_block, maps);
    uint32_t* g_suf_out = guarded(act_suf_out, n_block, maps);
    std::vector<uint2> agg(grid);
    uint2* g_agg = guarded(agg.data(), grid, maps);
    uint32_t* g_cnt_out = guarded(cnt_out, 1, maps);
    if (init) {
        run_grid(grid, kThreads, [&] { sa_groups_reduce_kernel<true>(g_keys, g_pos, g_cnt, g_agg); });
    } else {
        run_grid(grid, kThreads, [&] { sa_groups_reduce_kernel<false>(g_keys, g_pos, g_cnt, g_agg); });
    }
    run_grid(1, kThreads, [&] { sa_groups_scan_kernel(g_agg, (int)grid, g_cnt_out); });
    if (init) {
        run_grid(grid, kThreads, [&] {
            sa_groups_apply_kernel<true>(g_keys, g_vals, g_pos, g_cnt, n_block, g_agg, g_sa, g_rank, g_pos_out,
                                         g_suf_out, d_err);
        });
    } else {
        run_grid(grid, kThreads, [&] {
            sa_groups_apply_kernel<false>(g_keys, g_vals, g_pos, g_cnt, n_block, g_agg, g_sa, g_rank, g_pos_out,
                                          g_suf_out, d_err);
        });
    }
    memcpy(sa, g_sa, n_block * 4ull);
    memcpy(rank, g_rank, n_block * 4ull);
    memcpy(act_pos_out, g_pos_out, n_block * 4ull);
    memcpy(act_suf_out, g_suf_out, n_block * 4ull);
    *cnt_out = *g_cnt_out;
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
