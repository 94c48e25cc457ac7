// Host emulation of the local-sort kernels of suffix_sort.cu, for CPU tests.
//
// The kernel text itself is compiled here (the test extracts it from the
// CUDA source into the .inc files this file includes): one std::thread per
// GPU thread of a CTA, warp intrinsics as exchanges through a per-warp
// barrier, __syncthreads through a CTA barrier, shared variables as
// statics (CTAs run one after another).  Every device array is copied into
// memory with an inaccessible page right after its last element and right
// before its first, so an access outside it faults.  A lane that skips an
// intrinsic its warp executes hangs the emulation (the test's timeout).
#include "cuda_emu.h"

#include "constants.inc"
alignas(16) static unsigned char g_dyn_smem[(size_t)kLSlots * 20];  // the larger of the two CTA kernels' needs
#include "scan.inc"
#include "unit_scan.inc"
#include "cta_local.inc"
#include "warp_local.inc"
#include "round_gather.inc"
#include "cta_round.inc"
#include "warp_round.inc"

// The initial local sort of one block: the warp kernel (unless use_warp is
// 0: then every local unit is marked for the CTA kernel), then the CTA kernel.
extern "C" int emu_local_sort(uint32_t n, const uint32_t* ll_t, const uint32_t* ll_row,
                              const unsigned long long* ll_key, uint32_t* beg, uint32_t* lcb, uint32_t* lct,
                              uint32_t* nlong, uint32_t* lofs, uint32_t* cnt, uint32_t nwin, uint32_t* sa,
                              uint32_t* rank, uint32_t* loc_act, uint32_t* d_cnt, uint32_t* d_err, int seg_shift,
                              unsigned warp_grid, unsigned cta_grid, int use_warp) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_ll_t = guarded(ll_t, n, maps);
    const uint32_t* g_ll_row = guarded(ll_row, n, maps);
    const unsigned long long* g_ll_key = guarded(ll_key, n, maps);
    uint32_t* g_sa = guarded(sa, n, maps);
    uint32_t* g_rank = guarded(rank, n, maps);
    uint32_t* g_loc = guarded(loc_act, n, maps);
    uint32_t* g_cnt = guarded(cnt, nwin, maps);
    Units u{guarded(beg, nwin, maps), guarded(lcb, nwin, maps), guarded(lct, nwin, maps), nullptr,
            guarded(nlong, nwin, maps), guarded(lofs, nwin, maps), g_cnt, nullptr};
    if (use_warp) {
        run_grid(warp_grid, kWWarps * 32, [&] {
            sa_local_sort_warp_kernel(n, g_ll_t, g_ll_row, g_ll_key, u, nwin, g_sa, g_rank, g_loc, d_cnt, seg_shift);
        });
    } else {
        for (uint32_t w = 0; w < nwin; ++w)
            if (u.beg[w] != kNone && u.lofs[w] == kNone && u.nlong[w] > 0) u.cnt[w] = kFallback;
    }
    run_grid(cta_grid, kLThreads, [&] {
        sa_local_sort_kernel(n, g_ll_t, g_ll_row, g_ll_key, u, nwin, g_sa, g_rank, g_loc, d_cnt, d_err, seg_shift);
    });
    memcpy(sa, g_sa, n * 4ull);
    memcpy(rank, g_rank, n * 4ull);
    memcpy(loc_act, g_loc, n * 4ull);
    memcpy(cnt, g_cnt, nwin * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// The next-rank gather of one round: loc_next[beg + k] = rank[loc_act[beg
// + k] + h] for the first cnt members of every local unit.
extern "C" int emu_round_gather(const uint32_t* loc_act, uint32_t* beg, uint32_t* lofs, uint32_t* cnt, uint32_t nwin,
                                const uint32_t* rank, uint32_t h, uint32_t n, uint32_t* loc_next, uint32_t* d_err,
                                unsigned grid) {
    std::vector<std::pair<void*, size_t>> maps;
    const uint32_t* g_loc = guarded(loc_act, n, maps);
    const uint32_t* g_rank = guarded(rank, n, maps);
    uint32_t* g_next = guarded(loc_next, n, maps);
    Units u{guarded(beg, nwin, maps), nullptr, nullptr, nullptr, nullptr, guarded(lofs, nwin, maps),
            guarded(cnt, nwin, maps), nullptr};
    run_grid(grid, kThreads, [&] { sa_round_gather_local_kernel(g_loc, u, nwin, g_rank, h, n, g_next, d_err); });
    memcpy(loc_next, g_next, n * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// One unit-local round: the warp kernel, then the CTA kernel.  *d_left
// (zero on entry) counts the units the warp kernel left to the CTA kernel.
extern "C" int emu_round(uint32_t* loc_act, const uint32_t* loc_next, uint32_t* beg, uint32_t* lofs, uint32_t* cnt,
                         uint32_t nwin, uint32_t n, uint32_t* rank, uint32_t* sa, uint32_t* d_cnt, uint32_t* d_err,
                         uint32_t* d_left, unsigned warp_grid, unsigned cta_grid) {
    std::vector<std::pair<void*, size_t>> maps;
    uint32_t* g_loc = guarded(loc_act, n, maps);
    const uint32_t* g_next = guarded(loc_next, n, maps);
    uint32_t* g_rank = guarded(rank, n, maps);
    uint32_t* g_sa = guarded(sa, n, maps);
    uint32_t* g_cnt = guarded(cnt, nwin, maps);
    Units u{guarded(beg, nwin, maps), nullptr, nullptr, nullptr, nullptr, guarded(lofs, nwin, maps), g_cnt, nullptr};
    run_grid(warp_grid, kWWarps * 32, [&] {
        sa_round_local_warp_kernel(g_loc, g_next, u, nwin, n, g_rank, g_sa, d_cnt, d_err, d_left);
    });
    run_grid(cta_grid, kLThreads, [&] {
        sa_round_local_kernel(g_loc, g_next, u, nwin, n, g_rank, g_sa, d_cnt, d_err, d_left);
    });
    memcpy(loc_act, g_loc, n * 4ull);
    memcpy(rank, g_rank, n * 4ull);
    memcpy(sa, g_sa, n * 4ull);
    memcpy(cnt, g_cnt, nwin * 4ull);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}

// The unit scan of one block (one CTA): unit ends, long counts, owners,
// global-path offsets, zeroed counts and round counters.  Unit fields are
// laid out as on the device (one stride of words per field).
extern "C" int emu_unit_scan(uint32_t* fields, uint64_t stride, uint32_t nwin, uint32_t n, uint32_t* d_large_n,
                             uint32_t* zero_slots, int nzero, int zero_stride, uint32_t* left_slots, int nleft) {
    std::vector<std::pair<void*, size_t>> maps;
    uint32_t* g = guarded(fields, stride * 8, maps);
    uint32_t* gz = guarded(zero_slots, (size_t)nzero * zero_stride, maps);
    Units u{g, g + stride, g + 2 * stride, g + 3 * stride, g + 4 * stride, g + 5 * stride, g + 6 * stride,
            g + 7 * stride};
    uint32_t* gl = guarded(left_slots, (size_t)nleft, maps);
    run_grid(1, kScanThreads, [&] {
        sa_unit_scan_kernel(u, nwin, n, d_large_n, gz, nzero, zero_stride, gl, nleft);
    });
    memcpy(fields, g, stride * 8 * 4);
    memcpy(zero_slots, gz, (size_t)nzero * zero_stride * 4);
    memcpy(left_slots, gl, (size_t)nleft * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
