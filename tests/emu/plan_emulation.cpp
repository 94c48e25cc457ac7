// Host emulation of the append planning (plan.cu), for CPU tests: the check
// of an append's offsets (and its longest read) and the greedy block table
// of Algorithm 1.
//
// The kernel text is compiled here unchanged (the test cuts it out of the
// CUDA sources into the .inc files below) on the emulation in cuda_emu.h:
// one std::thread per GPU thread, CTA barriers emulated, every array
// between inaccessible pages.
#include "cuda_emu.h"

#include "plan_types.inc"
#include "plan.inc"

// plan_check with the library's grid, then plan_blocks (one thread).  The
// table holds `cap` entries; summary = (bad, blocks, max_len, npos).
extern "C" int emu_plan(const uint64_t* offsets, uint64_t m, uint64_t M, uint64_t max_block, PlanBlock* table,
                        unsigned cap, PlanSummary* summary) {
    std::vector<std::pair<void*, size_t>> maps;
    const unsigned long long* g_off =
        guarded(reinterpret_cast<const unsigned long long*>(offsets), (size_t)m + 1, maps);
    PlanBlock* g_table = guarded(table, cap ? cap : 1, maps);
    PlanSummary zero{};
    PlanSummary* g_sum = guarded(&zero, 1, maps);
    const unsigned grid = (unsigned)std::min<uint64_t>(1024, (m + kThreads - 1) / kThreads + 1);
    run_grid(grid, kThreads, [&] { plan_check_kernel(g_off, m, max_block, g_sum); });
    run_grid(1, 1, [&] { plan_blocks_kernel(g_off, m, M, g_table, cap, g_sum); });
    memcpy(table, g_table, (size_t)cap * sizeof(PlanBlock));
    *summary = *g_sum;
    for (auto& mp : maps) munmap(mp.first, mp.second);
    return 0;
}
