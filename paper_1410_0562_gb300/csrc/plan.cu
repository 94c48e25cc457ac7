// plan.cu -- checks an append's device-resident offsets and plans its
// blocks on the device, so that only a small block table crosses to the host.
//
// Blocks follow Algorithm 1 of arXiv 1410.0562 (blocks of roughly M
// suffixes): greedily, whole reads while the block holds at most M suffixes;
// a read longer than M is a block alone.  Read j's first suffix sits at
// text position rpos(j) = offsets[j] + j, so the reads [j, j') hold
// rpos(j') - rpos(j) suffixes and the greedy end of the block that starts at
// j is the largest j' with rpos(j') - rpos(j) <= M (at least j + 1).
#include <algorithm>

#include "sbwt_kernels.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;

// Offsets must start at 0 and never decrease; every read must fit a block of
// 2^31 suffixes.  Also the longest read.
__global__ void __launch_bounds__(kThreads) plan_check_kernel(const unsigned long long* __restrict__ off,
                                                              unsigned long long m,
                                                              unsigned long long max_block,
                                                              PlanSummary* __restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && off[0] != 0) atomicOr(&out->bad, 1u);
    unsigned long long local_max = 0;
    bool bad = false;
    for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < m; j += (uint64_t)gridDim.x * kThreads) {
        const unsigned long long a = off[j], b = off[j + 1];
        if (b < a || b - a + 1 > max_block) bad = true;
        else local_max = max(local_max, b - a);
    }
    // one atomic per CTA, not per thread
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&out->bad, 1u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    __shared__ unsigned long long warp_max[kThreads / 32];
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = local_max;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long mx = 0;
        for (int w = 0; w < kThreads / 32; ++w) mx = max(mx, warp_max[w]);
        if (mx) atomicMax(&out->max_len, mx);
    }
}

__device__ __forceinline__ unsigned long long rpos(const unsigned long long* off, unsigned long long j) {
    return off[j] + j;
}

// One thread walks the greedy partition with a binary search per block.
__global__ void plan_blocks_kernel(const unsigned long long* __restrict__ off, unsigned long long m,
                                   unsigned long long M, PlanBlock* __restrict__ table, unsigned cap,
                                   PlanSummary* __restrict__ out) {
    if (out->bad) return;
    unsigned long long j = 0;
    unsigned k = 0;
    while (j < m) {
        const unsigned long long start = rpos(off, j);
        unsigned long long lo = j + 1, hi = m;  // largest j' in [j+1, m] with rpos(j') - start <= M
        if (rpos(off, lo) - start <= M) {
            while (lo < hi) {
                const unsigned long long mid = hi - (hi - lo) / 2;
                if (rpos(off, mid) - start <= M) lo = mid; else hi = mid - 1;
            }
        }
        if (k < cap) {
            table[k].j0 = j;
            table[k].j1 = lo;
            table[k].base = start;
            table[k].n_int = rpos(off, lo) - start;
        }
        ++k;
        j = lo;
    }
    out->blocks = k;
    out->npos = rpos(off, m);
}

}  // namespace

void launch_plan(Launcher& L, const uint64_t* d_offsets, uint64_t m, uint64_t M, uint64_t max_block,
                 PlanBlock* table, unsigned cap, PlanSummary* summary) {
    cudaMemsetAsync(summary, 0, sizeof(PlanSummary), L.stream);
    const auto* off = reinterpret_cast<const unsigned long long*>(d_offsets);
    const unsigned grid = (unsigned)std::min<uint64_t>(1024, (m + kThreads - 1) / kThreads + 1);
    SBWT_LAUNCH(L, "plan_check", 8.0 * (m + 1), 0, nullptr, plan_check_kernel, grid, kThreads, 0, off,
                (unsigned long long)m, (unsigned long long)max_block, summary);
    SBWT_LAUNCH(L, "plan_blocks", 0, 0, nullptr, plan_blocks_kernel, 1, 1, 0, off, (unsigned long long)m,
                (unsigned long long)M, table, cap, summary);
}

}  // namespace sbwt
