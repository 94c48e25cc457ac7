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
#include <algorithm>
#include <atomic>
#include <barrier>
#include <cstdint>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>
#include <sys/mman.h>
#include <unistd.h>

using std::max;
using std::min;

struct Dim { unsigned x = 0, y = 0, z = 0; };
thread_local Dim threadIdx, blockIdx;
static Dim blockDim, gridDim;
thread_local unsigned emu_lane;

struct EmuWarp {
    std::barrier<> bar{32};
    unsigned long long xch[32];
};
thread_local EmuWarp* g_warp;
struct EmuCta {
    std::unique_ptr<std::barrier<>> bar;
    std::vector<int> xch;
};
static EmuCta g_cta;

static inline void __syncwarp(unsigned = 0xffffffffu) { g_warp->bar.arrive_and_wait(); }
template <class T>
static T emu_get(T v, unsigned src) {
    g_warp->xch[emu_lane] = (unsigned long long)v;
    g_warp->bar.arrive_and_wait();
    T r = (T)g_warp->xch[src];
    g_warp->bar.arrive_and_wait();
    return r;
}
static inline unsigned __ballot_sync(unsigned, int pred) {
    g_warp->xch[emu_lane] = pred ? 1 : 0;
    g_warp->bar.arrive_and_wait();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (unsigned)(g_warp->xch[l] & 1) << l;
    g_warp->bar.arrive_and_wait();
    return m;
}
template <class T>
static T __shfl_up_sync(unsigned, T v, int d) { return emu_get(v, emu_lane >= (unsigned)d ? emu_lane - d : emu_lane); }
template <class T>
static T __shfl_sync(unsigned, T v, int src) { return emu_get(v, (unsigned)src); }
static inline unsigned __reduce_max_sync(unsigned, unsigned v) {
    g_warp->xch[emu_lane] = v;
    g_warp->bar.arrive_and_wait();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m = std::max(m, (unsigned)g_warp->xch[l]);
    g_warp->bar.arrive_and_wait();
    return m;
}
static inline void __syncthreads() { g_cta.bar->arrive_and_wait(); }
static inline int __syncthreads_count(int pred) {
    g_cta.xch[threadIdx.x] = pred ? 1 : 0;
    g_cta.bar->arrive_and_wait();
    int c = 0;
    for (int v : g_cta.xch) c += v;
    g_cta.bar->arrive_and_wait();
    return c;
}
static inline int __syncthreads_or(int pred) { return __syncthreads_count(pred) > 0; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline unsigned atomicAdd(uint32_t* p, uint32_t v) { return std::atomic_ref<uint32_t>(*p).fetch_add(v); }
static inline unsigned atomicOr(uint32_t* p, uint32_t v) { return std::atomic_ref<uint32_t>(*p).fetch_or(v); }
static inline unsigned atomicMin(uint32_t* p, uint32_t v) {
    std::atomic_ref<uint32_t> a(*p);
    uint32_t cur = a.load();
    while (v < cur && !a.compare_exchange_weak(cur, v)) {
    }
    return cur;
}

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__ __restrict
#define __launch_bounds__(...)
#define __shared__ static
#define __align__(n) alignas(n)

struct uint4 {
    unsigned x, y, z, w;
};
static inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return uint4{a, b, c, d}; }

#include "constants.inc"
alignas(16) static unsigned char g_dyn_smem[(size_t)kLSlots * 20];  // the larger of the two CTA kernels' needs
#include "scan.inc"
#include "unit_scan.inc"
#include "cta_local.inc"
#include "warp_local.inc"
#include "cta_round.inc"
#include "warp_round.inc"

template <class T>
static T* guarded(const T* src, size_t count, std::vector<std::pair<void*, size_t>>& maps) {
    const size_t pg = (size_t)sysconf(_SC_PAGESIZE);
    const size_t bytes = count * sizeof(T);
    const size_t body = (bytes + pg - 1) / pg * pg;
    const size_t total = body + 2 * pg;
    char* m = (char*)mmap(nullptr, total, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    mprotect(m, pg, PROT_NONE);
    mprotect(m + pg + body, pg, PROT_NONE);
    maps.push_back({m, total});
    T* p = (T*)(m + pg + body - bytes);
    if (bytes) memcpy(p, src, bytes);
    return p;
}

template <class F>
static void run_grid(unsigned grid, unsigned threads, F body) {
    gridDim.x = grid;
    blockDim.x = threads;
    for (unsigned b = 0; b < grid; ++b) {
        g_cta.bar = std::make_unique<std::barrier<>>(threads);
        g_cta.xch.assign(threads, 0);
        std::vector<EmuWarp> warps(threads / 32);
        std::vector<std::thread> th;
        for (unsigned i = 0; i < threads; ++i)
            th.emplace_back([&, b, i] {
                blockIdx.x = b;
                threadIdx.x = i;
                emu_lane = i & 31;
                g_warp = &warps[i >> 5];
                body();
            });
        for (auto& t : th) t.join();
    }
}

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

// One unit-local round: the warp kernel, then the CTA kernel.
extern "C" int emu_round(uint32_t* loc_act, const uint32_t* loc_next, uint32_t* beg, uint32_t* lofs, uint32_t* cnt,
                         uint32_t nwin, uint32_t n, uint32_t* rank, uint32_t* sa, uint32_t* d_cnt, uint32_t* d_err,
                         unsigned warp_grid, unsigned cta_grid) {
    std::vector<std::pair<void*, size_t>> maps;
    uint32_t* g_loc = guarded(loc_act, n, maps);
    const uint32_t* g_next = guarded(loc_next, n, maps);
    uint32_t* g_rank = guarded(rank, n, maps);
    uint32_t* g_sa = guarded(sa, n, maps);
    uint32_t* g_cnt = guarded(cnt, nwin, maps);
    Units u{guarded(beg, nwin, maps), nullptr, nullptr, nullptr, nullptr, guarded(lofs, nwin, maps), g_cnt, nullptr};
    run_grid(warp_grid, kWWarps * 32, [&] {
        sa_round_local_warp_kernel(g_loc, g_next, u, nwin, n, g_rank, g_sa, d_cnt, d_err);
    });
    run_grid(cta_grid, kLThreads, [&] {
        sa_round_local_kernel(g_loc, g_next, u, nwin, n, g_rank, g_sa, d_cnt, d_err);
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
                             uint32_t* zero_slots, int nzero, int zero_stride) {
    std::vector<std::pair<void*, size_t>> maps;
    uint32_t* g = guarded(fields, stride * 8, maps);
    uint32_t* gz = guarded(zero_slots, (size_t)nzero * zero_stride, maps);
    Units u{g, g + stride, g + 2 * stride, g + 3 * stride, g + 4 * stride, g + 5 * stride, g + 6 * stride,
            g + 7 * stride};
    run_grid(1, kScanThreads, [&] { sa_unit_scan_kernel(u, nwin, n, d_large_n, gz, nzero, zero_stride); });
    memcpy(fields, g, stride * 8 * 4);
    memcpy(zero_slots, gz, (size_t)nzero * zero_stride * 4);
    for (auto& m : maps) munmap(m.first, m.second);
    return 0;
}
