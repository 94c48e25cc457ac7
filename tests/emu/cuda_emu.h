// cuda_emu.h -- host emulation of the CUDA features the CPU tests of the
// kernels need: one std::thread per GPU thread of a CTA, warp intrinsics as
// exchanges through a per-warp barrier, __syncthreads through a CTA barrier,
// shared variables as statics (CTAs run one after another), and device
// arrays copied between inaccessible pages so an access outside one faults.
// A lane that skips an intrinsic its warp executes hangs the emulation (the
// test's timeout); every warp intrinsic here expects all 32 lanes to call it,
// each with its own mask.
#pragma once
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

#include <type_traits>

template <class A, class B>
static inline std::common_type_t<A, B> min(A a, B b) { return a < b ? (std::common_type_t<A, B>)a : (std::common_type_t<A, B>)b; }
template <class A, class B>
static inline std::common_type_t<A, B> max(A a, B b) { return a < b ? (std::common_type_t<A, B>)b : (std::common_type_t<A, B>)a; }

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
template <class T>
static T __shfl_xor_sync(unsigned, T v, int m) { return emu_get(v, emu_lane ^ (unsigned)m); }
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
static inline int __syncthreads_and(int pred) { return __syncthreads_count(pred) == (int)blockDim.x; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline unsigned atomicAdd(uint32_t* p, uint32_t v) { return std::atomic_ref<uint32_t>(*p).fetch_add(v); }
static inline unsigned atomicOr(uint32_t* p, uint32_t v) { return std::atomic_ref<uint32_t>(*p).fetch_or(v); }
static inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
    std::atomic_ref<unsigned long long> r(*p);
    unsigned long long cur = r.load();
    while (cur < v && !r.compare_exchange_weak(cur, v)) {
    }
    return cur;
}
static inline unsigned atomicMin(uint32_t* p, uint32_t v) {
    std::atomic_ref<uint32_t> a(*p);
    uint32_t cur = a.load();
    while (v < cur && !a.compare_exchange_weak(cur, v)) {
    }
    return cur;
}

template <class T>
static unsigned __match_any_sync(unsigned, T v) {
    g_warp->xch[emu_lane] = (unsigned long long)v;
    g_warp->bar.arrive_and_wait();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (g_warp->xch[l] == (unsigned long long)v ? 1u : 0u) << l;
    g_warp->bar.arrive_and_wait();
    return m;
}
static inline unsigned __reduce_or_sync(unsigned mask, unsigned v) {
    g_warp->xch[emu_lane] = v;
    g_warp->bar.arrive_and_wait();
    unsigned r = 0;
    for (int l = 0; l < 32; ++l)
        if ((mask >> l) & 1u) r |= (unsigned)g_warp->xch[l];
    g_warp->bar.arrive_and_wait();
    return r;
}
static inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
template <class T>
static inline T __ldg(const T* p) { return *p; }
static inline int __ffsll(long long x) { return __builtin_ffsll(x); }
struct ulonglong2 {
    unsigned long long x, y;
};
static inline ulonglong2 make_ulonglong2(unsigned long long a, unsigned long long b) { return ulonglong2{a, b}; }

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
struct uint2 {
    unsigned x, y;
};
static inline uint2 make_uint2(unsigned a, unsigned b) { return uint2{a, b}; }
static inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return uint4{a, b, c, d}; }

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
        std::vector<EmuWarp> warps((threads + 31) / 32);  // a one-thread grid still gets its (unused) warp
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

