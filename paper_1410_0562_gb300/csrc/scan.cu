// scan.cu -- device-wide scans over 32-bit values whose length lives in
// device memory (reduce -> scan of CTA partials -> downsweep).  Used for the
// radix-sort digit offsets, the compaction of unsorted suffix groups and the
// group-head propagation of the suffix sort.
#include "sbwt_internal.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = kScanTile / kThreads;  // 16

__device__ __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> 5); }

template <class Op>
__global__ void __launch_bounds__(kThreads) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                               const uint32_t* __restrict__ d_len,
                                                               uint32_t* __restrict__ partial) {
    const uint32_t len = *d_len;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    if (base >= len) return;
    uint32_t acc = Op::template id<uint32_t>();
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        uint64_t i = base + (uint64_t)q * kThreads + threadIdx.x;
        if (i < len) acc = Op::f(acc, in[i]);
    }
    uint32_t tot;
    cta_exclusive_scan<Op, kThreads>(acc, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class Op>
__global__ void __launch_bounds__(kThreads) scan_partials_kernel(uint32_t* __restrict__ partial,
                                                                 const uint32_t* __restrict__ d_len,
                                                                 uint32_t* __restrict__ d_total) {
    const uint32_t len = *d_len;
    const uint32_t nchunks = (uint32_t)(((uint64_t)len + kScanTile - 1) / kScanTile);
    uint32_t carry = Op::template id<uint32_t>();
    for (uint32_t base = 0; base < nchunks; base += kThreads) {
        uint32_t i = base + threadIdx.x;
        uint32_t v = i < nchunks ? partial[i] : Op::template id<uint32_t>();
        uint32_t tot;
        uint32_t ex = cta_exclusive_scan<Op, kThreads>(v, tot);
        if (i < nchunks) partial[i] = Op::f(carry, ex);
        carry = Op::f(carry, tot);
    }
    if (d_total != nullptr && threadIdx.x == 0) *d_total = carry;
}

template <class Op, bool kInclusive>
__global__ void __launch_bounds__(kThreads) scan_down_kernel(const uint32_t* in, uint32_t* out,
                                                             const uint32_t* __restrict__ d_len,
                                                             const uint32_t* __restrict__ partial) {
    __shared__ uint32_t tile[kScanTile + kScanTile / 32];
    const uint32_t len = *d_len;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    if (base >= len) return;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        uint32_t i = q * kThreads + threadIdx.x;
        tile[pad(i)] = base + i < len ? in[base + i] : Op::template id<uint32_t>();
    }
    __syncthreads();
    uint32_t v[kItems];
    uint32_t acc = Op::template id<uint32_t>();
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        v[q] = tile[pad(threadIdx.x * kItems + q)];
        acc = Op::f(acc, v[q]);
    }
    uint32_t tot;
    uint32_t run = Op::f(partial[blockIdx.x], cta_exclusive_scan<Op, kThreads>(acc, tot));
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        if (kInclusive) {
            run = Op::f(run, v[q]);
            tile[pad(threadIdx.x * kItems + q)] = run;
        } else {
            tile[pad(threadIdx.x * kItems + q)] = run;
            run = Op::f(run, v[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        uint32_t i = q * kThreads + threadIdx.x;
        if (base + i < len) out[base + i] = tile[pad(i)];
    }
}

template <class Op, bool kInclusive>
void scan_impl(Launcher& L, const char* const names[3], const uint32_t* in, uint32_t* out, const uint32_t* d_len,
               uint64_t cap, uint32_t* temp, uint32_t* d_total) {
    unsigned grid = cap ? ceil_div_u(cap, kScanTile) : 1;
    SBWT_LAUNCH(L, names[0], 0, 4, d_len, scan_reduce_kernel<Op>, grid, kThreads, 0, in, d_len, temp);
    SBWT_LAUNCH(L, names[1], 8.0 * grid, 0, nullptr, scan_partials_kernel<Op>, 1, kThreads, 0, temp, d_len,
                d_total);
    SBWT_LAUNCH(L, names[2], 0, 8, d_len, (scan_down_kernel<Op, kInclusive>), grid, kThreads, 0, in, out, d_len,
                temp);
}

}  // namespace

size_t scan_temp_words(uint64_t cap) { return (size_t)(cap / kScanTile) + 2; }

void scan_exclusive_sum(Launcher& L, const uint32_t* in, uint32_t* out, const uint32_t* d_len, uint64_t cap,
                        uint32_t* temp, uint32_t* d_total) {
    static const char* const names[3] = {"scan_reduce", "scan_partials", "scan_downsweep"};
    scan_impl<SumOp, false>(L, names, in, out, d_len, cap, temp, d_total);
}

void scan_inclusive_max(Launcher& L, const uint32_t* in, uint32_t* out, const uint32_t* d_len, uint64_t cap,
                        uint32_t* temp) {
    static const char* const names[3] = {"scan_reduce", "scan_partials", "scan_downsweep"};
    scan_impl<MaxOp, true>(L, names, in, out, d_len, cap, temp, nullptr);
}

}  // namespace sbwt
