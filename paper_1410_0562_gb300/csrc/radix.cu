// radix.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs,
// 8-bit digits, element count in device memory.  Each digit pass is an
// upsweep (per-tile digit histograms), a device-wide scan of the
// digit-major histogram matrix, and a downsweep that ranks every key inside
// its tile with warp match/ballot, stages the tile in shared memory in digit
// order and writes it out in coalesced runs.  This is the sort under the
// suffix sorting of a block (Section 3 of arXiv 1410.0562 sorts suffixes by
// long integer keys of packed symbols, refined over iterations).
#include "sbwt_internal.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = kRadixTile / kThreads;      // 16 keys per thread
constexpr int kWarpItems = kRadixTile / kWarps;    // 512 consecutive keys per warp
constexpr int kBins = 1 << kRadixBits;             // 256
static_assert(kBins == kThreads, "one thread per digit in the downsweep");

constexpr size_t kScatterSmem = (size_t)kRadixTile * 8 + (size_t)kRadixTile * 4 + (size_t)kWarps * kBins * 4 +
                                (size_t)kBins * 4 * 2;

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const unsigned long long* __restrict__ keys,
                                                              const uint32_t* __restrict__ d_n, int shift,
                                                              uint32_t* __restrict__ hist,
                                                              uint32_t* __restrict__ d_hist_len) {
    __shared__ uint32_t h[kWarps * kBins];
    const uint32_t n = *d_n;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kRadixTile - 1) / kRadixTile);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_hist_len = ntiles * kBins;
    const uint32_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) h[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)tile * kRadixTile;
    const uint32_t cnt = (uint32_t)min((uint64_t)kRadixTile, (uint64_t)n - base);
#pragma unroll 4
    for (int q = 0; q < kItems; ++q) {
        uint32_t i = q * kThreads + threadIdx.x;
        if (i < cnt) {
            uint32_t d = (uint32_t)(keys[base + i] >> shift) & (kBins - 1);
            atomicAdd(&h[warp * kBins + d], 1u);
        }
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += h[w * kBins + d];
    hist[(uint64_t)d * ntiles + tile] = s;
}

__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(const unsigned long long* __restrict__ kin,
                                                                 const uint32_t* __restrict__ vin,
                                                                 unsigned long long* __restrict__ kout,
                                                                 uint32_t* __restrict__ vout,
                                                                 const uint32_t* __restrict__ d_n, int shift,
                                                                 const uint32_t* __restrict__ hist,
                                                                 uint32_t* __restrict__ d_err) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* skeys = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* svals = reinterpret_cast<uint32_t*>(skeys + kRadixTile);
    uint32_t* wcnt = svals + kRadixTile;     // [kWarps][kBins]
    uint32_t* dstart = wcnt + kWarps * kBins;  // tile-local start of each digit
    uint32_t* gstart = dstart + kBins;         // global start of each digit for this tile

    const uint32_t n = *d_n;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kRadixTile - 1) / kRadixTile);
    const uint32_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    const uint64_t base = (uint64_t)tile * kRadixTile;
    const uint32_t cnt = (uint32_t)min((uint64_t)kRadixTile, (uint64_t)n - base);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) wcnt[i] = 0;

    unsigned long long k[kItems];
    uint32_t v[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        uint32_t i = warp * kWarpItems + it * 32 + lane;
        bool valid = i < cnt;
        k[it] = valid ? kin[base + i] : 0ull;
        v[it] = valid ? vin[base + i] : 0u;
    }
    __syncthreads();

    // Rank each key among the equal digits of its warp, in index order.
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t dr[kItems];
    uint32_t* my = wcnt + warp * kBins;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        uint32_t i = warp * kWarpItems + it * 32 + lane;
        uint32_t d = i < cnt ? (uint32_t)(k[it] >> shift) & (kBins - 1) : (uint32_t)kBins;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t prior = d < kBins ? my[d] : 0u;
        __syncwarp();
        if (d < kBins && lane == __ffs(peers) - 1) my[d] = prior + __popc(peers);
        __syncwarp();
        dr[it] = (d << 16) | (prior + __popc(peers & lt));
    }
    __syncthreads();

    // Per digit: exclusive offsets across warps, then across digits.
    const int d = threadIdx.x;
    uint32_t tot_d = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t t = wcnt[w * kBins + d];
        wcnt[w * kBins + d] = tot_d;
        tot_d += t;
    }
    uint32_t tile_total;
    uint32_t start = cta_exclusive_scan<SumOp, kThreads>(tot_d, tile_total);
    dstart[d] = start;
    gstart[d] = hist[(uint64_t)d * ntiles + tile];
    __syncthreads();

#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        uint32_t dd = dr[it] >> 16;
        if (dd < kBins) {
            uint32_t pos = dstart[dd] + wcnt[warp * kBins + dd] + (dr[it] & 0xFFFFu);
            if (pos < kRadixTile) {
                skeys[pos] = k[it];
                svals[pos] = v[it];
            } else {
                atomicOr(d_err, 16u);
            }
        }
    }
    __syncthreads();

    for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
        unsigned long long key = skeys[s];
        uint32_t dd = (uint32_t)(key >> shift) & (kBins - 1);
        uint64_t o = (uint64_t)gstart[dd] + (s - dstart[dd]);
        if (o < n) {
            kout[o] = key;
            vout[o] = svals[s];
        } else {
            atomicOr(d_err, 16u);
        }
    }
}

}  // namespace

size_t radix_temp_words(uint64_t cap) {
    uint64_t tiles = cap / kRadixTile + 1;
    return 64 + (size_t)(tiles * kBins) + scan_temp_words(tiles * kBins) + 64;
}

void radix_init() {
    cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
}

bool radix_sort_pairs(Launcher& L, unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                      uint32_t* vals_alt, const uint32_t* d_n, uint64_t cap, int begin_bit, int end_bit,
                      uint32_t* temp, uint32_t* d_err) {
    const uint64_t max_tiles = cap / kRadixTile + 1;
    uint32_t* d_hist_len = temp;
    uint32_t* hist = temp + 64;
    uint32_t* stemp = hist + max_tiles * kBins;
    const unsigned grid = (unsigned)(cap ? ceil_div_u(cap, kRadixTile) : 1);
    bool alt = false;
    for (int shift = begin_bit; shift < end_bit; shift += kRadixBits) {
        unsigned long long* kin = alt ? keys_alt : keys;
        uint32_t* vin = alt ? vals_alt : vals;
        unsigned long long* ko = alt ? keys : keys_alt;
        uint32_t* vo = alt ? vals : vals_alt;
        SBWT_LAUNCH(L, "radix_upsweep", 0, 8, d_n, radix_hist_kernel, grid, kThreads, 0, kin, d_n, shift, hist,
                    d_hist_len);
        scan_exclusive_sum(L, hist, hist, d_hist_len, max_tiles * kBins, stemp, nullptr);
        SBWT_LAUNCH(L, "radix_downsweep", 0, 24, d_n, radix_scatter_kernel, grid, kThreads, kScatterSmem, kin,
                    vin, ko, vo, d_n, shift, hist, d_err);
        alt = !alt;
    }
    return alt;
}

}  // namespace sbwt
