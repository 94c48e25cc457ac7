// radix.cu -- stable LSD radix sort of (64-bit key, 32-bit value) pairs,
// 8-bit digits, element count in device memory.  This is the sort under the
// suffix sorting of a block (Section 3 of arXiv 1410.0562 sorts suffixes as
// long integer keys of packed symbols, refined over iterations).
//
// The digit histograms of every pass come from one read of the keys (or
// from the kernel that wrote them); each digit pass is then one persistent
// kernel (the single-pass "onesweep" scheme of Adinets and Merrill): a CTA
// takes the next tile in order, ranks its keys per digit (8 warp ballots give
// each lane the mask of lanes with the same digit), publishes its per-digit
// counts, finds the counts of all earlier tiles by decoupled look-back,
// stages the tile in shared memory in digit order and writes it out in
// coalesced runs.
#include <algorithm>
#include <atomic>

#include "sbwt_internal.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = kRadixTile / kThreads;      // 16 keys per thread
constexpr int kWarpItems = kRadixTile / kWarps;    // 512 consecutive keys per warp
constexpr int kBins = kRadixBins;
static_assert(kBins == kThreads, "one thread per digit");

constexpr size_t kScatterSmem = (size_t)kRadixTile * 8 + (size_t)kRadixTile * 4 + (size_t)kWarps * kBins * 4 +
                                (size_t)kBins * 4 * 3 + 16;

// Temp layout (32-bit words): [0, 8) tile counters of the passes, [8, 8 +
// 8*256) digit histograms / starts of every pass, then the look-back words.
constexpr size_t kCounters = 0;
constexpr size_t kDigitStart = 8;
constexpr size_t kLookback = kDigitStart + (size_t)kRadixMaxPasses * kBins + 8;

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const unsigned long long* __restrict__ keys,
                                                              const uint32_t* __restrict__ d_n, int begin_bit,
                                                              int passes, uint32_t* __restrict__ ghist) {
    __shared__ uint32_t h[kRadixMaxPasses * kBins];
    for (int i = threadIdx.x; i < passes * kBins; i += kThreads) h[i] = 0;
    __syncthreads();
    const uint32_t n = *d_n;
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kThreads)
        radix_hist_add(h, keys[i], begin_bit, passes);
    __syncthreads();
    radix_hist_flush<kThreads>(h, ghist, passes);
}

// Exclusive scan of each pass's histogram into digit start offsets.
__global__ void __launch_bounds__(kThreads) radix_digit_scan_kernel(uint32_t* __restrict__ ghist, int passes) {
    for (int p = 0; p < passes; ++p) {
        uint32_t tot;
        const uint32_t ex = cta_exclusive_scan<SumOp, kThreads>(ghist[p * kBins + threadIdx.x], tot);
        ghist[p * kBins + threadIdx.x] = ex;
    }
}

__global__ void __launch_bounds__(kThreads, 2) radix_onesweep_kernel(
    const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin, unsigned long long* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ d_n, int shift, const uint32_t* __restrict__ dstart_g,
    unsigned long long* __restrict__ lookback, uint32_t* __restrict__ tile_counter, unsigned long long epoch,
    uint32_t* __restrict__ d_err) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* skeys = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* svals = reinterpret_cast<uint32_t*>(skeys + kRadixTile);
    uint32_t* wcnt = svals + kRadixTile;       // [kWarps][kBins]
    uint32_t* dstart = wcnt + kWarps * kBins;  // tile-local start of each digit
    uint32_t* gstart = dstart + kBins;         // global start of each digit for this tile
    uint32_t* misc = gstart + kBins;

    const uint32_t n = *d_n;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kRadixTile - 1) / kRadixTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int d = threadIdx.x;  // the digit this thread publishes and looks back for
    const unsigned long long tag = lb_tag(epoch);

    for (;;) {
        if (threadIdx.x == 0) misc[0] = atomicAdd(tile_counter, 1u);
        for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) wcnt[i] = 0;
        __syncthreads();
        const uint32_t tile = misc[0];
        if (tile >= ntiles) break;
        const uint64_t base = (uint64_t)tile * kRadixTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kRadixTile, (uint64_t)n - base);

        unsigned long long k[kItems];
        uint32_t v[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t i = warp * kWarpItems + it * 32 + lane;
            const bool valid = i < cnt;
            k[it] = valid ? kin[base + i] : 0ull;
            v[it] = valid ? vin[base + i] : 0u;
        }

        // rank among equal digits of the warp, in index order
        uint32_t* my = wcnt + warp * kBins;
        uint32_t dr[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t i = warp * kWarpItems + it * 32 + lane;
            const bool valid = i < cnt;
            const uint32_t dg = (uint32_t)(k[it] >> shift) & (kBins - 1);
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
#pragma unroll
            for (int b = 0; b < kRadixBits; ++b) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
                peers &= ((dg >> b) & 1u) ? bal : ~bal;
            }
            const uint32_t prior = valid ? my[dg] : 0u;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) my[dg] = prior + __popc(peers);
            __syncwarp();
            dr[it] = valid ? ((dg << 16) | (prior + __popc(peers & lt))) : 0xFFFFFFFFu;
        }
        __syncthreads();

        // tile counts per digit; exclusive offsets across warps
        uint32_t cnt_d = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcnt[w * kBins + d];
            wcnt[w * kBins + d] = cnt_d;
            cnt_d += t;
        }
        // publish this tile's count, then look back for the earlier tiles'
        unsigned long long* lb = lookback + (uint64_t)tile * kBins + d;
        uint32_t excl = 0;
        if (tile == 0) {
            lb_store(lb, tag | kLbPrefix | cnt_d);
        } else {
            lb_store(lb, tag | kLbAggregate | cnt_d);
            excl = lb_lookback<SumOp>(lookback + d, kBins, tile, tag, d_err, 64u);
            lb_store(lb, tag | kLbPrefix | (excl + cnt_d));
        }
        uint32_t tile_total;
        dstart[d] = cta_exclusive_scan<SumOp, kThreads>(cnt_d, tile_total);
        gstart[d] = dstart_g[d] + excl;
        __syncthreads();

#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            if (dr[it] == 0xFFFFFFFFu) continue;
            const uint32_t dd = dr[it] >> 16;
            const uint32_t pos = dstart[dd] + wcnt[warp * kBins + dd] + (dr[it] & 0xFFFFu);
            if (pos < kRadixTile) {
                skeys[pos] = k[it];
                svals[pos] = v[it];
            } else {
                atomicOr(d_err, 16u);
            }
        }
        __syncthreads();

        for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
            const unsigned long long key = skeys[s];
            const uint32_t dd = (uint32_t)(key >> shift) & (kBins - 1);
            const uint64_t o = (uint64_t)gstart[dd] + (s - dstart[dd]);
            if (o < n) {
                kout[o] = key;
                vout[o] = svals[s];
            } else {
                atomicOr(d_err, 16u);
            }
        }
        __syncthreads();
    }
}

std::atomic<unsigned long long> g_epoch{0};
unsigned g_onesweep_ctas[64] = {0};
unsigned g_hist_ctas[64] = {0};

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

}  // namespace

unsigned long long lb_next_epoch() {
    unsigned long long e;
    do {
        e = (++g_epoch) & 0x3FFFFFFFull;
    } while (e == 0);
    return e;
}

unsigned persistent_ctas(const void* kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    cudaGetLastError();
    return (unsigned)(std::max(1, sms) * std::max(1, per_sm));
}

size_t radix_temp_words(uint64_t cap) {
    const uint64_t tiles = cap / kRadixTile + 1;
    return kLookback + 2 * (size_t)tiles * kBins + 64;
}

void radix_init() {
    cudaFuncSetAttribute(radix_onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    const int dev = current_device();
    g_onesweep_ctas[dev] = persistent_ctas((const void*)radix_onesweep_kernel, kThreads, kScatterSmem);
    g_hist_ctas[dev] = persistent_ctas((const void*)radix_hist_kernel, kThreads, 0);
}

uint32_t* radix_histograms(uint32_t* temp) { return temp + kDigitStart; }

void radix_hist_clear(Launcher& L, uint32_t* temp) {
    cudaMemsetAsync(temp, 0, (kDigitStart + (size_t)kRadixMaxPasses * kBins) * 4, L.stream);
}

bool radix_sort_pairs(Launcher& L, unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                      uint32_t* vals_alt, const uint32_t* d_n, uint64_t cap, int begin_bit, int end_bit,
                      uint32_t* temp, uint32_t* d_err, bool hist_ready) {
    const int passes = radix_passes(begin_bit, end_bit);
    if (passes <= 0) return false;
    uint32_t* counters = temp + kCounters;
    uint32_t* ghist = temp + kDigitStart;
    unsigned long long* lookback = reinterpret_cast<unsigned long long*>(temp + kLookback);
    const int dev = current_device();
    const uint64_t tiles = cap / kRadixTile + 1;
    const unsigned grid = (unsigned)std::min<uint64_t>(std::max(1u, g_onesweep_ctas[dev]), tiles);
    if (!hist_ready) {
        radix_hist_clear(L, temp);
        const unsigned hgrid = (unsigned)std::min<uint64_t>(std::max(1u, g_hist_ctas[dev]), cap / kThreads + 1);
        SBWT_LAUNCH(L, "radix_histogram", 0, 8, d_n, radix_hist_kernel, hgrid, kThreads, 0, keys, d_n, begin_bit,
                    passes, ghist);
    }
    SBWT_LAUNCH(L, "radix_digit_scan", 8.0 * kBins * passes, 0, nullptr, radix_digit_scan_kernel, 1, kThreads, 0,
                ghist, passes);
    bool alt = false;
    for (int p = 0; p < passes; ++p) {
        const unsigned long long* kin = alt ? keys_alt : keys;
        const uint32_t* vin = alt ? vals_alt : vals;
        unsigned long long* ko = alt ? keys : keys_alt;
        uint32_t* vo = alt ? vals : vals_alt;
        SBWT_LAUNCH(L, "radix_onesweep", 0, 24, d_n, radix_onesweep_kernel, grid, kThreads, kScatterSmem, kin, vin,
                    ko, vo, d_n, begin_bit + kRadixBits * p, ghist + p * kBins, lookback, counters + p,
                    lb_next_epoch(), d_err);
        alt = !alt;
    }
    return alt;
}

}  // namespace sbwt
