// radix.cu -- stable LSD radix sort of 64-bit keys, alone or with 32-bit
// values, 8-bit digits, element count in device memory.  This is the sort
// under the suffix sorting of a block (Section 3 of arXiv 1410.0562 sorts
// suffixes as long integer keys of packed symbols, refined over iterations).
//
// Each digit pass is reduce-then-scan over chunks: a persistent grid of G
// CTAs splits the keys into G contiguous chunks of whole tiles; the upsweep
// counts the digits of every chunk, one CTA turns the G x 256 counts into the
// output offset of every (chunk, digit), and the downsweep walks each chunk
// tile by tile with running offsets.  Nothing waits on another CTA.  Inside
// a tile, each warp ranks its keys stably: every lane sets its bit in a
// shared-memory mask word of its digit, so the word it reads back holds the
// lanes with the same digit; the tile is staged in shared memory in digit
// order and written out in runs.  A sort of keys alone moves one 8-byte
// element per key: its runs are twice as long in bytes as those of separate
// key and value arrays, which is what the scatter's speed depends on.
#include <algorithm>

#include "sbwt_internal.cuh"

namespace sbwt {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                           // keys per thread per tile
constexpr int kTile = kThreads * kItems;            // 2048 keys per tile
static_assert(kTile == (int)kRadixTile, "one tile size for the sort and the kernels that count for it");
constexpr int kWarpItems = kTile / kWarps;          // 256 consecutive keys per warp
constexpr int kBins = kRadixBins;
constexpr int kMaxChunks = 2048;
static_assert(kBins == kThreads, "one thread per digit");

// shared memory of the downsweep: TMA input tile (keys, then values when
// kPairs), the staged output tile (same layout), warp digit counters and
// peer masks, three digit tables, the mbarrier
template <class KeyT, bool kPairs>
__host__ __device__ constexpr size_t down_smem() {
    return 2 * (size_t)kTile * (sizeof(KeyT) + (kPairs ? 4 : 0)) + 2 * (size_t)kWarps * kBins * 4 +
           (size_t)kBins * 4 * 3 + 16;
}
static_assert(3 * (down_smem<unsigned long long, true>() + 1024) <= 228 * 1024, "three CTAs per SM");

// Temp layout (32-bit words): two arrays of digit totals (pass p adds into
// array p & 1; the chunk scan of pass p clears the other one for pass p + 1),
// the fused sort's grid barrier and per-group partial counts, then the chunk
// x digit offsets.
constexpr size_t kTotals = 0;
constexpr size_t kGridBar = 2 * kBins;  // grid barrier of the fused sort: arrivals, generation
constexpr int kFusedGroups = 8;         // chunk groups of the fused sort's offset scan
constexpr size_t kPartials = kGridBar + 8;
constexpr size_t kChunkOffsets = kPartials + (size_t)kFusedGroups * kBins;
constexpr uint32_t kGridSpinLimit = 1u << 22;

// Chunk c of a grid of `grid` CTAs: tiles [t0, t1) (radix_chunk_tiles).
// Only the first ceil(ntiles / per) chunks hold tiles.
__device__ __forceinline__ uint32_t tiles_per_chunk(uint32_t n, uint32_t grid, uint32_t& ntiles) {
    ntiles = (uint32_t)(((uint64_t)n + kTile - 1) / kTile);
    return (ntiles + grid - 1) / grid;
}
__device__ __forceinline__ void chunk_range(uint32_t n, uint32_t& t0, uint32_t& t1) {
    radix_chunk_tiles(n, gridDim.x, blockIdx.x, t0, t1);
}

// Two keys from L2 (not through L1: in the fused sort other CTAs wrote them
// earlier in the same launch).
__device__ __forceinline__ void ld_cg_pair(const unsigned long long* p, unsigned long long& a,
                                           unsigned long long& b) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}

// Digit counts of this CTA's chunk (per-warp sub-histograms in shared
// memory h, kWarps x kBins words), also added to the digit totals of the
// whole pass.  A chunk without tiles writes nothing: the scans skip it.
// Whole tiles are read as 16-byte pairs, a tile's loads all issued before
// its counts (the key arrays start on a 16-byte boundary).
template <class KeyT>
__device__ __forceinline__ void up_phase(const KeyT* __restrict__ keys, uint32_t n, int shift,
                                         uint32_t* __restrict__ chunk_counts, uint32_t* __restrict__ totals,
                                         uint32_t* h) {
    static_assert(sizeof(KeyT) == 8, "pairs of 64-bit keys");
    uint32_t t0, t1;
    chunk_range(n, t0, t1);
    if (t0 >= t1) return;
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) h[i] = 0;
    __syncthreads();
    const uint64_t i_end = min((uint64_t)n, (uint64_t)t1 * kTile);
    const uint64_t whole_end = (uint64_t)t0 * kTile + (i_end - (uint64_t)t0 * kTile) / kTile * kTile;
    uint32_t* my = h + (threadIdx.x >> 5) * kBins;
    for (uint64_t b = (uint64_t)t0 * kTile; b < whole_end; b += kTile) {
        unsigned long long v[kItems];
#pragma unroll
        for (int j = 0; j < kItems / 2; ++j)
            ld_cg_pair(reinterpret_cast<const unsigned long long*>(keys) + b + 2 * (j * kThreads + threadIdx.x),
                       v[2 * j], v[2 * j + 1]);
#pragma unroll
        for (int j = 0; j < kItems; ++j) atomicAdd(&my[(uint32_t)(v[j] >> shift) & (kBins - 1)], 1u);
    }
    for (uint64_t i = whole_end + threadIdx.x; i < i_end; i += kThreads)
        atomicAdd(&my[(uint32_t)(keys[i] >> shift) & (kBins - 1)], 1u);
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += h[w * kBins + threadIdx.x];
    chunk_counts[(uint64_t)blockIdx.x * kBins + threadIdx.x] = s;
    if (s) atomicAdd(&totals[threadIdx.x], s);
}

template <class KeyT>
__global__ void __launch_bounds__(kThreads) radix_upsweep_kernel(const KeyT* __restrict__ keys,
                                                                 const uint32_t* __restrict__ d_n, int shift,
                                                                 uint32_t* __restrict__ chunk_counts,
                                                                 uint32_t* __restrict__ totals) {
    __shared__ uint32_t h[kWarps * kBins];
    up_phase(keys, *d_n, shift, chunk_counts, totals, h);
}

// Output offset of every (chunk, digit): the digit's start in the sorted
// output (exclusive scan of the totals) plus the same digit's count in all
// earlier chunks.  One warp per digit (kBins / kScanWarps CTAs): 32 chunks
// at a time, four such loads in flight, each scanned across the warp.
constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kScanBatch = 4;

__global__ void __launch_bounds__(kScanThreads) radix_chunk_scan_kernel(uint32_t* __restrict__ chunk_counts,
                                                                        int grid, const uint32_t* __restrict__ totals,
                                                                        uint32_t* __restrict__ next_totals,
                                                                        const uint32_t* __restrict__ d_n) {
    const int lane = threadIdx.x & 31;
    const uint32_t d = blockIdx.x * kScanWarps + (threadIdx.x >> 5);
    uint32_t ntiles;
    const uint32_t tpc = tiles_per_chunk(*d_n, (uint32_t)grid, ntiles);
    const uint32_t nchunks = tpc ? (ntiles + tpc - 1) / tpc : 0;  // chunks that hold tiles
    if (blockIdx.x == 0 && threadIdx.x < kBins) next_totals[threadIdx.x] = 0;
    uint32_t run = 0;
    for (uint32_t e = lane; e < d; e += 32) run += totals[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
    for (uint32_t cb = 0; cb < nchunks; cb += 32 * kScanBatch) {
        uint32_t v[kScanBatch];
#pragma unroll
        for (int j = 0; j < kScanBatch; ++j) {
            const uint32_t c = cb + j * 32 + lane;
            v[j] = c < nchunks ? chunk_counts[(uint64_t)c * kBins + d] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kScanBatch; ++j) {
            const uint32_t c = cb + j * 32 + lane;
            uint32_t x = v[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (c < nchunks) chunk_counts[(uint64_t)c * kBins + d] = run + x - v[j];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// The scatter of one pass over this CTA's chunk: whole tiles arrive by TMA
// one tile ahead (a partial tile, only the very last one, is read with plain
// loads); each tile is ranked, staged in digit order in shared memory and
// written out in runs.  Without kPairs there are no values (vin, vout
// unused).  smem: down_smem<KeyT, kPairs>() bytes, its mbarrier already
// initialised; parity is the mbarrier's phase, carried across calls.
// Returns false when a copy did not land (flagged in *d_err, bit 8).
template <class KeyT, bool kPairs>
__device__ __forceinline__ bool down_phase(const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
                                           KeyT* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
                                           int shift, const uint32_t* __restrict__ chunk_offsets,
                                           uint32_t* __restrict__ d_err, unsigned char* smem, uint32_t& parity) {
    constexpr uint32_t kValWords = kPairs ? kTile : 0;
    KeyT* in_keys = reinterpret_cast<KeyT*>(smem);  // next tile, filled by TMA
    uint32_t* in_vals = reinterpret_cast<uint32_t*>(in_keys + kTile);
    KeyT* skeys = reinterpret_cast<KeyT*>(in_vals + kValWords);  // tile in digit order
    uint32_t* svals = reinterpret_cast<uint32_t*>(skeys + kTile);
    uint32_t* wcnt = svals + kValWords;        // [kWarps][kBins] digit counts
    uint32_t* wmask = wcnt + kWarps * kBins;   // [kWarps][kBins] lanes holding each digit, kept zero
    uint32_t* dstart = wmask + kWarps * kBins;  // tile-local start of each digit
    uint32_t* gnext = dstart + kBins;           // running output offset of each digit
    uint32_t* shift_out = gnext + kBins;        // gnext - dstart: tile slot -> output index
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(shift_out + kBins);

    uint32_t t0, t1;
    chunk_range(n, t0, t1);
    if (t0 >= t1) return true;  // a chunk without tiles
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int d = threadIdx.x;
    gnext[d] = chunk_offsets[(uint64_t)blockIdx.x * kBins + d];
    for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) wmask[i] = 0;
    __syncthreads();

    auto full = [&](uint32_t tile) { return (uint64_t)(tile + 1) * kTile <= n; };
    auto prefetch = [&](uint32_t tile) {
        mbar_expect_tx(bar, kTile * (uint32_t)(sizeof(KeyT) + (kPairs ? 4 : 0)));
        tma_bulk_load(in_keys, kin + (uint64_t)tile * kTile, kTile * (uint32_t)sizeof(KeyT), bar);
        if (kPairs) tma_bulk_load(in_vals, vin + (uint64_t)tile * kTile, kTile * 4u, bar);
    };
    if (threadIdx.x == 0 && full(t0)) {
        fence_proxy_async_smem();
        prefetch(t0);
    }
    for (uint32_t tile = t0; tile < t1; ++tile) {
        const uint64_t base = (uint64_t)tile * kTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kTile, (uint64_t)n - base);
        const bool whole = full(tile);
        bool ok = true;
        if (whole) {
            ok = mbar_wait(bar, parity, kMbarSpinLimit);
            parity ^= 1u;
        } else {
            for (uint32_t i = threadIdx.x; i < cnt; i += kThreads) {
                in_keys[i] = kin[base + i];
                if (kPairs) in_vals[i] = vin[base + i];
            }
        }
        for (int i = threadIdx.x; i < kWarps * kBins; i += kThreads) wcnt[i] = 0;
        if (!__syncthreads_and(ok)) {
            // gave up on the copy: flag it, give the copy one more bounded
            // chance to land (it writes this CTA's shared memory), and stop
            if (threadIdx.x == 0) atomicOr(d_err, 256u);
            mbar_wait(bar, parity ^ 1u, kMbarSpinLimit);
            return false;
        }
        KeyT k[kItems];
        uint32_t v[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t i = warp * kWarpItems + it * 32 + lane;
            k[it] = i < cnt ? in_keys[i] : KeyT(0);
            v[it] = (kPairs && i < cnt) ? in_vals[i] : 0u;
        }
        __syncthreads();  // the input buffer is free: fetch the next tile
        if (threadIdx.x == 0 && tile + 1 < t1 && full(tile + 1)) {
            fence_proxy_async_smem();
            prefetch(tile + 1);
        }

        // rank among equal digits of the warp, in index order: the lanes
        // with digit dg are the bits set in wm[dg] once every lane has set
        // its own; the lowest of them adds their number to the warp's count
        // and clears the mask word for the next item
        uint32_t* my = wcnt + warp * kBins;
        uint32_t* wm = wmask + warp * kBins;
        uint32_t dr[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const uint32_t i = warp * kWarpItems + it * 32 + lane;
            const bool valid = i < cnt;
            const uint32_t dg = (uint32_t)(k[it] >> shift) & (kBins - 1);
            if (valid) atomicOr(&wm[dg], 1u << lane);
            __syncwarp();
            const uint32_t peers = valid ? wm[dg] : 0u;
            const uint32_t prior = valid ? my[dg] : 0u;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) {
                my[dg] = prior + __popc(peers);
                wm[dg] = 0;
            }
            __syncwarp();
            dr[it] = valid ? ((dg << 16) | (prior + __popc(peers & lt))) : 0xFFFFFFFFu;
        }
        __syncthreads();

        // tile counts per digit; exclusive offsets across warps and digits
        uint32_t cnt_d = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcnt[w * kBins + d];
            wcnt[w * kBins + d] = cnt_d;
            cnt_d += t;
        }
        uint32_t tile_total;
        const uint32_t ds = cta_exclusive_scan<SumOp, kThreads>(cnt_d, tile_total);
        dstart[d] = ds;
        shift_out[d] = gnext[d] - ds;
        __syncthreads();

#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            if (dr[it] == 0xFFFFFFFFu) continue;
            const uint32_t dd = dr[it] >> 16;
            const uint32_t pos = dstart[dd] + wcnt[warp * kBins + dd] + (dr[it] & 0xFFFFu);
            if (pos < kTile) {
                skeys[pos] = k[it];
                if (kPairs) svals[pos] = v[it];
            } else {
                atomicOr(d_err, 16u);
            }
        }
        __syncthreads();

        if (whole) {
            // all loads of the thread's slots first, then all stores
            uint32_t o[kItems];
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                const uint32_t s = threadIdx.x + j * kThreads;
                k[j] = skeys[s];
                if (kPairs) v[j] = svals[s];
            }
#pragma unroll
            for (int j = 0; j < kItems; ++j)
                o[j] = shift_out[(uint32_t)(k[j] >> shift) & (kBins - 1)] + threadIdx.x + j * kThreads;
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                if (o[j] < n) {
                    kout[o[j]] = k[j];
                    if (kPairs) vout[o[j]] = v[j];
                } else {
                    atomicOr(d_err, 16u);
                }
            }
        } else {
            for (uint32_t s = threadIdx.x; s < cnt; s += kThreads) {
                const KeyT key = skeys[s];
                const uint32_t o = shift_out[(uint32_t)(key >> shift) & (kBins - 1)] + s;
                if (o < n) {
                    kout[o] = key;
                    if (kPairs) vout[o] = svals[s];
                } else {
                    atomicOr(d_err, 16u);
                }
            }
        }
        __syncthreads();
        gnext[d] += cnt_d;
    }
    return true;
}

template <class KeyT, bool kPairs>
__global__ void __launch_bounds__(kThreads, 3) radix_downsweep_kernel(
    const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin, KeyT* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ d_n, int shift,
    const uint32_t* __restrict__ chunk_offsets, uint32_t* __restrict__ d_err) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + down_smem<KeyT, kPairs>() - 16);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    uint32_t parity = 0;
    down_phase<KeyT, kPairs>(kin, vin, kout, vout, *d_n, shift, chunk_offsets, d_err, smem, parity);
}

// ---------------------------------------------------------------------------
// Fused sort: every pass of one sort in a single cooperative launch (all
// CTAs resident), the phases separated by grid barriers.  It serves lists
// whose length is only known on the device and is often zero: then every
// CTA returns at once and the sort costs one launch.

// Grid barrier on two words: arrivals and a generation number.  The last CTA
// to arrive resets the count and advances the generation; the others wait
// for the generation to move, for at most kGridSpinLimit polls (then flag
// *d_err bit 9 and report failure).
__device__ __forceinline__ bool grid_barrier(unsigned* gbar, unsigned& gen, uint32_t* d_err) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned prev = atomicAdd(&gbar[0], 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&gbar[0], 0u);
            __threadfence();
            atomicAdd(&gbar[1], 1u);
        } else {
            uint32_t polls = 0;
            while (*reinterpret_cast<volatile unsigned*>(&gbar[1]) == gen) {
                if (++polls > kGridSpinLimit) {
                    ok = 0;
                    atomicOr(d_err, 512u);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ++gen;
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Output offsets of every (chunk, digit) from the chunk counts, in two
// steps over work items (digit d, group q of consecutive chunks), one warp
// per item: first the count of each group, then each group's running sum.
__device__ __forceinline__ void chunk_groups(uint32_t nchunks, uint32_t& per) {
    per = (nchunks + kFusedGroups - 1) / kFusedGroups;
}
__device__ __forceinline__ void scan_a_phase(const uint32_t* __restrict__ chunk_counts, uint32_t nchunks,
                                             uint32_t* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * kWarps;
    uint32_t per;
    chunk_groups(nchunks, per);
    for (uint32_t item = blockIdx.x * kWarps + (threadIdx.x >> 5); item < (uint32_t)kBins * kFusedGroups;
         item += warps) {
        const uint32_t d = item % kBins, q = item / kBins;
        const uint32_t c0 = min(nchunks, q * per), c1 = min(nchunks, c0 + per);
        uint32_t sum = 0;
        for (uint32_t c = c0 + lane; c < c1; c += 32) sum += chunk_counts[(uint64_t)c * kBins + d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) partials[q * kBins + d] = sum;
    }
}
__device__ __forceinline__ void scan_b_phase(uint32_t* __restrict__ chunk_counts, uint32_t nchunks,
                                             const uint32_t* __restrict__ partials,
                                             const uint32_t* __restrict__ totals) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * kWarps;
    uint32_t per;
    chunk_groups(nchunks, per);
    for (uint32_t item = blockIdx.x * kWarps + (threadIdx.x >> 5); item < (uint32_t)kBins * kFusedGroups;
         item += warps) {
        const uint32_t d = item % kBins, q = item / kBins;
        // start of digit d in the output, plus its count in earlier groups
        uint32_t run = 0;
        for (uint32_t e = lane; e < d; e += 32) run += totals[e];
        for (uint32_t g = lane; g < q; g += 32) run += partials[g * kBins + d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xffffffffu, run, o);
        const uint32_t c0 = min(nchunks, q * per), c1 = min(nchunks, c0 + per);
        for (uint32_t cb = c0; cb < c1; cb += 32) {
            const uint32_t c = cb + lane;
            const uint32_t v = c < c1 ? chunk_counts[(uint64_t)c * kBins + d] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (c < c1) chunk_counts[(uint64_t)c * kBins + d] = run + x - v;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

template <class KeyT>
__global__ void __launch_bounds__(kThreads, 3) radix_sort_fused_kernel(KeyT* __restrict__ keys,
                                                                       uint32_t* __restrict__ vals,
                                                                       KeyT* __restrict__ keys_alt,
                                                                       uint32_t* __restrict__ vals_alt,
                                                                       const uint32_t* __restrict__ d_n,
                                                                       int begin_bit, int passes,
                                                                       uint32_t* __restrict__ temp,
                                                                       uint32_t* __restrict__ d_err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t n = *d_n;
    if (n == 0) return;  // the whole grid leaves together
    unsigned* gbar = temp + kGridBar;
    unsigned gen = *reinterpret_cast<volatile unsigned*>(&gbar[1]);  // read before this CTA's first arrival
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + down_smem<KeyT, true>() - 16);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    uint32_t parity = 0;
    uint32_t ntiles;
    const uint32_t tpc = tiles_per_chunk(n, gridDim.x, ntiles);
    const uint32_t nchunks = tpc ? (ntiles + tpc - 1) / tpc : 0;
    uint32_t* chunk = temp + kChunkOffsets;
    uint32_t* partials = temp + kPartials;
    for (int p = 0; p < passes; ++p) {
        const bool alt = p & 1;
        const KeyT* kin = alt ? keys_alt : keys;
        const uint32_t* vin = alt ? vals_alt : vals;
        KeyT* ko = alt ? keys : keys_alt;
        uint32_t* vo = alt ? vals : vals_alt;
        const int shift = begin_bit + kRadixBits * p;
        uint32_t* totals = temp + kTotals + (size_t)kBins * (p & 1);
        uint32_t* next_totals = temp + kTotals + (size_t)kBins * ((p + 1) & 1);
        up_phase(kin, n, shift, chunk, totals, reinterpret_cast<uint32_t*>(smem));
        if (!grid_barrier(gbar, gen, d_err)) return;
        scan_a_phase(chunk, nchunks, partials);
        if (blockIdx.x == 0) next_totals[threadIdx.x] = 0;
        if (!grid_barrier(gbar, gen, d_err)) return;
        scan_b_phase(chunk, nchunks, partials, totals);
        if (!grid_barrier(gbar, gen, d_err)) return;
        if (!down_phase<KeyT, true>(kin, vin, ko, vo, n, shift, chunk, d_err, smem, parity)) return;
        if (!grid_barrier(gbar, gen, d_err)) return;
    }
}

unsigned g_keys_ctas[64] = {0};  // downsweep CTAs of the keys-only sort, per device
unsigned g_fused_ctas[64] = {0};


int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

}  // namespace

unsigned persistent_ctas(const void* kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    cudaGetLastError();
    return (unsigned)(std::max(1, sms) * std::max(1, per_sm));
}

unsigned radix_keys_grid(uint64_t cap) {
    const uint64_t tiles = cap / kTile + 1;
    return (unsigned)std::min<uint64_t>(std::max(1u, g_keys_ctas[current_device()]), tiles);
}

uint32_t* radix_first_counts(uint32_t* temp) { return temp + kChunkOffsets; }
uint32_t* radix_first_totals(uint32_t* temp) { return temp + kTotals; }

void radix_clear(Launcher& L, uint32_t* temp) { cudaMemsetAsync(temp, 0, (kGridBar + 2) * 4, L.stream); }

size_t radix_temp_words(uint64_t cap) {
    const uint64_t chunks = std::min<uint64_t>(kMaxChunks, cap / kTile + 1);
    return kChunkOffsets + (size_t)chunks * kBins + 64;
}

void radix_init() {
    using u64 = unsigned long long;
    const size_t ks = down_smem<u64, false>();
    cudaFuncSetAttribute(radix_downsweep_kernel<u64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks);
    g_keys_ctas[current_device()] =
        std::min<unsigned>(kMaxChunks, persistent_ctas((const void*)radix_downsweep_kernel<u64, false>, kThreads, ks));
    const size_t smem = down_smem<u64, true>();
    cudaFuncSetAttribute(radix_sort_fused_kernel<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_fused_ctas[current_device()] =
        std::min<unsigned>(kMaxChunks, persistent_ctas((const void*)radix_sort_fused_kernel<u64>, kThreads, smem));
}

bool radix_sort_keys(Launcher& L, unsigned long long* keys, unsigned long long* keys_alt, const uint32_t* d_n,
                     uint64_t cap, int begin_bit, int end_bit, uint32_t* temp, uint32_t* d_err,
                     bool first_counted) {
    using u64 = unsigned long long;
    const int passes = radix_passes(begin_bit, end_bit);
    if (passes <= 0) return false;
    uint32_t* chunk = temp + kChunkOffsets;
    const unsigned grid = radix_keys_grid(cap);
    auto* const down_kernel = radix_downsweep_kernel<u64, false>;
    const size_t down_bytes = down_smem<u64, false>();
    bool alt = false;
    for (int p = 0; p < passes; ++p) {
        const u64* kin = alt ? keys_alt : keys;
        u64* ko = alt ? keys : keys_alt;
        const int shift = begin_bit + kRadixBits * p;
        uint32_t* totals = temp + kTotals + (size_t)kBins * (p & 1);
        uint32_t* next_totals = temp + kTotals + (size_t)kBins * ((p + 1) & 1);
        if (p > 0 || !first_counted) {
            if (p == 0) radix_clear(L, temp);
            SBWT_LAUNCH(L, "radix_upsweep", 0, 8, d_n, radix_upsweep_kernel<u64>, grid, kThreads, 0, kin, d_n,
                        shift, chunk, totals);
        }
        SBWT_LAUNCH(L, "radix_chunk_scan", 12.0 * grid * kBins, 0, nullptr, radix_chunk_scan_kernel,
                    kBins / kScanWarps, kScanThreads, 0, chunk, (int)grid, totals, next_totals, d_n);
        // per key: the 8-byte key read and written once
        SBWT_LAUNCH(L, "radix_downsweep", 0, 16, d_n, down_kernel, grid, kThreads, down_bytes, kin, nullptr, ko,
                    nullptr, d_n, shift, chunk, d_err);
        alt = !alt;
    }
    return alt;
}

bool radix_sort_pairs_fused(Launcher& L, unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                            uint32_t* vals_alt, const uint32_t* d_n, uint64_t cap, int begin_bit, int end_bit,
                            uint32_t* temp, uint32_t* d_err) {
    int passes = radix_passes(begin_bit, end_bit);
    if (passes <= 0) return false;
    const int dev = current_device();
    const uint64_t tiles = cap / kTile + 1;
    const unsigned grid = (unsigned)std::min<uint64_t>(std::max(1u, g_fused_ctas[dev]), tiles);
    cudaMemsetAsync(temp, 0, (kGridBar + 2) * 4, L.stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = down_smem<unsigned long long, true>();
    cfg.stream = L.stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // per element and pass: the key read by the count, key and value read
    // and written by the scatter
    const int tok = L.before("radix_sort_fused", 0, (8.0 + 24.0) * passes, d_n);
    cudaLaunchKernelEx(&cfg, radix_sort_fused_kernel<unsigned long long>, keys, vals, keys_alt, vals_alt, d_n,
                       begin_bit, passes, temp, d_err);
    L.after(tok);
    return passes & 1;
}

}  // namespace sbwt
