// noalloc.cu -- sbwt_bwt_noalloc: the BWT of a small read set computed
// without allocating any device memory.
//
// Some callers cannot allocate: a process whose device memory is handed out
// by another framework's pool (every free byte already reserved), a service
// that forbids allocation after start-up so its latency and footprint stay
// fixed, or a plug-in whose host owns the device allocator.  This entry point
// serves them.  All of its working memory is one file-scope device array of
// fixed size, so a read set is limited to SBWT_NOALLOC_MAX_SUFFIXES suffixes
// (reads plus one terminator each).
//
// For a read set that fits one block, Algorithm 1 reduces to ConstructSA and
// B_int (the index it inserts into is empty, so every g is 0 and Insert puts
// new symbol i on row i): B = B_int.  The kernels are the ones sbwt_append
// runs; only their buffers differ.
#include <mutex>

#include "sbwt.h"
#include "sbwt_kernels.cuh"

using namespace sbwt;

namespace {

constexpr uint64_t kMax = SBWT_NOALLOC_MAX_SUFFIXES;

constexpr size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of the scratch array (byte offsets); every part 256-byte aligned.
constexpr size_t kReads = 0;
constexpr size_t kOffsets = kReads + up256(kMax);
constexpr size_t kText = kOffsets + up256((kMax + 1) * 8);
constexpr size_t kTerm = kText + up256(((kMax + 31) / 32 * 2 + kTextPadWords) * 4);
constexpr size_t kKeys = kTerm + up256(((kMax + 31) / 32 + kTermPadWords) * 4);
constexpr size_t kKeysAlt = kKeys + up256(kMax * 8);
constexpr size_t kU32 = kKeysAlt + up256(kMax * 8);  // ten arrays of kMax uint32
constexpr size_t kUnits = kU32 + 10 * up256(kMax * 4);
constexpr size_t kUnitsBytes = 16384;  // suffix_sort_unit_bytes(kMax) must fit (checked at set-up)
constexpr size_t kRadixTemp = kUnits + kUnitsBytes;
constexpr size_t kRadixTempBytes = 256 * 1024;  // radix_temp_words(kMax) * 4 must fit (checked at set-up)
constexpr size_t kChunks = kRadixTemp + kRadixTempBytes;
constexpr size_t kChunksBytes = 16384;  // suffix_sort_chunk_words(kMax) * 8 must fit (checked at set-up)
constexpr size_t kCountLog = kChunks + kChunksBytes;
constexpr size_t kCountLogBytes = 256;
constexpr size_t kBint = kCountLog + kCountLogBytes;
constexpr size_t kOut = kBint + up256(kMax);
constexpr size_t kErr = kOut + up256(kMax);
constexpr size_t kScratchBytes = kErr + 256;

// The scratch.  Every GPU that loads this library holds these bytes until the
// process exits; all calls on a device share them.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceState {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    Launcher L;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

// Once per device, with that device current: look up the array's device
// address (the host-side symbol is only a stand-in) and set the kernel
// attributes the sort needs.
int setup(int dev, DeviceState** out) {
    if (dev < 0 || dev >= kMaxDevices) return SBWT_EDEVICE;
    DeviceState& st = g_dev[dev];
    if (!st.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return SBWT_EDEVICE;
        }
        if (radix_temp_words(kMax) * 4 > kRadixTempBytes || suffix_sort_chunk_words(kMax) * 8 > kChunksBytes ||
            suffix_sort_log_slots((uint32_t)kMax, 2) * 4 > kCountLogBytes || suffix_sort_unit_bytes(kMax) > kUnitsBytes)
            return SBWT_EDEVICE;
        suffix_sort_init();
        st.base = static_cast<unsigned char*>(p);
        st.ready = true;
    }
    *out = &st;
    return SBWT_OK;
}

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) bint_to_bytes_kernel(const uint8_t* __restrict__ bint, uint32_t n,
                                                                 uint32_t alpha4, uint8_t* __restrict__ out) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = bint[i];
    out[i] = c == kBintDollar ? (uint8_t)'$' : (uint8_t)(alpha4 >> (8 * (c & 3)));
}

int parse_alphabet(const char* alphabet, uint32_t* alpha4, int* sigma) {
    if (!alphabet) return SBWT_EINVAL;
    int len = 0;
    while (alphabet[len] && len < 5) ++len;
    if (len < 1 || len > 4) return SBWT_EINVAL;
    uint32_t a4 = 0;
    for (int a = 0; a < len; ++a) {
        const uint8_t c = (uint8_t)alphabet[a];
        if (c == '$' || (a > 0 && c <= (uint8_t)alphabet[a - 1])) return SBWT_EINVAL;
    }
    for (int a = 0; a < 4; ++a) a4 |= (uint32_t)(uint8_t)alphabet[a < len ? a : 0] << (8 * a);
    *alpha4 = a4;
    *sigma = len;
    return SBWT_OK;
}

}  // namespace

extern "C" int sbwt_bwt_noalloc(const char* alphabet, const uint8_t* reads, const uint64_t* offsets, uint64_t m,
                                uint8_t* out, uint64_t cap, uint64_t* n_out, void* stream) {
    if (!offsets || !n_out) return SBWT_EINVAL;
    uint32_t alpha4 = 0;
    int sigma = 0;
    if (parse_alphabet(alphabet, &alpha4, &sigma)) return SBWT_EINVAL;
    if (offsets[0] != 0) return SBWT_EINVAL;
    // Every read adds at least its terminator, so more than kMax reads can
    // never fit; the byte count and the read count are tested against the
    // limit one at a time, so no sum of caller values can wrap.
    if (m > kMax) return SBWT_EINVAL;
    uint64_t max_len = 0;
    for (uint64_t j = 0; j < m; ++j) {
        if (offsets[j + 1] < offsets[j]) return SBWT_EINVAL;
        if (offsets[j + 1] > kMax || j + 1 > kMax - offsets[j + 1]) return SBWT_EINVAL;  // over the maximum
        if (offsets[j + 1] - offsets[j] > max_len) max_len = offsets[j + 1] - offsets[j];
    }
    const uint64_t nbytes = offsets[m];
    const uint64_t n = nbytes + m;
    *n_out = n;
    if (n > kMax) return SBWT_EINVAL;
    if (cap < n) return SBWT_ERANGE;
    if (n == 0) return SBWT_OK;
    if (!out || (nbytes && !reads)) return SBWT_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SBWT_EDEVICE;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState* st = nullptr;
    if (int rc = setup(dev, &st)) return rc;
    unsigned char* b = st->base;
    cudaStream_t s = (cudaStream_t)stream;
    Launcher& L = st->L;
    L.stream = s;
    L.unit_log = nullptr;
    L.unit_log_len = 0;

    uint8_t* d_reads = b + kReads;
    uint64_t* d_off = reinterpret_cast<uint64_t*>(b + kOffsets);
    uint32_t* text = reinterpret_cast<uint32_t*>(b + kText);
    uint32_t* term = reinterpret_cast<uint32_t*>(b + kTerm);
    uint32_t* err = reinterpret_cast<uint32_t*>(b + kErr);
    uint8_t* d_out = b + kOut;
    uint32_t* u32 = reinterpret_cast<uint32_t*>(b + kU32);
    const size_t stride = up256(kMax * 4) / 4;
    SuffixSortBuffers sb;
    sb.keys = reinterpret_cast<unsigned long long*>(b + kKeys);
    sb.keys_alt = reinterpret_cast<unsigned long long*>(b + kKeysAlt);
    sb.vals = u32;
    sb.vals_alt = u32 + stride;
    sb.sa = u32 + 2 * stride;
    sb.rank = u32 + 3 * stride;
    sb.act_pos[0] = u32 + 4 * stride;
    sb.act_pos[1] = u32 + 5 * stride;
    sb.act_suf[0] = u32 + 6 * stride;
    sb.act_suf[1] = u32 + 7 * stride;
    sb.loc_act = u32 + 8 * stride;
    sb.loc_next = u32 + 9 * stride;
    sb.units = b + kUnits;
    sb.radix_temp = reinterpret_cast<uint32_t*>(b + kRadixTemp);
    sb.chunks = reinterpret_cast<unsigned long long*>(b + kChunks);
    sb.count_log = reinterpret_cast<uint32_t*>(b + kCountLog);
    sb.err = err;
    uint8_t* bint = b + kBint;

    // The array keeps the previous call's contents: clear what must start at
    // zero (the error word and the padding past the packed text).
    const uint64_t text_words = (n + 31) / 32 * 2, term_words = (n + 31) / 32;
    uint32_t h_err = 0;
    bool ok = true;
    if (nbytes) ok &= cudaMemcpyAsync(d_reads, reads, nbytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok &= cudaMemcpyAsync(d_off, offsets, (m + 1) * 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok &= cudaMemsetAsync(text + text_words, 0, kTextPadWords * 4, s) == cudaSuccess;
    ok &= cudaMemsetAsync(term + term_words, 0, kTermPadWords * 4, s) == cudaSuccess;
    ok &= cudaMemsetAsync(err, 0, 4, s) == cudaSuccess;
    if (!ok) {
        // copies queued before the failure may still be writing the shared
        // array: let them finish before the lock is released
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return SBWT_EDEVICE;
    }
    launch_pack(L, d_reads, d_off, m, n, alpha4, sigma, text, term, err);
    suffix_sort_block(L, text, term, 0, (uint32_t)n, (uint32_t)max_len, 2, sigma, sb);
    launch_bint(L, text, term, 0, sb.sa, (uint32_t)n, bint);
    SBWT_LAUNCH(L, "bint_to_bytes", 2.0 * n, 0, nullptr, bint_to_bytes_kernel, ceil_div_u(n, kThreads), kThreads, 0,
                bint, (uint32_t)n, alpha4, d_out);
    ok &= cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok &= cudaMemcpyAsync(out, d_out, n, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok &= cudaGetLastError() == cudaSuccess;
    // always drain the stream before the lock is released, even after a
    // failed launch or copy, so no later call can overlap this one's work
    ok &= cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return SBWT_EDEVICE;
    }
    if (h_err & 1u) return SBWT_EINVAL;  // a byte outside the alphabet
    if (h_err) return SBWT_EDEVICE;
    return SBWT_OK;
}
