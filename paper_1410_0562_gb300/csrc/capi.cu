// capi.cu -- the index runtime behind include/sbwt.h: device state, the
// memory plan under the HBM budget, block planning and the per-block
// pipeline of Algorithm 1 (arXiv 1410.0562):
//   ConstructSA -> B_int -> ComputeRanks -> g[SA_int] -> Insert.
// Host code only orchestrates; every step of the path is a CUDA kernel.
#include <algorithm>
#include <chrono>
#include <functional>
#include <string>
#include <thread>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sbwt.h"
#include "sbwt_kernels.cuh"
#include "sbwt_serve.h"

using namespace sbwt;

namespace {

// A buffer in HBM, or (host tier) in mapped pinned host memory that kernels
// reach over the host link through the same unified address.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool host = false;
};

struct Dict {
    DevBuf blocks, super, C;
};

struct BlockPlan {
    uint64_t j0, j1;    // reads [j0, j1) of the append
    uint64_t n_int;     // suffixes (symbols + terminators)
    uint64_t base;      // text position of the block's first suffix
    uint64_t max_len;   // longest read
};

constexpr uint64_t kDefaultBlock = 1ull << 24;
constexpr uint64_t kMaxBlock = 1ull << 31;
constexpr unsigned kPlanCap = 4096;  // blocks a device-planned append may have

}  // namespace

struct sbwt_index {
    uint8_t alphabet[16] = {0};
    int sigma = 0;
    uint32_t alpha4 = 0;     // the first four symbols, packed (2-bit kernels)
    Alphabet16 alpha16 = {};  // all symbols (4-bit kernels, read-back)
    int code_bits = 2;       // 2 for up to 4 symbols, 4 for 5 to 16
    int occ_k = 1;           // occurrence sampling of 64 occ_k rows (1, 2 or 4; 1 for 4-bit codes)
    sbwt_tile_shapes tiles = {};  // launch shapes the autotuner may pick (0 = the built-in choice)
    size_t budget = 0;
    uint32_t index_bits = 0;
    uint64_t M = kDefaultBlock;
    bool host_tier_allowed = true;  // dictionaries may move to pinned host memory
    bool dict_host = false;         // they live there now
    bool host_tier_forced = false;  // keep them there even when HBM has room
    int device = -1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // The suffix sorts of an append's blocks run on a second stream, ahead of
    // the ComputeRanks -> B_int/g_sa -> Insert chain on `stream`: a block's
    // sort reads only the packed text.  Its SA_int goes to one of two buffers
    // (sa, sa2 by block parity).
    cudaStream_t side = nullptr;
    bool overlap = true;  // sorts on `side` ahead of the chain; off: every step in turn on `stream`
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_sorted[2] = {nullptr, nullptr},
                ev_consumed[2] = {nullptr, nullptr};
    // host appends: block k's text is packed as soon as its reads arrive;
    // its sort waits on ev_packed[k] (grown on demand)
    std::vector<cudaEvent_t> ev_packed;
    bool dev_ready = false;

    uint64_t n = 0, m = 0;
    Dict dict[3];
    int cur = 0;

    DevBuf reads, offsets, text, term, err;
    DevBuf keys, keys_alt, vals, vals_alt, sa, sa2, rank, act_pos0, act_pos1, act_suf0, act_suf1, loc_act, loc_next;
    DevBuf units;
    DevBuf radix_temp, chunks, count_log, g, gsa, bint, sb_tot, ins_plan, stage;
    // The host tier rewrites its one dictionary in place: an append that
    // fails after the rewrite began leaves it broken until sbwt_reset.
    bool broken = false;
    DevBuf out_bytes, q_codes, q_ks, q_out, c_pats, c_offs;

    uint32_t* h_err = nullptr;      // pinned
    uint64_t* h_offsets = nullptr;  // pinned staging for device-side offsets (fallback planning)
    size_t h_offsets_cap = 0;
    DevBuf plan;                     // device block table + summary
    PlanBlock* h_plan = nullptr;     // pinned copy of the table
    PlanSummary* h_summary = nullptr;

    Launcher L;
    // Instantiated CUDA graphs of whole appends, one per pipeline shape (the
    // sequence of kernels an append launches); each append is captured and
    // updates the graph of its shape in place before it is launched.
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        Launcher::GraphLog log;
    };
    bool graph_replay = false;
    std::vector<GraphEntry> graphs;  // most recent last
    void* server = nullptr;           // continuous-batching server, when serving
    std::thread::id server_worker;    // the only thread that may change the index then
    bool capture = false;
    bool last_valid = false;
    uint64_t last_n = 0;
    bool last_idx64 = false;
    const void* last_sa = nullptr;  // the SA_int buffer of the last block

    std::vector<DevBuf*> all_bufs() {
        std::vector<DevBuf*> v = {&reads,      &offsets,  &text,      &term,     &err,      &keys,
                                  &keys_alt,   &vals,     &vals_alt,  &sa,       &rank,     &act_pos0,
                                  &act_pos1,   &act_suf0, &act_suf1,  &loc_act,  &loc_next, &units,     &sa2,
                                  &radix_temp, &chunks,
                                  &count_log,  &g,        &gsa,       &bint,     &sb_tot,   &ins_plan, &stage, &out_bytes,
                                  &q_codes,    &q_ks,     &q_out,     &plan,     &c_pats,   &c_offs};
        for (auto& d : dict) {
            v.push_back(&d.blocks);
            v.push_back(&d.super);
            v.push_back(&d.C);
        }
        return v;
    }
    size_t held_bytes(bool host = false) {
        size_t s = 0;
        for (DevBuf* b : all_bufs())
            if (b->host == host) s += b->bytes;
        return s;
    }
};

namespace {

// While a server runs, only its worker may use the index (besides
// submit/wait and the read-only size query).
bool busy(const sbwt_index* idx) { return idx->server && std::this_thread::get_id() != idx->server_worker; }

int set_device(sbwt_index* idx) {
    if (idx->device >= 0 && cudaSetDevice(idx->device) != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

void free_buf(DevBuf& b) {
    if (b.p) {
        if (b.host)
            cudaFreeHost(b.p);
        else
            cudaFree(b.p);
    }
    b.p = nullptr;
    b.bytes = 0;
    b.host = false;
}

void* alloc_tier(size_t bytes, bool host) {
    void* p = nullptr;
    cudaError_t e = host ? cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable)
                         : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Makes b hold at least `bytes` in the given tier (contents are not kept
// when it grows or moves).
int grow(DevBuf& b, size_t bytes, bool host = false) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (b.bytes >= bytes && b.host == host) return SBWT_OK;
    free_buf(b);
    b.p = alloc_tier(bytes, host);
    if (!b.p) return SBWT_ENOMEM;
    b.bytes = bytes;
    b.host = host;
    return SBWT_OK;
}

constexpr int kZeroThreads = 256;
__global__ void zero_words_kernel(unsigned long long* p, uint64_t words) {
    const uint64_t i = (uint64_t)blockIdx.x * kZeroThreads + threadIdx.x;
    if (i < words) p[i] = 0ull;
}

// Zeroes the first `bytes` (a multiple of 8) of a buffer in either tier.
void zero_async(const DevBuf& b, size_t bytes, cudaStream_t s) {
    const uint64_t words = bytes / 8;
    if (words) zero_words_kernel<<<ceil_div_u(words, kZeroThreads), kZeroThreads, 0, s>>>(
        (unsigned long long*)b.p, words);
}

int device_init(sbwt_index* idx) {
    if (idx->dev_ready) return set_device(idx);
    if (idx->device < 0) {
        if (cudaGetDevice(&idx->device) != cudaSuccess) return SBWT_EDEVICE;
    }
    if (set_device(idx)) return SBWT_EDEVICE;
    if (!idx->stream) {
        if (cudaStreamCreateWithFlags(&idx->stream, cudaStreamNonBlocking) != cudaSuccess) return SBWT_EDEVICE;
        idx->own_stream = true;
    }
    idx->L.stream = idx->stream;
    if (cudaStreamCreateWithFlags(&idx->side, cudaStreamNonBlocking) != cudaSuccess) return SBWT_EDEVICE;
    for (cudaEvent_t* e : {&idx->ev_fork, &idx->ev_join, &idx->ev_sorted[0], &idx->ev_sorted[1],
                           &idx->ev_consumed[0], &idx->ev_consumed[1]})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return SBWT_EDEVICE;
    suffix_sort_init();
    if (cudaMallocHost(&idx->h_err, sizeof(uint32_t)) != cudaSuccess) return SBWT_EDEVICE;
    if (cudaMallocHost(&idx->h_plan, kPlanCap * sizeof(PlanBlock)) != cudaSuccess) return SBWT_EDEVICE;
    if (cudaMallocHost(&idx->h_summary, sizeof(PlanSummary)) != cudaSuccess) return SBWT_EDEVICE;
    // the committed dictionary starts empty: one zero block, one zero superblock, C = 0
    Dict& d = idx->dict[idx->cur];
    const size_t bb = dict_block_bytes(idx->code_bits, idx->occ_k), cb = 8 * dict_codes(idx->code_bits);
    if (grow(d.blocks, bb) || grow(d.super, cb) || grow(d.C, cb)) return SBWT_ENOMEM;
    zero_async(d.blocks, bb, idx->stream);
    zero_async(d.super, cb, idx->stream);
    zero_async(d.C, cb, idx->stream);
    if (grow(idx->err, 4)) return SBWT_ENOMEM;
    if (cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
    idx->dev_ready = true;
    return SBWT_OK;
}

int validate_offsets(const uint64_t* off, uint64_t m) {
    if (off[0] != 0) return SBWT_EINVAL;
    for (uint64_t j = 0; j < m; ++j) {
        if (off[j + 1] < off[j]) return SBWT_EINVAL;
        if (off[j + 1] - off[j] + 1 > kMaxBlock) return SBWT_EINVAL;  // block-local indices are 32-bit
    }
    return SBWT_OK;
}

// Greedy partition (Algorithm 1: blocks of roughly M suffixes): whole reads
// while the block stays within M suffixes; a longer read is a block alone.
std::vector<BlockPlan> plan_blocks(const uint64_t* off, uint64_t m, uint64_t M) {
    std::vector<BlockPlan> v;
    uint64_t j = 0;
    while (j < m) {
        BlockPlan b{j, j, 0, off[j] + j, 0};
        while (j < m) {
            const uint64_t len = off[j + 1] - off[j];
            if (b.n_int > 0 && b.n_int + len + 1 > M) break;
            b.n_int += len + 1;
            b.max_len = std::max(b.max_len, len);
            ++j;
        }
        b.j1 = j;
        v.push_back(b);
    }
    return v;
}

struct Plan {
    std::vector<BlockPlan> blocks;
    uint64_t npos = 0, nbytes = 0, cap = 0, max_len = 0;
    size_t slots = 0;
    bool idx64 = false;
    bool prepend = false;  // the reads go before every read in the index (blocks run last to first)
};

struct Need {
    DevBuf* buf;
    size_t bytes;
    bool dict = false;  // a dictionary buffer: may live in the host tier
};

// The buffers an append needs: the block working set, and either the two
// scratch dictionaries blocks alternate between (in HBM, or in the host tier
// if the committed one is there), or, in place (the host tier), the staging
// buffer of the chunked in-place Insert.
std::vector<Need> buffer_needs(sbwt_index* idx, const Plan& p, bool host_input, uint64_t m_new,
                               bool in_place = false) {
    const uint64_t cap = std::max<uint64_t>(p.cap, 1);
    const size_t w = p.idx64 ? 8 : 4;
    const uint64_t n_final = idx->n + p.npos;
    std::vector<Need> v;
    if (host_input) {
        v.push_back({&idx->reads, (size_t)p.nbytes});
        v.push_back({&idx->offsets, (size_t)(m_new + 1) * 8});
    }
    v.push_back({&idx->text, (size_t)(text_words(p.npos, idx->code_bits) + kTextPadWords) * 4});
    v.push_back({&idx->term, (size_t)((p.npos + 31) / 32 + kTermPadWords) * 4});
    for (DevBuf* b : {&idx->keys, &idx->keys_alt}) v.push_back({b, (size_t)cap * 8});
    for (DevBuf* b : {&idx->vals, &idx->vals_alt, &idx->sa, &idx->sa2, &idx->rank, &idx->act_pos0, &idx->act_pos1,
                      &idx->act_suf0, &idx->act_suf1, &idx->loc_act, &idx->loc_next})
        v.push_back({b, (size_t)cap * 4});
    v.push_back({&idx->units, suffix_sort_unit_bytes(cap)});
    v.push_back({&idx->radix_temp, radix_temp_words(cap) * 4});
    v.push_back({&idx->chunks, suffix_sort_chunk_words(cap) * 8});
    v.push_back({&idx->count_log, p.slots * p.blocks.size() * 4});
    v.push_back({&idx->g, (size_t)cap * w});
    v.push_back({&idx->gsa, (size_t)cap * w});
    v.push_back({&idx->bint, (size_t)cap});
    const int cb = idx->code_bits;
    const uint64_t nsb = dict_supers_of(n_final, cb);
    // superblock totals, then the superblock scan's per-256 totals (insert.cu)
    const size_t sb_words = (size_t)((nsb * dict_codes(cb) + 3) & ~3ull);
    v.push_back({&idx->sb_tot, sb_words * 4 + (size_t)(nsb / 256 + 1) * 8 * dict_codes(cb)});
    v.push_back({&idx->ins_plan, (size_t)(nsb + 1) * 4});  // Insert's first new symbol per superblock
    if (in_place) {
        v.push_back({&idx->stage, (size_t)insert_stage_blocks(cb, idx->occ_k, n_final) *
                                      dict_block_bytes(cb, idx->occ_k)});
        return v;
    }
    for (int k = 0; k < 3; ++k) {
        if (k == idx->cur) continue;
        v.push_back({&idx->dict[k].blocks, (size_t)dict_blocks(n_final, idx->occ_k) * dict_block_bytes(cb, idx->occ_k),
                     true});
        v.push_back({&idx->dict[k].super, (size_t)nsb * 8 * dict_codes(cb), true});
        v.push_back({&idx->dict[k].C, 8 * dict_codes(cb), true});
    }
    return v;
}

void drop_graphs(sbwt_index* idx) {
    for (auto& g : idx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        idx->L.recycle(g.log);
    }
    idx->graphs.clear();
}

size_t rounded(size_t b) { return (b + 255) & ~(size_t)255; }

// HBM the index would hold after growing to `needs`, with the dictionaries
// in the host tier or not.
size_t hbm_after(sbwt_index* idx, const std::vector<Need>& needs, bool dict_host) {
    size_t total = 0;
    for (DevBuf* b : idx->all_bufs()) {
        bool counted = false;
        for (const Need& n : needs)
            if (n.buf == b) {
                counted = true;
                const bool host = n.dict && dict_host;
                if (!host) total += std::max(rounded(n.bytes), b->host ? 0 : b->bytes);
            }
        if (!counted) {
            const bool is_dict = b == &idx->dict[0].blocks || b == &idx->dict[0].super || b == &idx->dict[0].C ||
                                 b == &idx->dict[1].blocks || b == &idx->dict[1].super || b == &idx->dict[1].C ||
                                 b == &idx->dict[2].blocks || b == &idx->dict[2].super || b == &idx->dict[2].C;
            if (!b->host && !(is_dict && dict_host)) total += b->bytes;
        }
    }
    return total;
}

// Moves the committed dictionary to the host tier (its contents are kept);
// the scratch dictionaries follow on their next growth.
int move_dicts_to_host(sbwt_index* idx) {
    Dict& d = idx->dict[idx->cur];
    for (DevBuf* b : {&d.blocks, &d.super, &d.C}) {
        if (b->host || !b->p) continue;
        void* h = alloc_tier(b->bytes, true);
        if (!h) return SBWT_ENOMEM;
        if (cudaMemcpyAsync(h, b->p, b->bytes, cudaMemcpyDeviceToHost, idx->stream) != cudaSuccess ||
            cudaStreamSynchronize(idx->stream) != cudaSuccess) {
            cudaFreeHost(h);
            return SBWT_EDEVICE;
        }
        cudaFree(b->p);
        b->p = h;
        b->host = true;
    }
    for (int k = 0; k < 3; ++k)
        if (k != idx->cur)
            for (DevBuf* b : {&idx->dict[k].blocks, &idx->dict[k].super, &idx->dict[k].C})
                if (!b->host) free_buf(*b);
    idx->dict_host = true;
    return SBWT_OK;
}

// Budget check first (nothing changes on failure), then growth.  When the
// HBM budget cannot hold the dictionaries, they move to pinned host memory
// (Section 5 keeps B_ext in system memory) and only the working set stays in HBM.
int reserve(sbwt_index* idx, const std::vector<Need>& needs) {
    bool dict_host = idx->dict_host || idx->host_tier_forced;
    if (idx->budget && hbm_after(idx, needs, dict_host) > idx->budget) {
        if (dict_host || !idx->host_tier_allowed || hbm_after(idx, needs, true) > idx->budget) return SBWT_ENOMEM;
        dict_host = true;
    }
    if (dict_host && !idx->dict_host) {
        if (int rc = move_dicts_to_host(idx)) return rc;
    }
    // (a buffer that grows or moves needs no graph dropped: every append's
    // capture names the current buffers, and a graph is updated from it
    // before each launch)
    for (const Need& n : needs) {
        const bool host = n.dict && dict_host;
        if (int rc = grow(*n.buf, n.bytes, host)) return rc;
    }
    return SBWT_OK;
}

// Grows b to at least `bytes` in its tier, keeping its contents (the host
// tier's one dictionary grows in place; a quarter of slack per growth).
int grow_keep(DevBuf& b, size_t bytes, cudaStream_t s) {
    bytes = rounded(bytes);
    if (b.bytes >= bytes) return SBWT_OK;
    const size_t nb = std::max(bytes, rounded(b.bytes + b.bytes / 4));
    void* p = alloc_tier(nb, b.host);
    if (!p) return SBWT_ENOMEM;
    if (b.p && b.bytes &&
        (cudaMemcpyAsync(p, b.p, b.bytes, cudaMemcpyDefault, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)) {
        cudaGetLastError();
        if (b.host) cudaFreeHost(p); else cudaFree(p);
        return SBWT_EDEVICE;
    }
    if (b.p) {
        if (b.host) cudaFreeHost(b.p); else cudaFree(b.p);
    }
    b.p = p;
    b.bytes = nb;
    return SBWT_OK;
}

// The buffers of an append under the HBM budget.  While the dictionaries fit
// it, blocks alternate between two scratch dictionaries in HBM and the
// committed one is switched at the end.  Beyond it (or with the host tier
// forced) the index keeps ONE dictionary, in mapped pinned host memory
// (Section 5 keeps B_ext in system memory under a constant working set,
// Section 6): Insert rewrites it in place, so the host holds about 4 bits per
// row (3.25 with sampling 256) instead of three copies, and HBM holds only the
// block working set and the staging buffer.
int reserve_append(sbwt_index* idx, const Plan& p, bool host_input, uint64_t m_new, bool* in_place) {
    *in_place = false;
    if (!(idx->dict_host || idx->host_tier_forced)) {
        auto needs = buffer_needs(idx, p, host_input, m_new, false);
        if (!idx->budget || hbm_after(idx, needs, false) <= idx->budget) return reserve(idx, needs);
        if (!idx->host_tier_allowed) return SBWT_ENOMEM;
    }
    auto needs = buffer_needs(idx, p, host_input, m_new, true);
    if (idx->budget && hbm_after(idx, needs, true) > idx->budget) return SBWT_ENOMEM;
    if (!idx->dict_host) {
        if (int rc = move_dicts_to_host(idx)) return rc;
    }
    for (const Need& n : needs)
        if (int rc = grow(*n.buf, n.bytes, false)) return rc;
    const int cb = idx->code_bits;
    const uint64_t n_final = idx->n + p.npos;
    Dict& d = idx->dict[idx->cur];
    if (int rc = grow_keep(d.blocks, (size_t)dict_blocks(n_final, idx->occ_k) * dict_block_bytes(cb, idx->occ_k),
                           idx->stream))
        return rc;
    if (int rc = grow_keep(d.super, (size_t)dict_supers_of(n_final, cb) * 8 * dict_codes(cb), idx->stream)) return rc;
    if (int rc = grow_keep(d.C, 8 * dict_codes(cb), idx->stream)) return rc;
    *in_place = true;
    return SBWT_OK;
}

// Block k of the append, the q-th to run (q = k unless the append prepends).
template <class IdxT>
void run_block(sbwt_index* idx, const BlockPlan& bp, const uint64_t* d_offsets, const Dict& src, Dict& dst,
               uint64_t n_ext, uint64_t m_ext, size_t slots, size_t k, size_t q, bool prepend,
               cudaEvent_t packed, bool in_place) {
    Launcher& L = idx->L;
    const uint32_t n = (uint32_t)bp.n_int;
    SuffixSortBuffers b;
    b.keys = (unsigned long long*)idx->keys.p;
    b.keys_alt = (unsigned long long*)idx->keys_alt.p;
    b.vals = (uint32_t*)idx->vals.p;
    b.vals_alt = (uint32_t*)idx->vals_alt.p;
    b.sa = (uint32_t*)((q & 1) ? idx->sa2.p : idx->sa.p);
    b.rank = (uint32_t*)idx->rank.p;
    b.act_pos[0] = (uint32_t*)idx->act_pos0.p;
    b.act_pos[1] = (uint32_t*)idx->act_pos1.p;
    b.act_suf[0] = (uint32_t*)idx->act_suf0.p;
    b.act_suf[1] = (uint32_t*)idx->act_suf1.p;
    b.loc_act = (uint32_t*)idx->loc_act.p;
    b.loc_next = (uint32_t*)idx->loc_next.p;
    b.units = idx->units.p;
    b.radix_temp = (uint32_t*)idx->radix_temp.p;
    b.chunks = (unsigned long long*)idx->chunks.p;
    b.count_log = (uint32_t*)idx->count_log.p + slots * k;
    b.err = (uint32_t*)idx->err.p;
    const uint32_t* text = (const uint32_t*)idx->text.p;
    const uint32_t* term = (const uint32_t*)idx->term.p;

    // the sort, on the side stream (or, without overlap, on the index's
    // stream, before this block's other steps); its SA buffer is free once
    // the gather of block k - 2 has read it
    const cudaStream_t s = L.stream;
    const cudaStream_t ss = idx->overlap ? idx->side : s;
    if (q >= 2) cudaStreamWaitEvent(ss, idx->ev_consumed[q & 1], 0);
    if (packed) cudaStreamWaitEvent(ss, packed, 0);  // this block's text is in place
    L.stream = ss;
    suffix_sort_block(L, text, term, bp.base, n, (uint32_t)bp.max_len, idx->code_bits, idx->sigma, b);
    cudaEventRecord(idx->ev_sorted[q & 1], ss);
    L.stream = s;
    // ComputeRanks needs only the dictionary; the gather waits for the sort
    launch_compute_ranks<IdxT>(L, text, d_offsets, bp.j0, bp.j1 - bp.j0, bp.n_int, bp.max_len, (const void*)src.blocks.p,
                               (const unsigned long long*)src.super.p, (const unsigned long long*)src.C.p, n_ext,
                               prepend ? 0 : m_ext, (IdxT*)idx->g.p, (uint32_t*)idx->err.p, idx->code_bits,
                               idx->occ_k, idx->tiles.rank_segment ? idx->tiles.rank_segment : 256u);
    cudaStreamWaitEvent(s, idx->ev_sorted[q & 1], 0);
    // the 2-bit Insert takes its plan (first new symbol per superblock) from the gather
    uint32_t* plan = idx->code_bits == 2 ? (uint32_t*)idx->ins_plan.p : nullptr;
    launch_bint_gather<IdxT>(L, text, term, bp.base, b.sa, (const IdxT*)idx->g.p, n, (uint8_t*)idx->bint.p,
                             (IdxT*)idx->gsa.p, idx->code_bits, plan, dict_supers(n_ext + bp.n_int), kSuperShift);
    cudaEventRecord(idx->ev_consumed[q & 1], s);
    launch_insert<IdxT>(L, (const void*)src.blocks.p, n_ext, (const uint8_t*)idx->bint.p,
                        (const IdxT*)idx->gsa.p, bp.n_int, plan, (void*)dst.blocks.p,
                        (unsigned long long*)dst.super.p, (unsigned long long*)dst.C.p, m_ext + (bp.j1 - bp.j0),
                        (uint32_t*)idx->sb_tot.p, (uint32_t*)idx->err.p, idx->code_bits, idx->occ_k,
                        in_place ? (unsigned long long*)idx->stage.p : nullptr,
                        idx->stage.bytes / dict_block_bytes(idx->code_bits, idx->occ_k), (int)idx->tiles.insert_threads);
}

Plan host_plan(const uint64_t* h_off, uint64_t m_new, uint64_t M) {
    Plan p;
    p.nbytes = h_off[m_new];
    p.npos = p.nbytes + m_new;
    p.blocks = plan_blocks(h_off, m_new, M);
    return p;
}

int append_impl(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, const uint64_t* h_off,
                uint64_t m_new, bool host_input, const uint8_t* h_reads, Plan p,
                std::chrono::steady_clock::time_point t_start) {
    for (const BlockPlan& b : p.blocks) {
        p.cap = std::max(p.cap, b.n_int);
        p.max_len = std::max(p.max_len, b.max_len);
    }
    p.slots = suffix_sort_log_slots((uint32_t)p.max_len, idx->code_bits);
    const uint64_t n_final = idx->n + p.npos;
    if (idx->index_bits == 32 && n_final >= 0xFFFFFFFFull) return SBWT_EINVAL;
    p.idx64 = idx->index_bits == 64 || n_final >= 0xFFFFFFFFull;

    if (int rc = device_init(idx)) return rc;
    bool in_place = false;
    if (int rc = reserve_append(idx, p, host_input, m_new, &in_place)) return rc;
    cudaStream_t s = idx->stream;
    Launcher& L = idx->L;
    if (L.settle_units() != cudaSuccess) return SBWT_EDEVICE;  // the count log is about to be reused
    idx->last_valid = false;  // the scratch arrays are about to be overwritten
    L.unit_log = (const uint32_t*)idx->count_log.p;
    L.unit_log_len = p.slots * p.blocks.size();
    const auto t_plan = std::chrono::steady_clock::now();
    L.add_host("host:plan", std::chrono::duration<double, std::milli>(t_plan - t_start).count());

    // Host reads of an append with several blocks arrive block by block: the
    // copy of block k's bytes, then the packing of its words, and its sort
    // starts while the later blocks' bytes are still on the way.  Chunk k
    // packs the words up to the one holding block k's last position, so it
    // copies the bytes of every position below that word's end (a few
    // positions into block k + 1 at most).  Graph capture keeps one copy.
    // (in place, the foreign-byte check runs before the first block, so the
    // append is eager and packs all of its reads first)
    const bool graph = idx->graph_replay && !in_place;
    const bool pipelined = host_input && !graph && !in_place && p.blocks.size() > 1 && p.nbytes > 0;
    std::vector<uint64_t> chunk_bytes, chunk_words;
    if (pipelined) {
        for (const BlockPlan& b : p.blocks) {
            const uint64_t pos_end = std::min<uint64_t>(p.npos, ((b.base + b.n_int - 1) / 32 + 1) * 32);
            // first read whose first position is at or past pos_end
            uint64_t lo = 0, hi = m_new;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                if (h_off[mid] + mid < pos_end) lo = mid + 1; else hi = mid;
            }
            chunk_bytes.push_back(h_off[lo]);
            chunk_words.push_back((pos_end + 31) / 32);
        }
        chunk_bytes.back() = p.nbytes;
        chunk_words.back() = (p.npos + 31) / 32;
        while (idx->ev_packed.size() < p.blocks.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SBWT_EDEVICE;
            idx->ev_packed.push_back(e);
        }
    }
    if (host_input) {
        cudaMemcpyAsync(idx->offsets.p, h_off, (m_new + 1) * 8, cudaMemcpyHostToDevice, s);
        if (p.nbytes && !pipelined) cudaMemcpyAsync(idx->reads.p, h_reads, p.nbytes, cudaMemcpyHostToDevice, s);
        d_reads = (const uint8_t*)idx->reads.p;
        d_offsets = (const uint64_t*)idx->offsets.p;
    }
    // where each block reads and writes its dictionary, and the final state
    int other[2], o = 0;
    for (int k = 0; k < 3; ++k)
        if (k != idx->cur) other[o++] = k;
    int final_cur = idx->cur;
    uint64_t final_n = idx->n, final_m = idx->m;
    for (size_t k = 0; k < p.blocks.size(); ++k) {
        final_cur = in_place ? idx->cur : other[k & 1];
        final_n += p.blocks[k].n_int;
        final_m += p.blocks[k].j1 - p.blocks[k].j0;
    }

    // Everything the device does for this append, after the input copies:
    // the packing of the reads, then the blocks.
    auto enqueue_pack = [&]() {
        const uint64_t tw = text_words(p.npos, idx->code_bits), term_words = (p.npos + 31) / 32;
        cudaMemsetAsync((uint32_t*)idx->text.p + tw, 0, kTextPadWords * 4, s);
        cudaMemsetAsync((uint32_t*)idx->term.p + term_words, 0, kTermPadWords * 4, s);
        cudaMemsetAsync(idx->err.p, 0, 4, s);
        // A byte outside the alphabet sets bit 0 of the error word; the blocks
        // still run (into scratch dictionaries) and the check at the end
        // refuses the result, which saves a round trip on every valid append.
        auto pack = [&](uint64_t w0, uint64_t w1) {
            if (idx->code_bits == 4)
                launch_pack_w(L, d_reads, d_offsets, m_new, p.npos, idx->alpha16, idx->sigma,
                              (uint32_t*)idx->text.p, (uint32_t*)idx->term.p, (uint32_t*)idx->err.p, w0, w1);
            else
                launch_pack(L, d_reads, d_offsets, m_new, p.npos, idx->alpha4, idx->sigma, (uint32_t*)idx->text.p,
                            (uint32_t*)idx->term.p, (uint32_t*)idx->err.p, w0, w1);
        };
        if (pipelined) {
            uint64_t b0 = 0, w0 = 0;
            for (size_t k = 0; k < p.blocks.size(); ++k) {
                if (chunk_bytes[k] > b0)
                    cudaMemcpyAsync((uint8_t*)idx->reads.p + b0, h_reads + b0, chunk_bytes[k] - b0,
                                    cudaMemcpyHostToDevice, s);
                pack(w0, chunk_words[k]);
                cudaEventRecord(idx->ev_packed[k], s);
                b0 = std::max(b0, chunk_bytes[k]);
                w0 = std::max(w0, chunk_words[k]);
            }
        } else {
            pack(0, ~0ull);
        }
    };
    auto enqueue_blocks = [&]() {
        int src = idx->cur;
        uint64_t n_ext = idx->n, m_ext = idx->m;
        cudaEventRecord(idx->ev_fork, s);  // the sorts read the packed text
        if (!pipelined) cudaStreamWaitEvent(idx->side, idx->ev_fork, 0);
        const size_t nb = p.blocks.size();
        for (size_t q = 0; q < nb; ++q) {
            // prepending runs the blocks last to first, so each one's reads go
            // before those of the blocks already inserted
            const size_t k = p.prepend ? nb - 1 - q : q;
            const BlockPlan& bp = p.blocks[k];
            const int dst = in_place ? src : other[q & 1];
            cudaEvent_t packed = pipelined ? idx->ev_packed[k] : nullptr;
            if (p.idx64)
                run_block<unsigned long long>(idx, bp, d_offsets, idx->dict[src], idx->dict[dst], n_ext, m_ext,
                                              p.slots, k, q, p.prepend, packed, in_place);
            else
                run_block<uint32_t>(idx, bp, d_offsets, idx->dict[src], idx->dict[dst], n_ext, m_ext, p.slots, k, q,
                                    p.prepend, packed, in_place);
            n_ext += bp.n_int;
            m_ext += bp.j1 - bp.j0;
            src = dst;
        }
        cudaEventRecord(idx->ev_join, idx->side);
        cudaStreamWaitEvent(s, idx->ev_join, 0);
        cudaMemcpyAsync(idx->h_err, idx->err.p, 4, cudaMemcpyDeviceToHost, s);
    };
    auto enqueue = [&]() {
        enqueue_pack();
        enqueue_blocks();
    };

    const Launcher::GraphLog* replayed = nullptr;
    if (in_place) {
        // the one dictionary is about to be rewritten: refuse a byte outside
        // the alphabet first, so such an append leaves the index unchanged
        enqueue_pack();
        cudaMemcpyAsync(idx->h_err, idx->err.p, 4, cudaMemcpyDeviceToHost, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return SBWT_EDEVICE;
        if (*idx->h_err & 1u) return SBWT_EINVAL;
        if (*idx->h_err) return SBWT_EDEVICE;
        enqueue_blocks();
    } else if (graph) {
        // The batched form: the append is captured into a graph; the graph
        // instantiated for the same pipeline shape (the same kernels in the
        // same order) is updated in place with this append's sizes, buffers
        // and index state, and the whole append is launched as one unit.  A
        // shape seen for the first time is instantiated (at most 8 kept).
        sbwt_index::GraphEntry g;
        cudaGraph_t graph = nullptr;
        L.capture = &g.log;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue();
            e = cudaStreamEndCapture(s, &graph);
        }
        L.capture = nullptr;
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            L.recycle(g.log);
            cudaGetLastError();
            return SBWT_EDEVICE;
        }
        auto it = std::find_if(idx->graphs.begin(), idx->graphs.end(), [&](const sbwt_index::GraphEntry& x) {
            return x.log.launches == g.log.launches && x.log.timed.size() == g.log.timed.size();
        });
        if (it != idx->graphs.end()) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(it->exec, graph, &info) == cudaSuccess) {
                L.recycle(it->log);
                it->log = std::move(g.log);
                L.add_host("host:graph_update", 0.0);
            } else {  // not updatable after all: instantiate this shape anew
                cudaGetLastError();
                cudaGraphExecDestroy(it->exec);
                L.recycle(it->log);
                idx->graphs.erase(it);
                it = idx->graphs.end();
            }
        }
        if (it == idx->graphs.end()) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                L.recycle(g.log);
                cudaGetLastError();
                return SBWT_EDEVICE;
            }
            if (idx->graphs.size() >= 8) {
                cudaGraphExecDestroy(idx->graphs.front().exec);
                L.recycle(idx->graphs.front().log);
                idx->graphs.erase(idx->graphs.begin());
            }
            idx->graphs.push_back(std::move(g));
            it = idx->graphs.end() - 1;
            L.add_host("host:graph_instantiate", 0.0);
        }
        cudaGraphDestroy(graph);
        if (cudaGraphLaunch(it->exec, s) != cudaSuccess) return SBWT_EDEVICE;
        L.add_host("host:graph_launch", 0.0);
        replayed = &it->log;
    } else {
        enqueue();
    }
    const auto t_launch = std::chrono::steady_clock::now();
    L.add_host("host:launch", std::chrono::duration<double, std::milli>(t_launch - t_plan).count());
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        if (in_place) idx->broken = true;
        return SBWT_EDEVICE;
    }
    L.add_host("host:wait",
               std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_launch).count());
    if (L.settle_units() != cudaSuccess) return SBWT_EDEVICE;
    if (replayed && L.account_replay(*replayed) != cudaSuccess) return SBWT_EDEVICE;
    if (*idx->h_err & 1u) return SBWT_EINVAL;  // a byte outside the alphabet; the index is unchanged
    if (*idx->h_err) {  // a kernel caught an inconsistent index: keep the old one (rewritten in place: broken)
        if (in_place) idx->broken = true;
        return SBWT_EDEVICE;
    }
    idx->cur = final_cur;
    idx->n = final_n;
    idx->m = final_m;
    idx->last_valid = !p.blocks.empty();
    idx->last_n = p.blocks.empty() ? 0 : (p.prepend ? p.blocks.front().n_int : p.blocks.back().n_int);
    idx->last_idx64 = p.idx64;
    idx->last_sa = (p.blocks.size() & 1) ? idx->sa.p : idx->sa2.p;
    return SBWT_OK;
}

int parse_alphabet(const char* alphabet, sbwt_index* idx) {
    if (!alphabet) return SBWT_EINVAL;
    size_t len = strlen(alphabet);
    if (len < 1 || len > 16) return SBWT_EINVAL;
    for (size_t a = 0; a < len; ++a) {
        uint8_t c = (uint8_t)alphabet[a];
        if (c == '$') return SBWT_EINVAL;
        if (a > 0 && c <= (uint8_t)alphabet[a - 1]) return SBWT_EINVAL;
        idx->alphabet[a] = c;
    }
    idx->sigma = (int)len;
    idx->code_bits = len > 4 ? 4 : 2;
    idx->alpha4 = 0;
    for (int a = 0; a < 4; ++a) idx->alpha4 |= (uint32_t)idx->alphabet[a < (int)len ? a : 0] << (8 * a);
    for (int a = 0; a < 16; ++a) idx->alpha16.a[a] = idx->alphabet[a < (int)len ? a : 0];
    return SBWT_OK;
}

// ---------------------------------------------------------------------------
// Index files (sbwt_save / sbwt_load): a header, the committed dictionary
// (occurrence blocks, superblock counters, C[]), then a 64-bit FNV-1a
// checksum of everything before it.
// ---------------------------------------------------------------------------
constexpr char kFileMagic[8] = {'S', 'B', 'W', 'T', 'I', 'D', 'X', '1'};
// Version 3: up to 4 symbols, the bit-plane dictionary with the occurrence
// sampling in the header.  Version 2: 5 to 16 symbols, the 4-bit dictionary;
// symbols 5.. in alphabet_hi.  Version 1 (read only): up to 4 symbols, 2-bit
// codes interleaved in 64-row blocks (converted to bit planes on load).
constexpr uint32_t kFileVersionPacked = 1;
constexpr uint32_t kFileVersionWide = 2;
constexpr uint32_t kFileVersion = 3;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t sigma;
    uint8_t alphabet[4];
    uint32_t index_bits;
    uint64_t n, m;
    uint64_t n_blocks, n_supers;  // array lengths: dict_blocks(n, k), the superblocks of the layout
    uint8_t alphabet_hi[12];
    uint32_t occ_sampling;  // rows per occurrence block (version 3; 0 reads as 64)
    uint8_t reserved[16];
};
static_assert(sizeof(FileHeader) == 88, "fixed header layout");

struct Fnv1a {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const uint8_t* b = static_cast<const uint8_t*>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

// Random 32-byte sector reads (from mapped pinned host memory or from HBM),
// the access of ComputeRanks and rank queries to a dictionary that is not in
// L2.  Each thread reads kLinkReads sectors at pseudo-random offsets;
// `sectors` is a power of two.
constexpr int kLinkReads = 64;
constexpr int kLinkBatch = 8;
__global__ void __launch_bounds__(256) link_random_read_kernel(const ulonglong2* __restrict__ host, uint64_t sectors,
                                                               unsigned long long* __restrict__ sink) {
    uint64_t x = (uint64_t)blockIdx.x * 256 + threadIdx.x + 1;
    unsigned long long acc = 0;
    // kLinkBatch independent sectors in flight per thread: all addresses,
    // then all loads, then the sums
    for (int r = 0; r < kLinkReads; r += kLinkBatch) {
        uint64_t sct[kLinkBatch];
#pragma unroll
        for (int u = 0; u < kLinkBatch; ++u) {
            x = x * 6364136223846793005ull + 1442695040888963407ull;  // LCG step (Knuth's MMIX constants)
            sct[u] = (x >> 17) & (sectors - 1);
        }
        ulonglong2 a[kLinkBatch], b[kLinkBatch];
#pragma unroll
        for (int u = 0; u < kLinkBatch; ++u) {
            a[u] = host[2 * sct[u]];
            b[u] = host[2 * sct[u] + 1];
        }
#pragma unroll
        for (int u = 0; u < kLinkBatch; ++u) acc += a[u].x ^ a[u].y ^ b[u].x ^ b[u].y;
    }
    if (acc == 0x5bd1e995ull) sink[0] = acc;  // keeps the loads
}

}  // namespace

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------
namespace sbwt {

cudaEvent_t Launcher::take_event() {
    if (!free_events_.empty()) {
        cudaEvent_t e = free_events_.back();
        free_events_.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int Launcher::stat_index(const char* name) {
    for (size_t i = 0; i < stats.size(); ++i)
        if (stats[i].name == name) return (int)i;
    KernelStat k;
    k.name = name;
    stats.push_back(k);
    return (int)stats.size() - 1;
}

int Launcher::before(const char* name, double fixed, double per_unit, const uint32_t* d_units) {
    const int s = stat_index(name);
    const bool timed = profiling && (only.empty() || only == name);
    if (capture) {
        capture->launches.push_back(s);
        if (!timed) return -1;
        Pending p{s, take_event(), take_event(), fixed, per_unit, d_units, false};
        cudaEventRecordWithFlags(p.a, stream, cudaEventRecordExternal);
        capture->timed.push_back(p);
        return (int)capture->timed.size() - 1;
    }
    stats[s].launches++;
    if (!timed) return -1;
    Pending p{s, take_event(), take_event(), fixed, per_unit, d_units, d_units == nullptr};
    cudaEventRecord(p.a, stream);
    pending_.push_back(p);
    return (int)pending_.size() - 1;
}

void Launcher::after(int token) {
    if (token < 0) return;
    if (capture)
        cudaEventRecordWithFlags(capture->timed[token].b, stream, cudaEventRecordExternal);
    else
        cudaEventRecord(pending_[token].b, stream);
}

cudaError_t Launcher::account_replay(const GraphLog& g) {
    for (int s : g.launches) stats[s].launches++;
    if (g.timed.empty()) return cudaSuccess;
    std::vector<uint32_t> log(unit_log_len);
    cudaError_t err = cudaSuccess;
    if (unit_log_len) err = cudaMemcpy(log.data(), unit_log, unit_log_len * 4, cudaMemcpyDeviceToHost);
    for (const Pending& p : g.timed) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) stats[p.stat].ms += ms;
        uint32_t u = 0;
        if (p.units && p.units >= unit_log && p.units < unit_log + unit_log_len) u = log[p.units - unit_log];
        stats[p.stat].bytes += p.fixed + p.per_unit * u;
    }
    cudaGetLastError();
    return err;
}

cudaError_t Launcher::settle_units() {
    bool any = false;
    for (const Pending& p : pending_) any |= !p.settled;
    if (!any) return cudaSuccess;
    std::vector<uint32_t> log(unit_log_len);
    cudaError_t err = cudaSuccess;
    if (unit_log_len) err = cudaMemcpy(log.data(), unit_log, unit_log_len * 4, cudaMemcpyDeviceToHost);
    for (Pending& p : pending_) {
        if (p.settled) continue;
        uint32_t u = 0;
        if (p.units >= unit_log && p.units < unit_log + unit_log_len)
            u = log[p.units - unit_log];
        else
            cudaMemcpy(&u, p.units, 4, cudaMemcpyDeviceToHost);
        p.fixed += p.per_unit * u;
        p.per_unit = 0;
        p.settled = true;
    }
    return err;
}

cudaError_t Launcher::resolve() {
    cudaError_t err = settle_units();
    for (const Pending& p : pending_) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) stats[p.stat].ms += ms;
        stats[p.stat].bytes += p.fixed;
        free_events_.push_back(p.a);
        free_events_.push_back(p.b);
    }
    pending_.clear();
    cudaGetLastError();
    return err;
}

void Launcher::recycle(GraphLog& g) {
    for (const Pending& p : g.timed) {
        free_events_.push_back(p.a);
        free_events_.push_back(p.b);
    }
    g.timed.clear();
    g.launches.clear();
}

void Launcher::add_host(const char* name, double ms) {
    const int s = stat_index(name);
    stats[s].launches++;
    stats[s].ms += ms;
}

void Launcher::reset() {
    for (KernelStat& k : stats) {
        k.launches = 0;
        k.ms = 0;
        k.bytes = 0;
    }
}

void Launcher::release() {
    for (const Pending& p : pending_) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    pending_.clear();
    for (cudaEvent_t e : free_events_) cudaEventDestroy(e);
    free_events_.clear();
}

}  // namespace sbwt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

// Appends of at least this many reads are validated and planned on the
// device (two small kernels and one copy of the block table back) instead of
// in two host loops over the offsets.
constexpr uint64_t kDevicePlanMin = 1 << 16;

// Validates device-resident offsets and plans the blocks on the device; the
// host offsets (h_off, when the caller has them) serve the rare plan with
// more blocks than the table holds.
int plan_on_device(sbwt_index* idx, const uint64_t* d_offsets, const uint64_t* h_off, uint64_t m, Plan& p) {
    if (int rc = reserve(idx, {{&idx->plan, kPlanCap * sizeof(PlanBlock) + sizeof(PlanSummary)}})) return rc;
    PlanBlock* d_table = (PlanBlock*)idx->plan.p;
    PlanSummary* d_sum = (PlanSummary*)((char*)idx->plan.p + kPlanCap * sizeof(PlanBlock));
    launch_plan(idx->L, d_offsets, m, idx->M, kMaxBlock, d_table, kPlanCap, d_sum);
    cudaMemcpyAsync(idx->h_summary, d_sum, sizeof(PlanSummary), cudaMemcpyDeviceToHost, idx->stream);
    cudaMemcpyAsync(idx->h_plan, d_table, kPlanCap * sizeof(PlanBlock), cudaMemcpyDeviceToHost, idx->stream);
    if (cudaStreamSynchronize(idx->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SBWT_EDEVICE;
    const PlanSummary sum = *idx->h_summary;
    if (sum.bad) return SBWT_EINVAL;
    if (sum.blocks <= kPlanCap) {
        p.npos = sum.npos;
        p.nbytes = sum.npos - m;
        for (unsigned k = 0; k < sum.blocks; ++k) {
            const PlanBlock& b = idx->h_plan[k];
            p.blocks.push_back(BlockPlan{b.j0, b.j1, b.n_int, b.base, sum.max_len});
        }
        return SBWT_OK;
    }
    // more blocks than the table holds: plan on the host
    if (!h_off) {
        if (m + 1 > idx->h_offsets_cap) {
            if (idx->h_offsets) cudaFreeHost(idx->h_offsets);
            idx->h_offsets = nullptr;
            idx->h_offsets_cap = 0;
            if (cudaMallocHost(&idx->h_offsets, (m + 1) * 8) != cudaSuccess) return SBWT_ENOMEM;
            idx->h_offsets_cap = m + 1;
        }
        if (cudaMemcpyAsync(idx->h_offsets, d_offsets, (m + 1) * 8, cudaMemcpyDeviceToHost, idx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(idx->stream) != cudaSuccess)
            return SBWT_EDEVICE;
        h_off = idx->h_offsets;
    }
    p = host_plan(h_off, m, idx->M);
    return SBWT_OK;
}

}  // namespace

extern "C" {

const char* sbwt_strerror(int code) {
    switch (code) {
        case SBWT_OK: return "ok";
        case SBWT_EINVAL: return "invalid argument or input";
        case SBWT_ENOMEM: return "out of device memory or over the HBM budget";
        case SBWT_ERANGE: return "output buffer too small";
        case SBWT_EDEVICE: return "CUDA device error";
        case SBWT_ENOTSUP: return "not supported";
        case SBWT_EBUSY: return "the index is serving requests";
        case SBWT_ETIMEDOUT: return "not done yet";
        case SBWT_EIO: return "cannot read or write the file";
        default: return "unknown error";
    }
}

int sbwt_create_ex(const char* alphabet, size_t hbm_budget_bytes, const sbwt_options* opt, sbwt_index** out) {
    if (!out) return SBWT_EINVAL;
    *out = nullptr;
    sbwt_index* idx = new (std::nothrow) sbwt_index();
    if (!idx) return SBWT_ENOMEM;
    if (parse_alphabet(alphabet, idx)) {
        delete idx;
        return SBWT_EINVAL;
    }
    idx->budget = hbm_budget_bytes;
    if (opt) {
        bool bad = opt->index_bits != 0 && opt->index_bits != 32 && opt->index_bits != 64;
        bad |= opt->block_suffixes > kMaxBlock;
        bad |= opt->host_tier > 3;
        bad |= opt->occ_sampling != 0 && opt->occ_sampling != 64 && opt->occ_sampling != 128 &&
               opt->occ_sampling != 256;
        for (uint32_t r : opt->reserved) bad |= r != 0;
        if (bad) {
            delete idx;
            return SBWT_EINVAL;
        }
        if (idx->code_bits == 4 && opt->occ_sampling > 64) {  // the 4-bit dictionary samples every 64 rows only
            delete idx;
            return SBWT_ENOTSUP;
        }
        if (opt->occ_sampling) idx->occ_k = (int)(opt->occ_sampling / 64);
        idx->index_bits = opt->index_bits;
        if (opt->block_suffixes) idx->M = opt->block_suffixes;
        idx->stream = (cudaStream_t)opt->stream;
        idx->device = opt->device;
        idx->host_tier_allowed = opt->host_tier != 2;
        idx->host_tier_forced = opt->host_tier == 3;
    }
    *out = idx;
    return SBWT_OK;
}

int sbwt_create(const char* alphabet, size_t hbm_budget_bytes, sbwt_index** out) {
    return sbwt_create_ex(alphabet, hbm_budget_bytes, nullptr, out);
}

int sbwt_append(sbwt_index* idx, const uint8_t* reads, const uint64_t* offsets, uint64_t m) {
    if (!idx || !offsets) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    const auto t0 = std::chrono::steady_clock::now();
    if (m < kDevicePlanMin) {
        if (validate_offsets(offsets, m)) return SBWT_EINVAL;
        if (m == 0) return SBWT_OK;
        if (offsets[m] > 0 && !reads) return SBWT_EINVAL;
        return append_impl(idx, nullptr, nullptr, offsets, m, true, reads, host_plan(offsets, m, idx->M), t0);
    }
    // a large append: the offsets go to the device first, which validates
    // them and plans the blocks
    if (offsets[0] != 0) return SBWT_EINVAL;
    if (int rc = device_init(idx)) return rc;
    if (int rc = reserve(idx, {{&idx->offsets, (size_t)(m + 1) * 8}})) return rc;
    if (cudaMemcpyAsync(idx->offsets.p, offsets, (m + 1) * 8, cudaMemcpyHostToDevice, idx->stream) != cudaSuccess)
        return SBWT_EDEVICE;
    Plan p;
    if (int rc = plan_on_device(idx, (const uint64_t*)idx->offsets.p, offsets, m, p)) return rc;
    if (p.nbytes > 0 && !reads) return SBWT_EINVAL;
    return append_impl(idx, nullptr, nullptr, offsets, m, true, reads, p, t0);
}

int sbwt_prepend(sbwt_index* idx, const uint8_t* reads, const uint64_t* offsets, uint64_t m) {
    if (!idx || !offsets) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    const auto t0 = std::chrono::steady_clock::now();
    if (validate_offsets(offsets, m)) return SBWT_EINVAL;
    if (m == 0) return SBWT_OK;
    if (offsets[m] > 0 && !reads) return SBWT_EINVAL;
    Plan p = host_plan(offsets, m, idx->M);
    p.prepend = true;
    return append_impl(idx, nullptr, nullptr, offsets, m, true, reads, p, t0);
}

int sbwt_append_device(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m) {
    if (!idx || !d_offsets) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = device_init(idx)) return rc;
    if (m == 0) return SBWT_OK;
    // validate and plan on the device; only the block table comes back
    Plan p;
    if (int rc = plan_on_device(idx, d_offsets, nullptr, m, p)) return rc;
    if (p.nbytes > 0 && !d_reads) return SBWT_EINVAL;
    return append_impl(idx, d_reads, d_offsets, nullptr, m, false, nullptr, p, t0);
}

int sbwt_get_bwt(sbwt_index* idx, uint8_t* out, uint64_t cap, uint64_t* n_out) {
    if (!idx || !n_out) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    *n_out = idx->n;
    if (cap < idx->n) return SBWT_ERANGE;
    if (idx->n == 0) return SBWT_OK;
    if (!out) return SBWT_EINVAL;
    if (int rc = device_init(idx)) return rc;
    if (reserve(idx, {{&idx->out_bytes, (size_t)idx->n}}) != SBWT_OK) {
        // over the HBM budget: stage B in pinned host memory instead
        if (!idx->host_tier_allowed || grow(idx->out_bytes, idx->n, true) != SBWT_OK) return SBWT_ENOMEM;
    }
    // unpack in chunks on the index stream while the side stream copies the
    // chunks already unpacked
    constexpr uint64_t kChunkRows = 1ull << 24;
    const cudaStream_t s = idx->stream;
    const void* blocks = idx->dict[idx->cur].blocks.p;
    uint8_t* staged = (uint8_t*)idx->out_bytes.p;
    int e = 0;
    for (uint64_t r0 = 0; r0 < idx->n; r0 += kChunkRows, e ^= 1) {
        const uint64_t r1 = std::min(idx->n, r0 + kChunkRows);
        launch_unpack(idx->L, blocks, r0, r1, idx->alpha16, staged, idx->code_bits, idx->occ_k);
        cudaEventRecord(idx->ev_sorted[e], s);
        cudaStreamWaitEvent(idx->side, idx->ev_sorted[e], 0);
        cudaMemcpyAsync(out + r0, staged + r0, r1 - r0, cudaMemcpyDeviceToHost, idx->side);
    }
    cudaEventRecord(idx->ev_join, idx->side);
    cudaStreamWaitEvent(s, idx->ev_join, 0);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SBWT_EDEVICE;
    if (idx->out_bytes.host) free_buf(idx->out_bytes);  // the host tier keeps only its dictionary in host memory
    return SBWT_OK;
}

int sbwt_rank_batch(sbwt_index* idx, const uint8_t* cs, const uint64_t* ks, uint64_t q, uint64_t* out) {
    if (!idx || (q && (!cs || !ks || !out))) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    std::vector<uint8_t> codes(q);
    for (uint64_t i = 0; i < q; ++i) {
        if (ks[i] > idx->n) return SBWT_EINVAL;
        int code = -1;
        if (cs[i] == '$') code = (int)dict_codes(idx->code_bits);  // the terminator's query code
        for (int a = 0; a < idx->sigma; ++a)
            if (cs[i] == idx->alphabet[a]) code = a;
        if (code < 0) return SBWT_EINVAL;
        codes[i] = (uint8_t)code;
    }
    if (q == 0) return SBWT_OK;
    if (int rc = device_init(idx)) return rc;
    if (reserve(idx, {{&idx->q_codes, (size_t)q}, {&idx->q_ks, (size_t)q * 8}, {&idx->q_out, (size_t)q * 8}}) !=
        SBWT_OK) {
        // over the HBM budget: the query arrays go to pinned host memory
        if (!idx->host_tier_allowed || grow(idx->q_codes, q, true) || grow(idx->q_ks, q * 8, true) ||
            grow(idx->q_out, q * 8, true))
            return SBWT_ENOMEM;
    }
    cudaStream_t s = idx->stream;
    cudaMemcpyAsync(idx->q_codes.p, codes.data(), q, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(idx->q_ks.p, ks, q * 8, cudaMemcpyHostToDevice, s);
    const Dict& d = idx->dict[idx->cur];
    launch_rank_batch(idx->L, (const void*)d.blocks.p, (const unsigned long long*)d.super.p,
                      (const uint8_t*)idx->q_codes.p, (const unsigned long long*)idx->q_ks.p, q,
                      (unsigned long long*)idx->q_out.p, idx->code_bits, idx->occ_k);
    cudaMemcpyAsync(out, idx->q_out.p, q * 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

int sbwt_count(sbwt_index* idx, const uint8_t* patterns, const uint64_t* offsets, uint64_t q, uint64_t* counts) {
    if (!idx || (q && (!offsets || !counts))) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    if (q == 0) return SBWT_OK;
    if (offsets[0] != 0) return SBWT_EINVAL;
    for (uint64_t i = 0; i < q; ++i)
        if (offsets[i + 1] < offsets[i]) return SBWT_EINVAL;
    const uint64_t total = offsets[q];
    if (total && !patterns) return SBWT_EINVAL;
    if (int rc = device_init(idx)) return rc;
    if (reserve(idx, {{&idx->c_pats, (size_t)total + 1}, {&idx->c_offs, (size_t)(q + 1) * 8},
                      {&idx->q_out, (size_t)q * 8}}) != SBWT_OK) {
        if (!idx->host_tier_allowed || grow(idx->c_pats, total + 1, true) || grow(idx->c_offs, (q + 1) * 8, true) ||
            grow(idx->q_out, q * 8, true))
            return SBWT_ENOMEM;
    }
    cudaStream_t s = idx->stream;
    if (total) cudaMemcpyAsync(idx->c_pats.p, patterns, total, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(idx->c_offs.p, offsets, (q + 1) * 8, cudaMemcpyHostToDevice, s);
    const Dict& d = idx->dict[idx->cur];
    launch_count(idx->L, (const void*)d.blocks.p, (const unsigned long long*)d.super.p,
                 (const unsigned long long*)d.C.p, idx->n, idx->alpha16, idx->sigma, (const uint8_t*)idx->c_pats.p,
                 (const uint64_t*)idx->c_offs.p, q, total, (unsigned long long*)idx->q_out.p, idx->code_bits, idx->occ_k);
    cudaMemcpyAsync(counts, idx->q_out.p, q * 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

int sbwt_rank(sbwt_index* idx, uint8_t c, uint64_t k, uint64_t* out) {
    if (!out) return SBWT_EINVAL;
    return sbwt_rank_batch(idx, &c, &k, 1, out);
}

int sbwt_memory(const sbwt_index* idx, uint64_t* hbm_bytes, uint64_t* host_bytes) {
    if (!idx) return SBWT_EINVAL;
    sbwt_index* mut = const_cast<sbwt_index*>(idx);
    if (hbm_bytes) *hbm_bytes = mut->held_bytes(false);
    if (host_bytes) *host_bytes = mut->held_bytes(true);
    return SBWT_OK;
}

int sbwt_size(const sbwt_index* idx, uint64_t* n, uint64_t* m) {
    if (!idx) return SBWT_EINVAL;
    if (n) *n = idx->n;
    if (m) *m = idx->m;
    return SBWT_OK;
}

int sbwt_reset(sbwt_index* idx) {
    if (!idx) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    idx->n = idx->m = 0;
    idx->broken = false;
    idx->last_valid = false;
    if (!idx->dev_ready) return SBWT_OK;
    if (set_device(idx)) return SBWT_EDEVICE;
    Dict& d = idx->dict[idx->cur];
    zero_async(d.blocks, dict_block_bytes(idx->code_bits, idx->occ_k), idx->stream);
    zero_async(d.super, 8 * dict_codes(idx->code_bits), idx->stream);
    zero_async(d.C, 8 * dict_codes(idx->code_bits), idx->stream);
    if (cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

int sbwt_save(sbwt_index* idx, const char* path) {
    if (!idx || !path) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->broken) return SBWT_EDEVICE;  // an in-place append failed: reset first
    const int cb = idx->code_bits, k = idx->occ_k;
    const size_t bb = dict_block_bytes(cb, k), codes = dict_codes(cb);
    FileHeader h = {};
    memcpy(h.magic, kFileMagic, sizeof(h.magic));
    h.version = cb == 4 ? kFileVersionWide : kFileVersion;
    h.sigma = (uint32_t)idx->sigma;
    memcpy(h.alphabet, idx->alphabet, 4);
    memcpy(h.alphabet_hi, idx->alphabet + 4, 12);
    h.index_bits = idx->index_bits;
    h.occ_sampling = 64u * (uint32_t)k;
    h.n = idx->n;
    h.m = idx->m;
    h.n_blocks = dict_blocks(idx->n, k);
    h.n_supers = dict_supers_of(idx->n, cb);
    std::vector<uint8_t> blocks(h.n_blocks * bb, 0);
    std::vector<unsigned long long> super(codes * h.n_supers, 0ull), C(codes, 0ull);
    if (idx->dev_ready) {  // else the index is empty: all zero
        if (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
        const Dict& d = idx->dict[idx->cur];
        if (cudaMemcpy(blocks.data(), d.blocks.p, blocks.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(super.data(), d.super.p, super.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(C.data(), d.C.p, C.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return SBWT_EDEVICE;
        }
    }
    Fnv1a sum;
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return SBWT_EIO;
    auto put = [&](const void* p, size_t n) {
        sum.add(p, n);
        return fwrite(p, 1, n, out.f) == n;
    };
    bool ok = put(&h, sizeof(h)) && put(blocks.data(), blocks.size()) && put(super.data(), super.size() * 8) &&
              put(C.data(), C.size() * 8);
    const uint64_t digest = sum.h;
    ok = ok && fwrite(&digest, 1, 8, out.f) == 8;
    ok = fclose(out.f) == 0 && ok;
    out.f = nullptr;
    return ok ? SBWT_OK : SBWT_EIO;
}

int sbwt_load(const char* path, size_t hbm_budget_bytes, const sbwt_options* opt, sbwt_index** out) {
    if (!out) return SBWT_EINVAL;
    *out = nullptr;
    if (!path) return SBWT_EINVAL;
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return SBWT_EIO;
    FileHeader h;
    if (fread(&h, 1, sizeof(h), in.f) != sizeof(h)) return SBWT_EIO;
    if (memcmp(h.magic, kFileMagic, sizeof(h.magic)) != 0) return SBWT_EINVAL;
    const bool wide = h.version == kFileVersionWide, packed = h.version == kFileVersionPacked;
    if (h.version != kFileVersion && !wide && !packed) return SBWT_EINVAL;
    const int cb = wide ? 4 : 2;
    const uint32_t sampling = h.version == kFileVersion ? (h.occ_sampling ? h.occ_sampling : 64u) : 64u;
    if (sampling != 64 && sampling != 128 && sampling != 256) return SBWT_EINVAL;
    const int k = (int)(sampling / 64);
    if (h.sigma < 1 || h.sigma > (wide ? 16u : 4u) || (wide && h.sigma <= 4) ||
        (h.index_bits != 0 && h.index_bits != 32 && h.index_bits != 64) || h.n_blocks != dict_blocks(h.n, k) ||
        h.n_supers != dict_supers_of(h.n, cb) || h.m > h.n)
        return SBWT_EINVAL;
    const size_t bb = dict_block_bytes(cb, k), codes = dict_codes(cb);
    // the arrays must be exactly what the rest of the file holds
    if (fseek(in.f, 0, SEEK_END) != 0) return SBWT_EIO;
    const long size = ftell(in.f);
    const uint64_t want = sizeof(h) + h.n_blocks * bb + h.n_supers * codes * 8 + codes * 8 + 8;
    if (size < 0 || (uint64_t)size != want) return SBWT_EINVAL;
    if (fseek(in.f, (long)sizeof(h), SEEK_SET) != 0) return SBWT_EIO;
    std::vector<uint8_t> blocks(h.n_blocks * bb);
    std::vector<unsigned long long> super(codes * h.n_supers), C(codes);
    uint64_t digest = 0;
    if (fread(blocks.data(), 1, blocks.size(), in.f) != blocks.size() ||
        fread(super.data(), 1, super.size() * 8, in.f) != super.size() * 8 ||
        fread(C.data(), 1, C.size() * 8, in.f) != C.size() * 8 || fread(&digest, 1, 8, in.f) != 8)
        return SBWT_EIO;
    Fnv1a sum;
    sum.add(&h, sizeof(h));
    sum.add(blocks.data(), blocks.size());
    sum.add(super.data(), super.size() * 8);
    sum.add(C.data(), C.size() * 8);
    if (sum.h != digest) return SBWT_EINVAL;
    if (packed) {
        // version 1 blocks: two words of 2-bit codes (row q at bits 2 (q & 31)
        // of word q >> 5), the terminator mask and the counts; make them
        // bit planes
        unsigned long long* w = reinterpret_cast<unsigned long long*>(blocks.data());
        for (uint64_t b = 0; b < h.n_blocks; ++b, w += 4) {
            unsigned long long lo = 0, hi = 0;
            for (int q = 0; q < 64; ++q) {
                const unsigned long long c = (w[q >> 5] >> (2 * (q & 31))) & 3ull;
                lo |= (c & 1ull) << q;
                hi |= (c >> 1) << q;
            }
            w[0] = lo;
            w[1] = hi;
        }
    }

    char alpha[17] = {0};
    memcpy(alpha, h.alphabet, std::min<uint32_t>(h.sigma, 4));
    if (h.sigma > 4) memcpy(alpha + 4, h.alphabet_hi, h.sigma - 4);
    sbwt_options o = {};
    if (opt) o = *opt;
    if (o.index_bits == 0) o.index_bits = h.index_bits;
    if (o.occ_sampling != 0 && o.occ_sampling != sampling) return SBWT_EINVAL;  // the file's layout decides
    o.occ_sampling = sampling;
    if (h.n >= 0xFFFFFFFFull && o.index_bits == 32) return SBWT_EINVAL;
    sbwt_index* idx = nullptr;
    if (int rc = sbwt_create_ex(alpha, hbm_budget_bytes, &o, &idx)) return rc;
    auto fail = [&](int rc) {
        sbwt_destroy(idx);
        return rc;
    };
    if (int rc = device_init(idx)) return fail(rc);
    Dict& d = idx->dict[idx->cur];
    if (int rc = reserve(idx, {{&d.blocks, blocks.size(), true}, {&d.super, super.size() * 8, true},
                               {&d.C, C.size() * 8, true}}))
        return fail(rc);
    if (cudaMemcpy(d.blocks.p, blocks.data(), blocks.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.super.p, super.data(), super.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.C.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(SBWT_EDEVICE);
    }
    idx->n = h.n;
    idx->m = h.m;
    *out = idx;
    return SBWT_OK;
}

void sbwt_destroy(sbwt_index* idx) {
    if (!idx) return;
    if (idx->server) sbwt_serve_stop(idx);
    if (idx->dev_ready) {
        set_device(idx);
        cudaStreamSynchronize(idx->stream);
        drop_graphs(idx);
        idx->L.release();
        for (DevBuf* b : idx->all_bufs()) free_buf(*b);
        if (idx->h_err) cudaFreeHost(idx->h_err);
        if (idx->h_offsets) cudaFreeHost(idx->h_offsets);
        if (idx->h_plan) cudaFreeHost(idx->h_plan);
        if (idx->h_summary) cudaFreeHost(idx->h_summary);
        if (idx->side) {
            cudaStreamSynchronize(idx->side);
            cudaStreamDestroy(idx->side);
        }
        for (cudaEvent_t e : {idx->ev_fork, idx->ev_join, idx->ev_sorted[0], idx->ev_sorted[1],
                              idx->ev_consumed[0], idx->ev_consumed[1]})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : idx->ev_packed)
            if (e) cudaEventDestroy(e);
        if (idx->own_stream) cudaStreamDestroy(idx->stream);
    }
    delete idx;
}

int sbwt_get_stream(sbwt_index* idx, void** stream) {
    if (!idx || !stream) return SBWT_EINVAL;
    if (int rc = device_init(idx)) return rc;
    *stream = (void*)idx->stream;
    return SBWT_OK;
}

int sbwt_set_capture(sbwt_index* idx, int on) {
    if (!idx) return SBWT_EINVAL;
    idx->capture = on != 0;
    idx->last_valid = false;
    return SBWT_OK;
}

int sbwt_get_stage(sbwt_index* idx, int stage, void* out, uint64_t cap, uint64_t* count_out) {
    if (!idx || !count_out) return SBWT_EINVAL;
    if (!idx->capture || !idx->last_valid) return SBWT_EINVAL;
    const uint64_t n = idx->last_n;
    *count_out = n;
    size_t elem = 0;
    const void* src = nullptr;
    switch (stage) {
        case SBWT_STAGE_SA: elem = 4; src = idx->last_sa; break;
        case SBWT_STAGE_BINT: elem = 1; src = idx->bint.p; break;
        case SBWT_STAGE_G: elem = 8; src = idx->g.p; break;
        case SBWT_STAGE_GSA: elem = 8; src = idx->gsa.p; break;
        default: return SBWT_EINVAL;
    }
    if (cap < n * elem) return SBWT_ERANGE;
    if (n == 0) return SBWT_OK;
    if (!out) return SBWT_EINVAL;
    if (set_device(idx)) return SBWT_EDEVICE;
    if ((stage == SBWT_STAGE_G || stage == SBWT_STAGE_GSA) && !idx->last_idx64) {
        std::vector<uint32_t> tmp(n);
        if (cudaMemcpy(tmp.data(), src, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SBWT_EDEVICE;
        uint64_t* o = (uint64_t*)out;
        for (uint64_t i = 0; i < n; ++i) o[i] = tmp[i];
        return SBWT_OK;
    }
    if (cudaMemcpy(out, src, n * elem, cudaMemcpyDeviceToHost) != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

}  // extern "C"

namespace {

// Occurrence sampling of an empty index: 64 k rows per block.  The committed
// dictionary (empty: one zero block) is laid out again for k.
int set_occ_k(sbwt_index* idx, int k) {
    if (k != 1 && k != 2 && k != 4) return SBWT_EINVAL;
    if (idx->code_bits == 4 && k != 1) return SBWT_ENOTSUP;
    if (idx->n != 0) return SBWT_EINVAL;
    if (k == idx->occ_k) return SBWT_OK;
    idx->occ_k = k;
    if (!idx->dev_ready) return SBWT_OK;
    if (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
    Dict& d = idx->dict[idx->cur];
    const size_t bb = dict_block_bytes(idx->code_bits, k);
    if (int rc = grow(d.blocks, bb, d.blocks.host)) return rc;
    zero_async(d.blocks, bb, idx->stream);
    if (cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
    return SBWT_OK;
}

// Builds the reads' BWT three times with the index's current settings and
// returns the faster of the last two in ms (the first sizes the buffers),
// -1 when it does not fit the HBM budget.  The index is left empty.
int time_build(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m, double* ms_out) {
    double t_min = -1;
    for (int rep = 0; rep < 3; ++rep) {
        if (int rc = sbwt_reset(idx)) return rc;
        const auto t0 = std::chrono::steady_clock::now();
        const int a = sbwt_append_device(idx, d_reads, d_offsets, m);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (a == SBWT_ENOMEM) {
            t_min = -1;
            break;
        }
        if (a != SBWT_OK) return a;
        if (rep > 0 && (t_min < 0 || ms < t_min)) t_min = ms;
    }
    *ms_out = t_min;
    return sbwt_reset(idx);
}

}  // namespace

extern "C" {

int sbwt_set_tile_shapes(sbwt_index* idx, const sbwt_tile_shapes* shapes) {
    if (!idx || !shapes) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    const uint32_t it = shapes->insert_threads, rs = shapes->rank_segment;
    if ((it != 0 && it != 256 && it != 512) || (rs != 0 && rs != 256 && rs != 512 && rs != 1024)) return SBWT_EINVAL;
    for (uint32_t r : shapes->reserved)
        if (r) return SBWT_EINVAL;
    if (idx->dev_ready && (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess)) return SBWT_EDEVICE;
    idx->tiles = *shapes;
    return SBWT_OK;
}

int sbwt_get_tile_shapes(const sbwt_index* idx, sbwt_tile_shapes* out) {
    if (!idx || !out) return SBWT_EINVAL;
    *out = idx->tiles;
    return SBWT_OK;
}

int sbwt_autotune_tile_shapes(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m,
                              const sbwt_tile_shapes* candidates, int ncand, sbwt_tile_shapes* best_out,
                              double* ms_out) {
    static const sbwt_tile_shapes kDefaults[] = {
        {0, 256, {0, 0}}, {256, 256, {0, 0}}, {512, 256, {0, 0}}, {0, 512, {0, 0}}, {0, 1024, {0, 0}}};
    if (!idx || !d_offsets || m == 0) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (!candidates) {
        candidates = kDefaults;
        ncand = (int)(sizeof(kDefaults) / sizeof(kDefaults[0]));
    }
    if (ncand <= 0) return SBWT_EINVAL;
    const sbwt_tile_shapes saved = idx->tiles;
    const bool saved_replay = idx->graph_replay;
    idx->graph_replay = false;
    int best = -1;
    double best_ms = 0;
    int rc = sbwt_reset(idx);
    for (int c = 0; c < ncand && rc == SBWT_OK; ++c) {
        if ((rc = sbwt_set_tile_shapes(idx, &candidates[c])) != SBWT_OK) break;
        double t = -1;
        rc = time_build(idx, d_reads, d_offsets, m, &t);
        if (ms_out) ms_out[c] = t;
        if (rc == SBWT_OK && t >= 0 && (best < 0 || t < best_ms)) {
            best = c;
            best_ms = t;
        }
    }
    idx->graph_replay = saved_replay;
    const int rr = sbwt_reset(idx);
    if (rc == SBWT_OK && best < 0) rc = SBWT_ENOMEM;
    if (rc != SBWT_OK) {
        idx->tiles = saved;
        return rc;
    }
    idx->tiles = candidates[best];
    if (best_out) *best_out = candidates[best];
    return rr;
}

int sbwt_autotune_block_suffixes(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m,
                                 const uint64_t* candidates, int ncand, uint64_t* best_out, double* ms_out) {
    uint32_t sampling = 64u * (uint32_t)(idx ? idx->occ_k : 1);
    return sbwt_autotune(idx, d_reads, d_offsets, m, candidates, ncand, &sampling, 1, best_out, nullptr, ms_out);
}

int sbwt_autotune(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m,
                  const uint64_t* block_suffixes, int n_block, const uint32_t* samplings, int n_sampling,
                  uint64_t* best_block_out, uint32_t* best_sampling_out, double* ms_out) {
    static const uint64_t kDefaultM[] = {1ull << 22, 1ull << 23, 1ull << 24, 1ull << 25, 1ull << 26, 1ull << 27};
    static const uint32_t kDefaultS[] = {64, 128, 256};
    if (!idx || !d_offsets || m == 0) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (!block_suffixes) {
        block_suffixes = kDefaultM;
        n_block = (int)(sizeof(kDefaultM) / sizeof(kDefaultM[0]));
    }
    if (!samplings) {
        samplings = kDefaultS;
        n_sampling = idx->code_bits == 4 ? 1 : 3;
    }
    if (n_block <= 0 || n_sampling <= 0) return SBWT_EINVAL;
    for (int c = 0; c < n_block; ++c)
        if (block_suffixes[c] == 0 || block_suffixes[c] > kMaxBlock) return SBWT_EINVAL;
    for (int c = 0; c < n_sampling; ++c) {
        if (samplings[c] != 64 && samplings[c] != 128 && samplings[c] != 256) return SBWT_EINVAL;
        if (idx->code_bits == 4 && samplings[c] != 64) return SBWT_ENOTSUP;
    }
    const uint64_t saved_M = idx->M;
    const int saved_k = idx->occ_k;
    const bool saved_replay = idx->graph_replay;
    idx->graph_replay = false;
    uint64_t best_M = 0;
    int best_k = 0;
    double best_ms = 0;
    int rc = sbwt_reset(idx);
    for (int si = 0; si < n_sampling && rc == SBWT_OK; ++si) {
        if ((rc = set_occ_k(idx, (int)(samplings[si] / 64))) != SBWT_OK) break;
        for (int c = 0; c < n_block && rc == SBWT_OK; ++c) {
            idx->M = block_suffixes[c];
            double t = -1;
            rc = time_build(idx, d_reads, d_offsets, m, &t);
            if (ms_out) ms_out[(size_t)si * n_block + c] = t;
            if (rc == SBWT_OK && t >= 0 && (best_M == 0 || t < best_ms)) {
                best_M = block_suffixes[c];
                best_k = idx->occ_k;
                best_ms = t;
            }
        }
    }
    idx->graph_replay = saved_replay;
    const int rr = sbwt_reset(idx);
    if (rc == SBWT_OK && best_M == 0) rc = SBWT_ENOMEM;
    if (rc != SBWT_OK) {
        idx->M = saved_M;
        set_occ_k(idx, saved_k);
        return rc;
    }
    idx->M = best_M;
    if (int r2 = set_occ_k(idx, best_k)) return r2;
    if (best_block_out) *best_block_out = best_M;
    if (best_sampling_out) *best_sampling_out = 64u * (uint32_t)best_k;
    return rr;
}

int sbwt_measure_bandwidth(sbwt_index* idx, sbwt_bandwidth* out) {
    if (!idx || !out) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (int rc = device_init(idx)) return rc;
    constexpr size_t kBytes = 256ull << 20, kHbmRandom = 1ull << 30;  // the HBM buffer is far beyond L2
    static_assert((kBytes & (kBytes - 1)) == 0 && (kHbmRandom & (kHbmRandom - 1)) == 0, "sector counts of 2^k");
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, kBytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaMalloc(&d, kHbmRandom) != cudaSuccess) {
        cudaGetLastError();
        if (h) cudaFreeHost(h);
        return SBWT_ENOMEM;
    }
    const cudaStream_t s = idx->stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    memset(h, 1, kBytes);
    auto best_of = [&](auto&& body) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(a, s);
            body();
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;  // the first run warms up
        }
        return (double)best;
    };
    const double t_h2d = best_of([&] { cudaMemcpyAsync(d, h, kBytes, cudaMemcpyHostToDevice, s); });
    const double t_d2h = best_of([&] { cudaMemcpyAsync(h, d, kBytes, cudaMemcpyDeviceToHost, s); });
    cudaMemsetAsync(d, 1, kHbmRandom, s);
    const unsigned grid = persistent_ctas((const void*)link_random_read_kernel, 256, 0);
    unsigned long long* sink = static_cast<unsigned long long*>(d);
    const double t_host = best_of([&] {
        link_random_read_kernel<<<grid, 256, 0, s>>>(static_cast<const ulonglong2*>(h), kBytes / 32, sink);
    });
    const double t_hbm = best_of([&] {
        link_random_read_kernel<<<grid, 256, 0, s>>>(static_cast<const ulonglong2*>(d), kHbmRandom / 32, sink);
    });
    const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(d);
    cudaFreeHost(h);
    if (!ok) return SBWT_EDEVICE;
    const double random_bytes = (double)grid * 256 * kLinkReads * 32;
    out->h2d_gbs = kBytes / (t_h2d * 1e6);
    out->d2h_gbs = kBytes / (t_d2h * 1e6);
    out->host_random_gbs = random_bytes / (t_host * 1e6);
    out->hbm_random_gbs = random_bytes / (t_hbm * 1e6);
    return SBWT_OK;
}

int sbwt_set_block_overlap(sbwt_index* idx, int on) {
    if (!idx) return SBWT_EINVAL;
    if (busy(idx)) return SBWT_EBUSY;
    if (idx->dev_ready && (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess)) return SBWT_EDEVICE;
    idx->overlap = on != 0;
    return SBWT_OK;
}

int sbwt_set_graph_replay(sbwt_index* idx, int on) {
    if (!idx) return SBWT_EINVAL;
    idx->graph_replay = on != 0;
    if (!idx->graph_replay && idx->dev_ready) {
        if (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
        drop_graphs(idx);
    }
    return SBWT_OK;
}

int sbwt_set_profiling(sbwt_index* idx, int on) {
    if (!idx) return SBWT_EINVAL;
    idx->L.profiling = on != 0;
    idx->L.only.clear();
    return SBWT_OK;
}

int sbwt_set_profiling_only(sbwt_index* idx, const char* kernel) {
    if (!idx || !kernel) return SBWT_EINVAL;
    idx->L.profiling = true;
    idx->L.only = kernel;
    return SBWT_OK;
}

int sbwt_get_kernel_stats(sbwt_index* idx, sbwt_kernel_stat* out, int cap, int* n_out) {
    if (!idx || !n_out) return SBWT_EINVAL;
    if (idx->dev_ready) {
        if (set_device(idx) || cudaStreamSynchronize(idx->stream) != cudaSuccess) return SBWT_EDEVICE;
        if (idx->L.resolve() != cudaSuccess) return SBWT_EDEVICE;
    }
    const auto& st = idx->L.stats;
    *n_out = (int)st.size();
    for (int i = 0; i < cap && i < (int)st.size(); ++i) {
        memset(&out[i], 0, sizeof(out[i]));
        strncpy(out[i].name, st[i].name.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = st[i].launches;
        out[i].ms = st[i].ms;
        out[i].bytes = st[i].bytes;
    }
    return SBWT_OK;
}

int sbwt_reset_kernel_stats(sbwt_index* idx) {
    if (!idx) return SBWT_EINVAL;
    idx->L.reset();
    return SBWT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Server hooks
// ---------------------------------------------------------------------------
void* sbwt_serve_attached(sbwt_index* idx) { return idx->server; }
void sbwt_serve_attach(sbwt_index* idx, void* server) { idx->server = server; }
void sbwt_serve_set_worker(sbwt_index* idx, std::thread::id id) { idx->server_worker = id; }
int sbwt_serve_append_device(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m) {
    return sbwt_append_device(idx, d_reads, d_offsets, m);
}
int sbwt_serve_append_host(sbwt_index* idx, const uint8_t* reads, const uint64_t* offsets, uint64_t m) {
    return sbwt_append(idx, reads, offsets, m);
}
