// serve.cu -- continuous batching of append requests (the served form).
//
// Requests (read batches) are queued by sbwt_submit.  A stager thread takes
// the requests waiting at that moment, in arrival order and up to a size
// cap, concatenates them into one pinned host buffer and starts its copy to
// the device on a copy stream; a worker thread appends each staged batch to
// the index (every step of Algorithm 1 on the GPU) as soon as the previous
// one is committed.  So requests that arrive while a batch runs are admitted
// into the next batch, whose host-to-device copy overlaps the running
// batch's kernels.  Read ids follow arrival order: the final index equals
// appending the requests one by one, in that order.  A request whose bytes
// are not in the alphabet fails alone: its batch is retried request by
// request.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sbwt.h"
#include "sbwt_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> reads;
    std::vector<uint64_t> offsets;  // m + 1
    uint64_t m = 0;
    Clock::time_point t_submit;
    bool done = false;
    int status = SBWT_OK;
    uint64_t first_id = 0;
    double latency_ms = 0;
};

struct Slot {
    uint8_t* h_reads = nullptr;
    uint64_t* h_off = nullptr;
    uint8_t* d_reads = nullptr;
    uint64_t* d_off = nullptr;
    size_t cap_bytes = 0, cap_reads = 0;
    cudaEvent_t ready = nullptr;
    bool busy = false;
};

struct Staged {
    std::vector<Request*> reqs;
    int slot = 0;
    uint64_t m = 0;
};

}  // namespace

struct sbwt_server {
    sbwt_index* idx = nullptr;
    uint64_t max_batch_bases = 0;
    int device = 0;
    cudaStream_t copy_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::deque<Staged> staged;
    std::map<uint64_t, Request*> tickets;
    uint64_t next_ticket = 1;
    Slot slots[2];
    bool stop = false;
    int in_stage = 0;     // batches taken from the queue, not yet handed to the worker
    int fatal = SBWT_OK;  // a device error ends serving
    std::thread stager, worker;
};

namespace {

int ensure_slot(Slot& s, size_t bytes, size_t reads) {
    if (bytes > s.cap_bytes) {
        if (s.h_reads) cudaFreeHost(s.h_reads);
        if (s.d_reads) cudaFree(s.d_reads);
        s.h_reads = nullptr;
        s.d_reads = nullptr;
        s.cap_bytes = 0;
        const size_t want = std::max<size_t>(bytes + bytes / 4, 1 << 20);
        if (cudaMallocHost(&s.h_reads, want) != cudaSuccess || cudaMalloc(&s.d_reads, want) != cudaSuccess) {
            cudaGetLastError();
            return SBWT_ENOMEM;
        }
        s.cap_bytes = want;
    }
    if (reads + 1 > s.cap_reads) {
        if (s.h_off) cudaFreeHost(s.h_off);
        if (s.d_off) cudaFree(s.d_off);
        s.h_off = nullptr;
        s.d_off = nullptr;
        s.cap_reads = 0;
        const size_t want = std::max<size_t>(reads + reads / 4 + 1, 1 << 16);
        if (cudaMallocHost(&s.h_off, want * 8) != cudaSuccess || cudaMalloc(&s.d_off, want * 8) != cudaSuccess) {
            cudaGetLastError();
            return SBWT_ENOMEM;
        }
        s.cap_reads = want;
    }
    return SBWT_OK;
}

void finish(sbwt_server* sv, Request* r, int status, uint64_t first_id) {
    r->status = status;
    r->first_id = first_id;
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    r->done = true;
}

void stager_loop(sbwt_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv.wait(lk, [&] {
            return sv->fatal || (sv->stop && sv->queue.empty()) ||
                   (!sv->queue.empty() && (!sv->slots[0].busy || !sv->slots[1].busy));
        });
        if ((sv->stop && sv->queue.empty()) || sv->fatal) return;
        const int si = !sv->slots[0].busy ? 0 : 1;
        // admit the requests waiting now, in arrival order, up to the cap
        Staged st;
        st.slot = si;
        uint64_t bytes = 0;
        while (!sv->queue.empty()) {
            Request* r = sv->queue.front();
            const uint64_t b = r->offsets[r->m];
            if (!st.reqs.empty() && sv->max_batch_bases && bytes + b > sv->max_batch_bases) break;
            st.reqs.push_back(r);
            sv->queue.pop_front();
            bytes += b;
            st.m += r->m;
        }
        Slot& s = sv->slots[si];
        s.busy = true;
        ++sv->in_stage;
        lk.unlock();
        int rc = ensure_slot(s, bytes, st.m);
        if (rc == SBWT_OK) {
            uint64_t w = 0, j = 0;
            s.h_off[0] = 0;
            for (Request* r : st.reqs) {
                if (r->offsets[r->m]) memcpy(s.h_reads + w, r->reads.data(), r->offsets[r->m]);
                for (uint64_t q = 0; q < r->m; ++q) s.h_off[j + q + 1] = w + r->offsets[q + 1];
                w += r->offsets[r->m];
                j += r->m;
            }
            if ((bytes && cudaMemcpyAsync(s.d_reads, s.h_reads, bytes, cudaMemcpyHostToDevice, sv->copy_stream) !=
                              cudaSuccess) ||
                cudaMemcpyAsync(s.d_off, s.h_off, (st.m + 1) * 8, cudaMemcpyHostToDevice, sv->copy_stream) !=
                    cudaSuccess ||
                cudaEventRecord(s.ready, sv->copy_stream) != cudaSuccess)
                rc = SBWT_EDEVICE;
        }
        lk.lock();
        --sv->in_stage;
        if (rc != SBWT_OK) {
            for (Request* r : st.reqs) finish(sv, r, rc, 0);
            s.busy = false;
            sv->cv.notify_all();
            continue;
        }
        sv->staged.push_back(std::move(st));
        sv->cv.notify_all();
    }
}

void worker_loop(sbwt_server* sv) {
    cudaSetDevice(sv->device);
    void* stream_v = nullptr;
    sbwt_get_stream(sv->idx, &stream_v);
    cudaStream_t stream = (cudaStream_t)stream_v;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv.wait(lk, [&] {
            return !sv->staged.empty() || (sv->stop && sv->queue.empty() && sv->in_stage == 0) || sv->fatal;
        });
        if (sv->staged.empty()) return;
        Staged st = std::move(sv->staged.front());
        sv->staged.pop_front();
        lk.unlock();
        Slot& s = sv->slots[st.slot];
        uint64_t n0 = 0, m0 = 0;
        sbwt_size(sv->idx, &n0, &m0);
        cudaStreamWaitEvent(stream, s.ready, 0);
        int rc = sbwt_serve_append_device(sv->idx, s.d_reads, s.d_off, st.m);
        std::vector<std::pair<Request*, std::pair<int, uint64_t>>> results;
        if (rc == SBWT_OK) {
            uint64_t id = m0;
            for (Request* r : st.reqs) {
                results.push_back({r, {SBWT_OK, id}});
                id += r->m;
            }
        } else if (rc == SBWT_EINVAL && st.reqs.size() > 1) {
            // one request holds a byte outside the alphabet: append one by one
            for (Request* r : st.reqs) {
                uint64_t n1 = 0, m1 = 0;
                sbwt_size(sv->idx, &n1, &m1);
                const int r1 = sbwt_serve_append_host(sv->idx, r->reads.data(), r->offsets.data(), r->m);
                results.push_back({r, {r1, m1}});
                if (r1 != SBWT_OK && r1 != SBWT_EINVAL && r1 != SBWT_ENOMEM) rc = r1;
            }
            if (rc == SBWT_EINVAL) rc = SBWT_OK;
        } else {
            for (Request* r : st.reqs) results.push_back({r, {rc, 0}});
        }
        lk.lock();
        for (auto& x : results) finish(sv, x.first, x.second.first, x.second.second);
        s.busy = false;
        if (rc == SBWT_EDEVICE) sv->fatal = rc;
        sv->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int sbwt_serve_start(sbwt_index* idx, uint64_t max_batch_bases) {
    if (!idx) return SBWT_EINVAL;
    if (sbwt_serve_attached(idx)) return SBWT_EBUSY;
    void* stream = nullptr;
    if (int rc = sbwt_get_stream(idx, &stream)) return rc;  // creates the device state
    sbwt_server* sv = new (std::nothrow) sbwt_server();
    if (!sv) return SBWT_ENOMEM;
    sv->idx = idx;
    sv->max_batch_bases = max_batch_bases;
    cudaGetDevice(&sv->device);
    if (cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->slots[0].ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->slots[1].ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return SBWT_EDEVICE;
    }
    sbwt_serve_attach(idx, sv);
    sv->stager = std::thread(stager_loop, sv);
    sv->worker = std::thread(worker_loop, sv);
    sbwt_serve_set_worker(idx, sv->worker.get_id());
    return SBWT_OK;
}

int sbwt_submit(sbwt_index* idx, const uint8_t* reads, const uint64_t* offsets, uint64_t m, uint64_t* ticket) {
    sbwt_server* sv = idx ? (sbwt_server*)sbwt_serve_attached(idx) : nullptr;
    if (!sv || !offsets || !ticket) return SBWT_EINVAL;
    if (offsets[0] != 0) return SBWT_EINVAL;
    for (uint64_t j = 0; j < m; ++j)
        if (offsets[j + 1] < offsets[j] || offsets[j + 1] - offsets[j] + 1 > (1ull << 31)) return SBWT_EINVAL;
    if (offsets[m] && !reads) return SBWT_EINVAL;
    Request* r = new (std::nothrow) Request();
    if (!r) return SBWT_ENOMEM;
    r->m = m;
    r->offsets.assign(offsets, offsets + m + 1);
    r->reads.assign(reads, reads + offsets[m]);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop || sv->fatal) {
        delete r;
        return sv->fatal ? sv->fatal : SBWT_EBUSY;
    }
    r->ticket = sv->next_ticket++;
    sv->tickets[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    sv->cv.notify_all();
    return SBWT_OK;
}

int sbwt_wait(sbwt_index* idx, uint64_t ticket, uint64_t timeout_us, uint64_t* first_read_id, double* latency_ms) {
    sbwt_server* sv = idx ? (sbwt_server*)sbwt_serve_attached(idx) : nullptr;
    if (!sv) return SBWT_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return SBWT_EINVAL;
    Request* r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us == 0) {
        if (!ready()) return SBWT_ETIMEDOUT;
    } else if (!sv->cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return SBWT_ETIMEDOUT;
    }
    const int status = r->status;
    if (first_read_id) *first_read_id = r->first_id;
    if (latency_ms) *latency_ms = r->latency_ms;
    sv->tickets.erase(it);
    delete r;
    return status;
}

int sbwt_serve_stop(sbwt_index* idx) {
    sbwt_server* sv = idx ? (sbwt_server*)sbwt_serve_attached(idx) : nullptr;
    if (!sv) return SBWT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    sv->stager.join();
    sv->worker.join();
    const int status = sv->fatal;
    for (auto& t : sv->tickets) delete t.second;  // every queued request has a ticket
    for (Slot& s : sv->slots) {
        if (s.h_reads) cudaFreeHost(s.h_reads);
        if (s.h_off) cudaFreeHost(s.h_off);
        if (s.d_reads) cudaFree(s.d_reads);
        if (s.d_off) cudaFree(s.d_off);
        if (s.ready) cudaEventDestroy(s.ready);
    }
    cudaStreamDestroy(sv->copy_stream);
    sbwt_serve_attach(idx, nullptr);
    sbwt_serve_set_worker(idx, std::thread::id());
    delete sv;
    return status;
}

}  // extern "C"
