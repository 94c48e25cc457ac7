// sbwt_serve.h -- hooks between the index runtime (capi.cu) and the
// continuous-batching server (serve.cu).  Internal, not exported.
#pragma once

#include <thread>

#include "sbwt.h"

// The server attached to an index (NULL when not serving).
void* sbwt_serve_attached(sbwt_index* idx);
void sbwt_serve_attach(sbwt_index* idx, void* server);
// While serving, only this thread may change the index.
void sbwt_serve_set_worker(sbwt_index* idx, std::thread::id id);
// Appends used by the server's worker thread.
int sbwt_serve_append_device(sbwt_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint64_t m);
int sbwt_serve_append_host(sbwt_index* idx, const uint8_t* reads, const uint64_t* offsets, uint64_t m);
