// Process-wide cache of device memory, page-locked host memory, streams,
// events and square-root tables, so that analysers, servers and stateless
// measure calls created one after another reuse what the previous ones held
// instead of paying cudaMalloc/cudaFree (which also synchronises the device)
// and stream creation every time.
//
// A released block goes back to a free list of its device and size class and
// is handed out again for a request of the same class.  The caller must make
// sure that no GPU work still uses a block or stream it releases (synchronise
// the streams that used it first).  A failed cudaMalloc / cudaMallocHost
// empties the cache and is retried once.  pool_trim() returns everything
// cached to CUDA.  All functions are thread-safe.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace va {

cudaError_t pool_malloc(void** p, size_t bytes);        // on the current device
void pool_free(void* p);                                // null is ignored
cudaError_t pool_malloc_host(void** p, size_t bytes);   // page-locked
void pool_free_host(void* p);
cudaError_t pool_stream(cudaStream_t* s);               // non-blocking stream of the current device
void pool_release_stream(cudaStream_t s);
cudaError_t pool_event(cudaEvent_t* e, bool timing);    // event of the current device
void pool_release_event(cudaEvent_t e);
// Q(k) = floor(sqrt(k) * 2^16) for k = 0..qmax on the current device, built
// once per (device, qmax) and kept for the life of the process (a few tens of
// KB; live analysers point at it); `build` fills a host array of qmax + 1
// entries.
cudaError_t pool_qtab(int qmax, void (*build)(uint32_t* q, int qmax), const uint32_t** out);
void pool_trim();             // frees the cached blocks (not live ones, not the Q tables)
size_t pool_cached_bytes();   // device bytes held in free lists

}  // namespace va
