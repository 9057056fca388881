// Process-wide cache of CUDA resources (see va_pool.h).
#include "va_pool.h"

#include "../../include/analyser.h"

#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

namespace va {
namespace {

std::mutex g_mu;

// size classes: powers of two up to 1 MiB, then multiples of 2 MiB
size_t size_class(size_t bytes) {
  if (bytes <= ((size_t)1 << 20)) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    return c;
  }
  const size_t g = (size_t)2 << 20;
  return (bytes + g - 1) / g * g;
}

struct Block {
  int device;
  size_t cls;
};

std::multimap<std::pair<int, size_t>, void*> g_dev_free;
std::unordered_map<void*, Block> g_dev_live;
size_t g_dev_cached = 0;
std::multimap<size_t, void*> g_host_free;
std::unordered_map<void*, size_t> g_host_live;
std::map<int, std::vector<cudaStream_t>> g_streams;
std::unordered_map<cudaStream_t, int> g_stream_dev;
std::map<std::pair<int, bool>, std::vector<cudaEvent_t>> g_events;
std::unordered_map<cudaEvent_t, std::pair<int, bool>> g_event_key;
std::map<std::pair<int, int>, void*> g_qtabs;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

// frees every cached block of every device (caller holds g_mu)
void trim_locked() {
  int cur = current_device();
  for (auto& kv : g_dev_free) {
    cudaSetDevice(kv.first.first);
    cudaFree(kv.second);
  }
  g_dev_free.clear();
  g_dev_cached = 0;
  for (auto& kv : g_host_free) cudaFreeHost(kv.second);
  g_host_free.clear();
  cudaSetDevice(cur);
}

}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  const int dev = current_device();
  const size_t cls = size_class(bytes);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev_free.find({dev, cls});
  if (it != g_dev_free.end()) {
    *p = it->second;
    g_dev_free.erase(it);
    g_dev_cached -= cls;
    g_dev_live[*p] = {dev, cls};
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc(p, cls);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trim_locked();
    e = cudaMalloc(p, cls);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e;
    }
  }
  g_dev_live[*p] = {dev, cls};
  return cudaSuccess;
}

void pool_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev_live.find(p);
  if (it == g_dev_live.end()) return;
  g_dev_free.insert({{it->second.device, it->second.cls}, p});
  g_dev_cached += it->second.cls;
  g_dev_live.erase(it);
}

cudaError_t pool_malloc_host(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  const size_t cls = size_class(bytes);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_host_free.find(cls);
  if (it != g_host_free.end()) {
    *p = it->second;
    g_host_free.erase(it);
    g_host_live[*p] = cls;
    return cudaSuccess;
  }
  cudaError_t e = cudaMallocHost(p, cls);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trim_locked();
    e = cudaMallocHost(p, cls);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e;
    }
  }
  g_host_live[*p] = cls;
  return cudaSuccess;
}

void pool_free_host(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_host_live.find(p);
  if (it == g_host_live.end()) return;
  g_host_free.insert({it->second, p});
  g_host_live.erase(it);
}

cudaError_t pool_stream(cudaStream_t* s) {
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto& v = g_streams[dev];
    if (!v.empty()) {
      *s = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stream_dev[*s] = dev;
  }
  return e;
}

void pool_release_stream(cudaStream_t s) {
  if (!s) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_stream_dev.find(s);
  if (it == g_stream_dev.end()) return;
  g_streams[it->second].push_back(s);
}

cudaError_t pool_event(cudaEvent_t* ev, bool timing) {
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto& v = g_events[{dev, timing}];
    if (!v.empty()) {
      *ev = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  cudaError_t e = timing ? cudaEventCreate(ev) : cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_event_key[*ev] = {dev, timing};
  }
  return e;
}

void pool_release_event(cudaEvent_t ev) {
  if (!ev) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_event_key.find(ev);
  if (it == g_event_key.end()) return;
  g_events[it->second].push_back(ev);
}

cudaError_t pool_qtab(int qmax, void (*build)(uint32_t*, int), const uint32_t** out) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_qtabs.find({dev, qmax});
  if (it != g_qtabs.end()) {
    *out = static_cast<const uint32_t*>(it->second);
    return cudaSuccess;
  }
  std::vector<uint32_t> q((size_t)qmax + 1);
  build(q.data(), qmax);
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(uint32_t) * q.size());
  if (e == cudaSuccess) e = cudaMemcpy(d, q.data(), sizeof(uint32_t) * q.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (d) cudaFree(d);
    return e;
  }
  g_qtabs[{dev, qmax}] = d;
  *out = static_cast<const uint32_t*>(d);
  return cudaSuccess;
}

void pool_trim() {
  std::lock_guard<std::mutex> lk(g_mu);
  trim_locked();
}

size_t pool_cached_bytes() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_dev_cached;
}

}  // namespace va

extern "C" void analyser_trim_cache(void) { va::pool_trim(); }
extern "C" long long analyser_cached_bytes(void) { return (long long)va::pool_cached_bytes(); }
