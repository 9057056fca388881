// analyser_measure_pair_noalloc: one pair measure whose scratch memory (pyramid
// levels, job descriptors, accumulators, square-root table, status word) lives
// in a fixed device array owned by this library, so the call itself never
// allocates device memory.
//
// Who needs it: a caller embedded in a host application that reserves all of
// its device memory up front (a video pipeline or plugin host with a fixed
// budget and its own pool) must not call cudaMalloc/cudaFree while it runs:
// an allocation can fail against the host's reservation, and cudaMalloc /
// cudaFree synchronise the device, which breaks the pipeline's latency.
//
// Limits and sharing:
//   - kNoAllocScratchBytes (5.5 MiB) bounds the pyramids of the two images of
//     one pair; 3840x2160 frames fit, anything needing more is rejected with
//     ANALYSER_ERR_INVALID_ARG;
//   - the array exists once per device for the life of the process and is
//     shared by every call: calls whose GPU work overlaps (other threads or
//     streams) race on it; the accumulators and the status word are cleared at
//     the start of every call;
//   - the device address of the array is looked up once per device
//     (cudaGetSymbolAddress) by the first call for that device; make that
//     first call before any stream capture;
//   - every call waits for its stream before it returns (the record is read
//     back to host memory), and leaves the calling thread's current device as
//     it found it.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/analyser.h"
#include "va_kernels.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)11 << 19;   // 5.5 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round16(int v) { return (v + 15) / 16 * 16; }

// floor(sqrt(n)) by Newton's iteration on integers
uint64_t isqrt_newton(uint64_t n) {
  if (n < 2) return n;
  uint64_t x = n, y = (x + 1) / 2;
  while (y < x) {
    x = y;
    y = (x + n / x) / 2;
  }
  return x;
}

int scratch_ptr(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return ANALYSER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ANALYSER_ERR_CUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
  return ANALYSER_OK;
}

}  // namespace

extern "C" int analyser_measure_pair_noalloc(const analyser_params* p, int width, int height, int kind,
                                             const uint8_t* frame_a, const uint8_t* frame_b, long long pitch_bytes,
                                             int64_t* record, void* stream) {
  using namespace va;
  if (!p || !frame_a || !frame_b || !record) return ANALYSER_ERR_INVALID_ARG;
  if (kind < ANALYSER_PAIR_FRAME || kind > ANALYSER_PAIR_LOWER_LOWER) return ANALYSER_ERR_INVALID_ARG;
  if (width < 64 || height < 64 || (height & 1) || (long long)width * height > 11800000LL)
    return ANALYSER_ERR_INVALID_ARG;
  if (p->levels != 3 || p->block != 16 || p->radius_refine < 0 || p->radius_refine > 4 || p->mv_cost < 0 ||
      p->mv_cost > 64 || !pair_tile_supported(p->radius_coarse, p->tile_x ? p->tile_x : 8, p->tile_y ? p->tile_y : 4))
    return ANALYSER_ERR_INVALID_ARG;
  // field kinds double the pitch, and the kernels' plane descriptors hold it in an int
  if (pitch_bytes < width || pitch_bytes % 16 || pitch_bytes > INT_MAX / 2 || ((uintptr_t)frame_a % 16) ||
      ((uintptr_t)frame_b % 16))
    return ANALYSER_ERR_INVALID_ARG;

  // image geometry of this pair kind: a frame, or a field (pitch doubled)
  const bool field = kind != ANALYSER_PAIR_FRAME;
  const int h0 = field ? height / 2 : height;
  const long long p0 = field ? 2 * pitch_bytes : pitch_bytes;
  const bool i_lower = kind == ANALYSER_PAIR_LOWER_UPPER || kind == ANALYSER_PAIR_LOWER_LOWER;
  const bool j_lower = kind == ANALYSER_PAIR_UPPER_LOWER || kind == ANALYSER_PAIR_LOWER_LOWER;
  const uint8_t* I0 = i_lower ? frame_a + pitch_bytes : frame_a;
  const uint8_t* J0 = j_lower ? frame_b + pitch_bytes : frame_b;
  const int w1 = width / 2, h1 = h0 / 2, w2 = w1 / 2, h2 = h1 / 2;
  const int p1 = round16(w1), p2 = round16(w2);

  int vmax = p->radius_coarse;
  for (int l = 0; l < 2; l++) vmax = 2 * vmax + p->radius_refine;
  const int qmax = 2 * vmax * vmax;

  // scratch layout
  size_t off = 0;
  const size_t off_status = off; off = align_up(off + sizeof(int), 256);
  const size_t off_rec = off; off = align_up(off + sizeof(unsigned long long) * kRecWords, 256);
  const size_t off_q = off; off = align_up(off + sizeof(uint32_t) * (qmax + 1), 256);
  const size_t off_dj = off; off = align_up(off + sizeof(DownJob) * 4, 256);
  const size_t off_pj = off; off = align_up(off + sizeof(PairJob), 256);
  const size_t off_i1 = off; off = align_up(off + (size_t)p1 * h1 + 16, 256);
  const size_t off_j1 = off; off = align_up(off + (size_t)p1 * h1 + 16, 256);
  const size_t off_i2 = off; off = align_up(off + (size_t)p2 * h2 + 16, 256);
  const size_t off_j2 = off; off = align_up(off + (size_t)p2 * h2 + 16, 256);
  if (off > kNoAllocScratchBytes) return ANALYSER_ERR_INVALID_ARG;   // beyond the fixed scratch

  int prev_device = 0;
  if (cudaGetDevice(&prev_device) != cudaSuccess) return ANALYSER_ERR_CUDA;
  if (prev_device != p->device && cudaSetDevice(p->device) != cudaSuccess) return ANALYSER_ERR_CUDA;
  // the caller's current device is restored on every return below
  struct RestoreDevice {
    int dev, was;
    ~RestoreDevice() { if (dev != was) cudaSetDevice(was); }
  } restore{p->device, prev_device};
  unsigned char* s = nullptr;
  int rc = scratch_ptr(p->device, &s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;

  // descriptors built on the host stack; pageable copies complete their host read before returning
  static uint32_t qtab[2 * 140 * 140 + 1];
  static int qtab_n = -1;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (qtab_n < qmax) {
      for (int k = 0; k <= qmax; k++) qtab[k] = (uint32_t)isqrt_newton((uint64_t)k << 32);
      qtab_n = qmax;
    }
  }
  DownJob dj[4];
  dj[0] = {{I0, (int)p0, width, h0}, s + off_i1, p1};
  dj[1] = {{J0, (int)p0, width, h0}, s + off_j1, p1};
  dj[2] = {{s + off_i1, p1, w1, h1}, s + off_i2, p2};
  dj[3] = {{s + off_j1, p1, w1, h1}, s + off_j2, p2};
  const int tbx = p->tile_x ? p->tile_x : 8, tby = p->tile_y ? p->tile_y : 4;
  PairJob pj;
  std::memset(&pj, 0, sizeof(pj));
  pj.I[0] = {I0, (int)p0, width, h0};
  pj.J[0] = {J0, (int)p0, width, h0};
  pj.I[1] = {s + off_i1, p1, w1, h1};
  pj.J[1] = {s + off_j1, p1, w1, h1};
  pj.I[2] = {s + off_i2, p2, w2, h2};
  pj.J[2] = {s + off_j2, p2, w2, h2};
  pj.nbx = width / 16;
  pj.nby = h0 / 16;
  pj.tiles_x = (pj.nbx + tbx - 1) / tbx;
  pj.tiles_y = (pj.nby + tby - 1) / tby;
  pj.item_begin = 0;
  pj.rec = reinterpret_cast<unsigned long long*>(s + off_rec);
  pj.vec = nullptr;

  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  step(cudaMemsetAsync(s + off_status, 0, sizeof(int), st));
  step(cudaMemsetAsync(s + off_rec, 0, sizeof(unsigned long long) * kRecWords, st));
  step(cudaMemcpyAsync(s + off_q, qtab, sizeof(uint32_t) * (qmax + 1), cudaMemcpyHostToDevice, st));
  step(cudaMemcpyAsync(s + off_dj, dj, sizeof(dj), cudaMemcpyHostToDevice, st));
  step(cudaMemcpyAsync(s + off_pj, &pj, sizeof(pj), cudaMemcpyHostToDevice, st));
  const DownJob* ddj = reinterpret_cast<const DownJob*>(s + off_dj);
  step(launch_downsample(ddj, 2, h1, w1, st));
  step(launch_downsample(ddj + 2, 2, h2, w2, st));
  PairBatch b;
  b.jobs = reinterpret_cast<const PairJob*>(s + off_pj);
  b.njobs = 1;
  b.nitems = pj.tiles_x * pj.tiles_y;
  b.qtab = reinterpret_cast<const uint32_t*>(s + off_q);
  b.qmax = qmax;
  b.cfg = {p->levels, p->radius_coarse, p->radius_refine, p->mv_cost};
  b.status = reinterpret_cast<int*>(s + off_status);
  int sms = 0;
  step(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  const int per_sm = pair_blocks_per_sm(p->radius_coarse, tbx, tby);
  const int grid = b.nitems < sms * per_sm ? b.nitems : sms * per_sm;
  step(launch_pairs(b, tbx, tby, grid > 0 ? grid : 1, st));
  unsigned long long rec[kRecWords];
  int status = 0;
  step(cudaMemcpyAsync(rec, s + off_rec, sizeof(rec), cudaMemcpyDeviceToHost, st));
  step(cudaMemcpyAsync(&status, s + off_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  step(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return ANALYSER_ERR_CUDA;
  if (status) return ANALYSER_ERR_CUDA;
  for (int k = 0; k < kRecWords; k++) record[k] = (int64_t)rec[k];
  return ANALYSER_OK;
}
