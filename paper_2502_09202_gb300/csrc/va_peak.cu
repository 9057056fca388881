// Register-only throughput of the packed-SAD step the kernels use (sad4 in
// va_device.cuh): the denominator of the ALU roofline.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/analyser.h"
#include "va_device.cuh"

namespace {

// One packed step c + sum_k |a_k - b_k| as each measured sequence computes it:
//   0  vabsdiff4 with accumulate (the kernels' sad4)
//   1  sum-of-absolute-differences intrinsic, then an add
//   2  per-byte absolute differences, then dp4a with ones (sum on another pipe)
//   3  per-byte max minus per-byte min, then dp4a with ones
//   4  chains 0-3 as sequence 0 and chains 4-7 as sequence 2 (both pipes at once)
template <int SEQ>
__device__ __forceinline__ uint32_t packed_step(uint32_t a, uint32_t b, uint32_t c, int chain) {
  if constexpr (SEQ == 0) {
    return va::sad4(a, b, c);
  } else if constexpr (SEQ == 1) {
    return __vsadu4(a, b) + c;
  } else if constexpr (SEQ == 2) {
    return (uint32_t)__dp4a(__vabsdiffu4(a, b), 0x01010101u, c);
  } else if constexpr (SEQ == 3) {
    return (uint32_t)__dp4a(__vmaxu4(a, b) - __vminu4(a, b), 0x01010101u, c);
  } else {
    return chain < 4 ? packed_step<0>(a, b, c, chain) : packed_step<2>(a, b, c, chain);
  }
}

template <int SEQ>
__global__ void sad_peak_kernel(uint32_t* out, int iters, uint32_t seed) {
  // 8 accumulator chains x 16 operands: the 128 (a, b) pairs of an iteration are
  // distinct and every b changes each iteration, so no SAD can be shared with
  // another or hoisted out of the loop (16 adds per 128 SADs is the only other
  // work, which makes the figure a slight underestimate of the peak)
  uint32_t a[8], acc[8], bw[16];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    a[i] = seed * (threadIdx.x + 7u * i + 1u);
    acc[i] = 0;
  }
#pragma unroll
  for (int u = 0; u < 16; u++) bw[u] = (seed ^ blockIdx.x) * (2u * u + 1u);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = packed_step<SEQ>(a[i], bw[u], acc[i], i);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) bw[u] += 0x01030507u;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += acc[i];
  if (s == 0x12345678u) out[0] = s;   // keeps the chains live
}

template <int SEQ>
void launch_peak(int blocks, int threads, cudaStream_t st, uint32_t* d, int iters, uint32_t seed) {
  sad_peak_kernel<SEQ><<<blocks, threads, 0, st>>>(d, iters, seed);
}

void launch_seq(int seq, int blocks, int threads, cudaStream_t st, uint32_t* d, int iters, uint32_t seed) {
  switch (seq) {
    case 1: launch_peak<1>(blocks, threads, st, d, iters, seed); break;
    case 2: launch_peak<2>(blocks, threads, st, d, iters, seed); break;
    case 3: launch_peak<3>(blocks, threads, st, d, iters, seed); break;
    case 4: launch_peak<4>(blocks, threads, st, d, iters, seed); break;
    default: launch_peak<0>(blocks, threads, st, d, iters, seed); break;
  }
}

}  // namespace

extern "C" int analyser_measure_sad_sequence(int device, int sequence, double* tera_per_s) {
  if (!tera_per_s || sequence < 0 || sequence > 4) return ANALYSER_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return ANALYSER_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ANALYSER_ERR_CUDA;
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, sizeof(uint32_t)) != cudaSuccess) return ANALYSER_ERR_OOM;
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  launch_seq(sequence, blocks, threads, st, d, 16, 3u);
  float best = 1e30f;
  for (int r = 0; r < 5; r++) {
    cudaEventRecord(e0, st);
    launch_seq(sequence, blocks, threads, st, d, iters, 3u + r);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(d);
  if (err != cudaSuccess) return ANALYSER_ERR_CUDA;
  const double ops = (double)blocks * threads * iters * 16.0 * 8.0 * 4.0;   // |a-b| accumulates
  *tera_per_s = ops / (best * 1e-3) / 1e12;
  return ANALYSER_OK;
}

extern "C" int analyser_measure_sad_peak(int device, double* tera_per_s) {
  return analyser_measure_sad_sequence(device, 0, tera_per_s);
}
