// Dense sub-pixel flow by inverse search (the estimator the paper names in
// Sec. III.A, reference [8]), as an alternative to the block-matching motion
// field: for one pair of 8-bit frames in device memory,
//   1. box pyramid (2x2 mean with rounding, as the block-matching path);
//   2. per level, coarsest first, P x P patches of frame a on a grid of
//      stride S (the last patch of a row or column flush with the border);
//   3. per patch, `iters` inverse-compositional Gauss-Newton steps on the
//      patch's template: H from the template's central-difference gradients
//      (clamp-to-edge), damped by d = damp_rel * trace(H) + damp_abs;
//      r = J(x + u) - T(x) with J sampled bilinearly (clamp-to-edge);
//      u <- u - (H + d I)^-1 sum grad T r;
//   4. a patch starts from the next coarser level's dense flow, sampled
//      bilinearly at the patch centre ((fine - 0.5) / 2) and doubled;
//   5. densification: a pixel's flow is the mean of its covering patches'
//      flows weighted by 1 / max(1, |J(x + u_i) - I(x)|).
// There is no threshold anywhere (fixed step count, no patch rejection).  The
// steps run in FP32 by default or in FP64; in patches where the iteration does
// not converge, FP32 rounding (sample positions near x = 1000 are spaced about
// 1e-4 px apart) can grow over the steps, so only the FP64 instantiation is
// expected to match an FP64 evaluation element by element.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>

#include "../../include/analyser.h"
#include "va_pool.h"

namespace va {
namespace {

constexpr int kFlowPatch = 8;   // P (a warp holds a patch's 64 pixels, two per lane)

struct U8Plane {
  const uint8_t* p;
  int w, h, pitch;
};

__device__ __forceinline__ int px(const U8Plane& m, int x, int y) { return m.p[(size_t)y * m.pitch + x]; }

// Every kernel below is instantiated for F = float (the default) and
// F = double (the same steps in FP64: `analyser_flow_params.fp64`).

// v clamped to [0, hi]; NaN (a flow the damping cannot keep finite) maps to 0,
// so that a sample position always indexes inside the image
template <typename F>
__device__ __forceinline__ F clampf(F v, F hi) {
  if (!(v >= F(0))) return F(0);
  return v > hi ? hi : v;
}

// m sampled at (x, y): the position clamped to the image, then bilinear
// between the four surrounding pixels
template <typename F>
__device__ __forceinline__ F sample_u8(const U8Plane& m, F x, F y) {
  x = clampf(x, F(m.w - 1));
  y = clampf(y, F(m.h - 1));
  const F fx0 = floor(x), fy0 = floor(y);
  const int x0 = (int)fx0, y0 = (int)fy0;
  const int x1 = min(x0 + 1, m.w - 1), y1 = min(y0 + 1, m.h - 1);
  const F fx = x - fx0, fy = y - fy0;
  const F top = F(px(m, x0, y0)) * (F(1) - fx) + F(px(m, x1, y0)) * fx;
  const F bot = F(px(m, x0, y1)) * (F(1) - fx) + F(px(m, x1, y1)) * fx;
  return top * (F(1) - fy) + bot * fy;
}

// component c of a dense flow field (w x h pairs of F) sampled like sample_u8
template <typename F>
__device__ __forceinline__ F sample_flow(const F* f, int w, int h, F x, F y, int c) {
  x = clampf(x, F(w - 1));
  y = clampf(y, F(h - 1));
  const F fx0 = floor(x), fy0 = floor(y);
  const int x0 = (int)fx0, y0 = (int)fy0;
  const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
  const F fx = x - fx0, fy = y - fy0;
  auto at = [&](int xx, int yy) { return f[2 * ((size_t)yy * w + xx) + c]; };
  const F top = at(x0, y0) * (F(1) - fx) + at(x1, y0) * fx;
  const F bot = at(x0, y1) * (F(1) - fx) + at(x1, y1) * fx;
  return top * (F(1) - fy) + bot * fy;
}

template <typename F>
__device__ __forceinline__ F warp_sum(F v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// patch origin k along an axis of length n: k * S, the last one n - P
__device__ __forceinline__ int patch_origin(int k, int n, int S) { return min(k * S, n - kFlowPatch); }

// 2x2 box mean with rounding, floor(w/2) x floor(h/2)
__global__ void flow_down_kernel(const uint8_t* src, int spitch, uint8_t* dst, int dw, int dh, int dpitch) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= dw || y >= dh) return;
  const uint8_t* r0 = src + (size_t)(2 * y) * spitch + 2 * x;
  const uint8_t* r1 = r0 + spitch;
  dst[(size_t)y * dpitch + x] = (uint8_t)(((unsigned)r0[0] + r0[1] + r1[0] + r1[1] + 2u) >> 2);
}

// one warp per patch (step 3); lane l holds pixels l and l + 32 of the patch
// (row p / 8, column p % 8); flows and dense fields are pairs (u, v) of F
template <typename F>
__global__ void flow_search_kernel(U8Plane I, U8Plane J, const F* coarse, int cw, int ch, F* flows, int npx,
                                   int npy, int S, int iters, F damp_rel, F damp_abs) {
  const int patch = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (patch >= npx * npy) return;   // the whole warp
  const int x0 = patch_origin(patch % npx, I.w, S), y0 = patch_origin(patch / npx, I.h, S);
  F t[2], gx[2], gy[2], X[2], Y[2];
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int p = lane + 32 * k, x = x0 + (p & 7), y = y0 + (p >> 3);
    t[k] = F(px(I, x, y));
    gx[k] = F(px(I, min(x + 1, I.w - 1), y) - px(I, max(x - 1, 0), y)) * F(0.5);
    gy[k] = F(px(I, x, min(y + 1, I.h - 1)) - px(I, x, max(y - 1, 0))) * F(0.5);
    X[k] = F(x);
    Y[k] = F(y);
  }
  const F h00 = warp_sum(gx[0] * gx[0] + gx[1] * gx[1]);
  const F h01 = warp_sum(gx[0] * gy[0] + gx[1] * gy[1]);
  const F h11 = warp_sum(gy[0] * gy[0] + gy[1] * gy[1]);
  const F d = damp_rel * (h00 + h11) + damp_abs;
  const F a = h00 + d, c = h11 + d;
  const F det = a * c - h01 * h01;
  F ux = F(0), uy = F(0);
  if (coarse) {   // step 4
    const F cx = (F(x0) + F(0.5) * F(kFlowPatch - 1) - F(0.5)) * F(0.5);
    const F cy = (F(y0) + F(0.5) * F(kFlowPatch - 1) - F(0.5)) * F(0.5);
    ux = F(2) * sample_flow(coarse, cw, ch, cx, cy, 0);
    uy = F(2) * sample_flow(coarse, cw, ch, cx, cy, 1);
  }
  const int col = lane & 7, row = lane >> 3;   // pixel 0 at (row, col), pixel 1 at (row + 4, col)
  for (int it = 0; it < iters; it++) {
    F bx = F(0), by = F(0);
    // FP32: every pixel of the patch is sampled at the same offset u, so the
    // 9 x 9 bilinear footprint starts at integer (x0 + floor(ux), y0 + floor(uy))
    // with the same weights (ux - floor(ux), uy - floor(uy)) for all.  Where the
    // footprint lies inside J (no clamping), a lane reads its two pixels'
    // top-left values and takes the right and lower neighbours from the lanes
    // that read them (the patch's right column and bottom row read their own).
    // The FP64 instantiation, and FP32 elsewhere, sample each pixel at x + u as
    // the per-pixel definition does: the two agree in exact arithmetic, but the
    // rounding of x + u differs, and FP64 keeps the definition's rounding.
    // (The comparisons fail for a non-finite flow, which takes the per-pixel path.)
    const F fux = floor(ux), fuy = floor(uy);
    const bool fast = sizeof(F) == sizeof(float) && fux >= F(-x0) && fuy >= F(-y0) &&
                      fux <= F(J.w - 1 - kFlowPatch - x0) && fuy <= F(J.h - 1 - kFlowPatch - y0);
    if (fast) {   // warp-uniform
      const int ix = x0 + (int)fux, iy = y0 + (int)fuy;
      const F fx = ux - fux, fy = uy - fuy;
      const uint8_t* q = J.p + (size_t)(iy + row) * J.pitch + ix + col;
      const size_t p4 = (size_t)4 * J.pitch;
      const int a = q[0], b = q[p4];   // J(iy + row, ix + col), J(iy + row + 4, ix + col)
      int ar = __shfl_sync(0xFFFFFFFFu, a, lane + 1), br = __shfl_sync(0xFFFFFFFFu, b, lane + 1);
      if (col == 7) {
        ar = q[1];
        br = q[p4 + 1];
      }
      // the row below pixel 0: lane + 8's pixel 0 (row < 3) or column col's pixel 1 (row 3)
      const int sa = __shfl_sync(0xFFFFFFFFu, a, lane + 8), sar = __shfl_sync(0xFFFFFFFFu, ar, lane + 8);
      const int sb = __shfl_sync(0xFFFFFFFFu, b, col), sbr = __shfl_sync(0xFFFFFFFFu, br, col);
      const int ad = row < 3 ? sa : sb, adr = row < 3 ? sar : sbr;
      // the row below pixel 1: lane + 8's pixel 1 (row < 3) or row iy + 8 (row 3)
      int bd = __shfl_sync(0xFFFFFFFFu, b, lane + 8), bdr = __shfl_sync(0xFFFFFFFFu, br, lane + 8);
      if (row == 3) {   // q is on row iy + 3; the footprint's last row is iy + 8
        bd = q[(size_t)5 * J.pitch];
        bdr = q[(size_t)5 * J.pitch + 1];
      }
      const F v0 = (F(a) * (F(1) - fx) + F(ar) * fx) * (F(1) - fy) + (F(ad) * (F(1) - fx) + F(adr) * fx) * fy;
      const F v1 = (F(b) * (F(1) - fx) + F(br) * fx) * (F(1) - fy) + (F(bd) * (F(1) - fx) + F(bdr) * fx) * fy;
      const F r0 = v0 - t[0], r1 = v1 - t[1];
      bx = gx[0] * r0 + gx[1] * r1;
      by = gy[0] * r0 + gy[1] * r1;
    } else {
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const F r = sample_u8(J, X[k] + ux, Y[k] + uy) - t[k];
        bx += gx[k] * r;
        by += gy[k] * r;
      }
    }
    bx = warp_sum(bx);
    by = warp_sum(by);
    ux -= (c * bx - h01 * by) / det;
    uy -= (a * by - h01 * bx) / det;
  }
  if (lane == 0) {
    flows[2 * patch] = ux;
    flows[2 * patch + 1] = uy;
  }
}

// one thread per pixel (step 5): the covering patches in row-major patch order;
// `out` holds (u, v) per pixel as F, or as float when `out32` is set
template <typename F>
__global__ void flow_densify_kernel(U8Plane I, U8Plane J, const F* flows, int npx, int npy, int S, F* out,
                                    float* out32) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.w || y >= I.h) return;
  const F iv = F(px(I, x, y));
  F nx = F(0), ny = F(0), den = F(0);
  // patch k covers x when origin(k) <= x < origin(k) + P; k ranges over
  // ceil((x - P + 1) / S) .. floor(x / S), and one more for the flush last patch
  const int kx0 = max(0, (x - kFlowPatch + S) / S), kx1 = min(npx - 1, x / S + 1);
  const int ky0 = max(0, (y - kFlowPatch + S) / S), ky1 = min(npy - 1, y / S + 1);
  for (int ky = ky0; ky <= ky1; ky++) {
    const int oy = patch_origin(ky, I.h, S);
    if (oy > y || y >= oy + kFlowPatch) continue;
    for (int kx = kx0; kx <= kx1; kx++) {
      const int ox = patch_origin(kx, I.w, S);
      if (ox > x || x >= ox + kFlowPatch) continue;
      const F ux = flows[2 * (ky * npx + kx)], uy = flows[2 * (ky * npx + kx) + 1];
      const F e = sample_u8(J, F(x) + ux, F(y) + uy) - iv;
      const F ae = e < F(0) ? -e : e;
      const F wgt = F(1) / (ae > F(1) ? ae : F(1));
      nx += wgt * ux;
      ny += wgt * uy;
      den += wgt;
    }
  }
  const size_t o = 2 * ((size_t)y * I.w + x);
  if (out32) {
    out32[o] = (float)(nx / den);
    out32[o + 1] = (float)(ny / den);
  } else {
    out[o] = nx / den;
    out[o + 1] = ny / den;
  }
}

// The pair measures' sums over the dense flow U (float (u, v) per pixel): per
// pixel |U|, I(x) and Jw(x) = J(x + U(x)) (bilinear, clamp-to-edge, in F); a
// block's threads stride over the pixels accumulating in FP64 and the block
// writes its six partial sums (|U|, I, Jw, I^2, Jw^2, I Jw) to part[block]
constexpr int kMeasureThreads = 256, kMeasureBlocks = 1024;
template <typename F>
__global__ void __launch_bounds__(kMeasureThreads) flow_measure_kernel(U8Plane I, U8Plane J, const float* flow,
                                                                       double* part) {
  __shared__ double red[kMeasureThreads / 32][6];
  double v[6] = {0, 0, 0, 0, 0, 0};
  const long long n = (long long)I.w * I.h;
  for (long long i = blockIdx.x * (long long)kMeasureThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kMeasureThreads) {
    const int x = (int)(i % I.w), y = (int)(i / I.w);
    const F u = F(flow[2 * i]), w = F(flow[2 * i + 1]);
    const F iv = F(px(I, x, y));
    const F jw = sample_u8(J, F(x) + u, F(y) + w);
    v[0] += (double)sqrt(u * u + w * w);
    v[1] += (double)iv;
    v[2] += (double)jw;
    v[3] += (double)iv * (double)iv;
    v[4] += (double)jw * (double)jw;
    v[5] += (double)iv * (double)jw;
  }
#pragma unroll
  for (int k = 0; k < 6; k++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], off);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 6; k++) red[threadIdx.x >> 5][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int wp = 0; wp < kMeasureThreads / 32; wp++) s += red[wp][threadIdx.x];
    part[6 * blockIdx.x + threadIdx.x] = s;
  }
}

// sums[k] = the blocks' partials in block order (one thread per word): the
// same value on every call
__global__ void flow_sum_kernel(const double* part, int nblocks, double* sums) {
  if (threadIdx.x >= 6) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; b++) s += part[6 * b + threadIdx.x];
  sums[threadIdx.x] = s;
}

int patches_along(int n, int S) { return (n - kFlowPatch + S - 1) / S + 1; }

template <typename F>
int dense_flow(const analyser_flow_params* fp, int width, int height, const uint8_t* frame_a, const uint8_t* frame_b,
               long long pitch_bytes, float* flow, cudaStream_t st) {
  const int L = fp->levels, S = fp->stride;
  // scratch: levels 1..L-1 of both frames, the patch flows of the largest
  // level, the dense flows of levels L-1..1 (pairs of F)
  int w[3], h[3], pitch[3];
  w[0] = width;
  h[0] = height;
  pitch[0] = (int)pitch_bytes;
  size_t bytes = 0, off_img[3][2] = {}, off_dense[3] = {};
  for (int l = 1; l < L; l++) {
    w[l] = w[l - 1] / 2;
    h[l] = h[l - 1] / 2;
    pitch[l] = (w[l] + 15) / 16 * 16;
    for (int f = 0; f < 2; f++) {
      off_img[l][f] = bytes;
      bytes += ((size_t)pitch[l] * h[l] + 255) / 256 * 256;
    }
  }
  for (int l = 1; l < L; l++) {
    off_dense[l] = bytes;
    bytes += ((size_t)w[l] * h[l] * 2 * sizeof(F) + 255) / 256 * 256;
  }
  const size_t off_flows = bytes;
  bytes += (size_t)patches_along(w[0], S) * patches_along(h[0], S) * 2 * sizeof(F);
  uint8_t* scratch = nullptr;
  if (pool_malloc(reinterpret_cast<void**>(&scratch), bytes) != cudaSuccess) return ANALYSER_ERR_OOM;
  cudaError_t e = cudaSuccess;
  const uint8_t* img[3][2] = {{frame_a, frame_b}, {nullptr, nullptr}, {nullptr, nullptr}};
  for (int l = 1; l < L && e == cudaSuccess; l++) {
    for (int f = 0; f < 2; f++) {
      uint8_t* dst = scratch + off_img[l][f];
      const dim3 grid((w[l] + 127) / 128, h[l]);
      flow_down_kernel<<<grid, 128, 0, st>>>(img[l - 1][f], pitch[l - 1], dst, w[l], h[l], pitch[l]);
      img[l][f] = dst;
    }
    e = cudaGetLastError();
  }
  F* flows = reinterpret_cast<F*>(scratch + off_flows);
  const F* coarse = nullptr;
  for (int l = L - 1; l >= 0 && e == cudaSuccess; l--) {
    const U8Plane I{img[l][0], w[l], h[l], pitch[l]}, J{img[l][1], w[l], h[l], pitch[l]};
    const int npx = patches_along(w[l], S), npy = patches_along(h[l], S);
    const long long threads = (long long)npx * npy * 32;
    flow_search_kernel<F><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        I, J, coarse, l + 1 < L ? w[l + 1] : 0, l + 1 < L ? h[l + 1] : 0, flows, npx, npy, S, fp->iters,
        (F)fp->damp_rel, (F)fp->damp_abs);
    F* dense = reinterpret_cast<F*>(scratch + off_dense[l]);
    flow_densify_kernel<F><<<dim3((w[l] + 127) / 128, h[l]), 128, 0, st>>>(I, J, flows, npx, npy, S,
                                                                         l == 0 ? nullptr : dense,
                                                                         l == 0 ? flow : nullptr);
    e = cudaGetLastError();
    coarse = dense;
  }
  // the scratch goes back to the cache only once the kernels that use it are done
  const cudaError_t es = cudaStreamSynchronize(st);
  pool_free(scratch);
  if (e != cudaSuccess || es != cudaSuccess) return ANALYSER_ERR_CUDA;
  return ANALYSER_OK;
}

}  // namespace
}  // namespace va

extern "C" void analyser_default_flow_params(analyser_flow_params* p) {
  if (!p) return;
  p->levels = 3;
  p->patch = 8;
  p->stride = 4;
  p->iters = 8;
  p->fp64 = 0;
  p->damp_rel = 0.01;
  p->damp_abs = 1.0;
}

extern "C" int analyser_dense_flow(const analyser_flow_params* fp, int width, int height, const uint8_t* frame_a,
                                   const uint8_t* frame_b, long long pitch_bytes, float* flow, void* stream) {
  using namespace va;
  if (!fp || !frame_a || !frame_b || !flow) return ANALYSER_ERR_INVALID_ARG;
  const int L = fp->levels;
  if (L < 1 || L > 3 || fp->patch != kFlowPatch || fp->stride < 1 || fp->stride > kFlowPatch || fp->iters < 0 ||
      fp->iters > 64 || (fp->fp64 != 0 && fp->fp64 != 1) || !(fp->damp_rel >= 0.0) || !(fp->damp_abs > 0.0))
    return ANALYSER_ERR_INVALID_ARG;
  if (width < (kFlowPatch << (L - 1)) || height < (kFlowPatch << (L - 1)) || width > 16384 || height > 16384 ||
      pitch_bytes < width || pitch_bytes > INT_MAX)
    return ANALYSER_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  return fp->fp64 ? dense_flow<double>(fp, width, height, frame_a, frame_b, pitch_bytes, flow, st)
                  : dense_flow<float>(fp, width, height, frame_a, frame_b, pitch_bytes, flow, st);
}

extern "C" int analyser_flow_measure(const analyser_flow_params* fp, int width, int height, const uint8_t* frame_a,
                                     const uint8_t* frame_b, long long pitch_bytes, analyser_flow_measure_t* out,
                                     void* stream) {
  using namespace va;
  if (!out) return ANALYSER_ERR_INVALID_ARG;
  // the flow (float, w x h x 2), the blocks' partial sums and the six FP64
  // sums in one cached buffer
  const size_t flow_bytes = ((size_t)width * height * 2 * sizeof(float) + 255) / 256 * 256;
  if (width <= 0 || height <= 0 || width > 16384 || height > 16384) return ANALYSER_ERR_INVALID_ARG;
  const size_t part_bytes = (size_t)kMeasureBlocks * 6 * sizeof(double);
  uint8_t* buf = nullptr;
  if (pool_malloc(reinterpret_cast<void**>(&buf), flow_bytes + part_bytes + 6 * sizeof(double)) != cudaSuccess)
    return ANALYSER_ERR_OOM;
  float* flow = reinterpret_cast<float*>(buf);
  double* d_part = reinterpret_cast<double*>(buf + flow_bytes);
  double* d_sums = reinterpret_cast<double*>(buf + flow_bytes + part_bytes);
  const cudaStream_t st = (cudaStream_t)stream;
  int rc = analyser_dense_flow(fp, width, height, frame_a, frame_b, pitch_bytes, flow, stream);
  double s[6] = {0, 0, 0, 0, 0, 0};
  if (rc == ANALYSER_OK) {
    const U8Plane I{frame_a, width, height, (int)pitch_bytes}, J{frame_b, width, height, (int)pitch_bytes};
    if (fp->fp64) flow_measure_kernel<double><<<kMeasureBlocks, kMeasureThreads, 0, st>>>(I, J, flow, d_part);
    else flow_measure_kernel<float><<<kMeasureBlocks, kMeasureThreads, 0, st>>>(I, J, flow, d_part);
    flow_sum_kernel<<<1, 32, 0, st>>>(d_part, kMeasureBlocks, d_sums);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(s, d_sums, sizeof(s), cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e != cudaSuccess || es != cudaSuccess) rc = ANALYSER_ERR_CUDA;
  } else {
    cudaStreamSynchronize(st);
  }
  pool_free(buf);
  if (rc != ANALYSER_OK) return rc;
  // FP64 finalisation (Sec. III.A): NCC from the sums, SWR, AMM, ACT
  const double n = (double)width * (double)height;
  const double c = n * s[5] - s[1] * s[2];
  const double vi = n * s[3] - s[1] * s[1];
  const double vj = n * s[4] - s[2] * s[2];
  double ncc;
  if (vi <= 0.0 && vj <= 0.0) ncc = 1.0;
  else if (vi <= 0.0 || vj <= 0.0) ncc = 0.0;
  else ncc = c / sqrt(vi * vj);
  const double om = 1.0 - ncc;
  out->ncc = ncc;
  out->swr = om > 0.0 ? om : 0.0;
  out->amm = s[0] / n;
  out->act = sqrt(out->amm * out->swr);
  for (int k = 0; k < 6; k++) out->sums[k] = s[k];
  return ANALYSER_OK;
}
