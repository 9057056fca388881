// CUDA kernels of the analyser's hot path, written for sm_103a.
//
//   downsample_kernel  one pyramid level for a batch of planes (frames and fields)
//   pair_kernel        one fused pass per (pair, tile of blocks):
//                        coarse exhaustive block search on the coarsest level,
//                        refinement at every finer level, AMM sum, motion-
//                        compensated NCC sums and the absolute residual
//
// The arithmetic follows Sec. III.A of the paper (motion field, AMM, warped
// NCC); the estimator is integer block matching on a box-filter pyramid
// (the paper's own flow estimator is dense inverse search; block matching with
// a motion cost is the reading implemented here and in the oracle).
// All sums are exact integers; no floating point runs on the device.
#include "va_device.cuh"

namespace va {

// ---------------------------------------------------------------------------
// pyramid: dst(x, y) = (a + b + c + d + 2) >> 2 over src rows 2y, 2y+1, cols 2x, 2x+1
// ---------------------------------------------------------------------------

__global__ void downsample_kernel(const DownJob* __restrict__ jobs) {
  const DownJob jb = jobs[blockIdx.z];
  const int dw = jb.src.w / 2, dh = jb.src.h / 2;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int xg = blockIdx.x * blockDim.x + threadIdx.x;   // group of 4 output pixels
  const int x = xg * 4;
  if (y >= dh || x >= dw) return;
  const uint8_t* r0 = jb.src.p + (size_t)(2 * y) * jb.src.pitch;
  const uint8_t* r1 = r0 + jb.src.pitch;
  uint8_t* out = jb.dst + (size_t)y * jb.dst_pitch;
  if (x + 4 <= dw) {
    // 8 source bytes per row; src views are 8-byte aligned at even x groups
    const uint2 a = *reinterpret_cast<const uint2*>(r0 + 2 * x);
    const uint2 c = *reinterpret_cast<const uint2*>(r1 + 2 * x);
    const unsigned long long A = ((unsigned long long)a.y << 32) | a.x;
    const unsigned long long C = ((unsigned long long)c.y << 32) | c.x;
    const unsigned long long M = 0x00FF00FF00FF00FFull;
    // 16-bit lanes: (a0 + a1 + c0 + c1 + 2) for each of the 4 output pixels
    const unsigned long long s = (A & M) + ((A >> 8) & M) + (C & M) + ((C >> 8) & M) + 0x0002000200020002ull;
    const unsigned long long q = (s >> 2) & M;
    const uint32_t lo = (uint32_t)q, hi = (uint32_t)(q >> 32);
    *reinterpret_cast<uint32_t*>(out + x) = __byte_perm(lo, hi, 0x6420);
  } else {
    for (int k = x; k < dw; k++) {
      const int s = r0[2 * k] + r0[2 * k + 1] + r1[2 * k] + r1[2 * k + 1] + 2;
      out[k] = (uint8_t)(s >> 2);
    }
  }
}

// ---------------------------------------------------------------------------
// pyramid levels 1-2 of frames and fields in one pass over level 0
// ---------------------------------------------------------------------------

// (a + b + c + d + 2) >> 2 for the four 2x2 boxes of two 8-byte rows
__device__ __forceinline__ uint32_t box4(unsigned long long A, unsigned long long C) {
  const unsigned long long M = 0x00FF00FF00FF00FFull;
  const unsigned long long s = (A & M) + ((A >> 8) & M) + (C & M) + ((C >> 8) & M) + 0x0002000200020002ull;
  const unsigned long long q = (s >> 2) & M;
  return __byte_perm((uint32_t)q, (uint32_t)(q >> 32), 0x6420);
}

// 8 output bytes (two words) from two 16-byte rows
__device__ __forceinline__ uint2 box8(uint4 a, uint4 c) {
  const unsigned long long A0 = ((unsigned long long)a.y << 32) | a.x, A1 = ((unsigned long long)a.w << 32) | a.z;
  const unsigned long long C0 = ((unsigned long long)c.y << 32) | c.x, C1 = ((unsigned long long)c.w << 32) | c.z;
  return make_uint2(box4(A0, C0), box4(A1, C1));
}

__device__ __forceinline__ uint32_t box4w(uint2 a, uint2 c) {
  return box4(((unsigned long long)a.y << 32) | a.x, ((unsigned long long)c.y << 32) | c.x);
}

__device__ __forceinline__ int box_px(const uint8_t* r0, const uint8_t* r1, int x) {
  return (r0[2 * x] + r0[2 * x + 1] + r1[2 * x] + r1[2 * x + 1] + 2) >> 2;
}

// A thread covers level-0 rows 8Y..8Y+7 and columns 16X..16X+15.
__device__ __forceinline__ void pyramid_tile(const PyrJob& jb, int X, int Y) {
  const int W = jb.w, H = jb.h, x0 = 16 * X, y0 = 8 * Y;
  if (x0 >= W || y0 >= H) return;
  const int w1 = W / 2, w2 = W / 4, h1 = H / 2, h2 = H / 4, g1 = H / 4, g2 = H / 8;   // frame / field sizes
  const bool two = jb.out[1] != nullptr;
  if (x0 + 16 <= W) {
    uint4 r[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
      r[i] = (y0 + i < H) ? __ldg(reinterpret_cast<const uint4*>(jb.l0 + (size_t)(y0 + i) * jb.l0_pitch + x0))
                          : make_uint4(0, 0, 0, 0);
    uint2 f1[4], u1[2], l1[2];
#pragma unroll
    for (int k = 0; k < 4; k++) f1[k] = box8(r[2 * k], r[2 * k + 1]);
#pragma unroll
    for (int j = 0; j < 2; j++) {
      u1[j] = box8(r[4 * j], r[4 * j + 2]);
      l1[j] = box8(r[4 * j + 1], r[4 * j + 3]);
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (4 * Y + k < h1) *reinterpret_cast<uint2*>(jb.out[0] + (size_t)(4 * Y + k) * jb.pitch[0] + 8 * X) = f1[k];
#pragma unroll
    for (int j = 0; j < 2; j++)
      if (2 * Y + j < g1) {
        *reinterpret_cast<uint2*>(jb.out[2] + (size_t)(2 * Y + j) * jb.pitch[2] + 8 * X) = u1[j];
        *reinterpret_cast<uint2*>(jb.out[4] + (size_t)(2 * Y + j) * jb.pitch[4] + 8 * X) = l1[j];
      }
    if (two) {
#pragma unroll
      for (int m = 0; m < 2; m++)
        if (2 * Y + m < h2)
          *reinterpret_cast<uint32_t*>(jb.out[1] + (size_t)(2 * Y + m) * jb.pitch[1] + 4 * X) = box4w(f1[2 * m], f1[2 * m + 1]);
      if (Y < g2) {
        *reinterpret_cast<uint32_t*>(jb.out[3] + (size_t)Y * jb.pitch[3] + 4 * X) = box4w(u1[0], u1[1]);
        *reinterpret_cast<uint32_t*>(jb.out[5] + (size_t)Y * jb.pitch[5] + 4 * X) = box4w(l1[0], l1[1]);
      }
    }
    return;
  }
  // ragged right edge: pixel by pixel, level 1 first, level 2 from the stored level 1
  // (the same thread wrote the level-1 pixels it reads back)
  const uint8_t* row[8];
#pragma unroll
  for (int i = 0; i < 8; i++) row[i] = jb.l0 + (size_t)min(y0 + i, H - 1) * jb.l0_pitch;
  for (int x = x0 / 2; x < min(x0 / 2 + 8, w1); x++) {
    for (int k = 0; k < 4; k++)
      if (4 * Y + k < h1) jb.out[0][(size_t)(4 * Y + k) * jb.pitch[0] + x] = (uint8_t)box_px(row[2 * k], row[2 * k + 1], x);
    for (int j = 0; j < 2; j++)
      if (2 * Y + j < g1) {
        jb.out[2][(size_t)(2 * Y + j) * jb.pitch[2] + x] = (uint8_t)box_px(row[4 * j], row[4 * j + 2], x);
        jb.out[4][(size_t)(2 * Y + j) * jb.pitch[4] + x] = (uint8_t)box_px(row[4 * j + 1], row[4 * j + 3], x);
      }
  }
  if (!two) return;
  for (int x = x0 / 4; x < min(x0 / 4 + 4, w2); x++) {
    for (int m = 0; m < 2; m++)
      if (2 * Y + m < h2) {
        const uint8_t* a = jb.out[0] + (size_t)(4 * Y + 2 * m) * jb.pitch[0];
        jb.out[1][(size_t)(2 * Y + m) * jb.pitch[1] + x] = (uint8_t)box_px(a, a + jb.pitch[0], x);
      }
    if (Y < g2) {
      const uint8_t* a = jb.out[2] + (size_t)(2 * Y) * jb.pitch[2];
      jb.out[3][(size_t)Y * jb.pitch[3] + x] = (uint8_t)box_px(a, a + jb.pitch[2], x);
      const uint8_t* b = jb.out[4] + (size_t)(2 * Y) * jb.pitch[4];
      jb.out[5][(size_t)Y * jb.pitch[5] + x] = (uint8_t)box_px(b, b + jb.pitch[4], x);
    }
  }
}

// The 256-bin histogram of the thread's level-0 pixels, added into the CTA's
// shared bins and then into the frame's bins.  Called by every thread.
__device__ __forceinline__ void histogram_tile(const PyrJob& jb, int X, int Y, uint32_t* s_hist, int tid) {
  for (int i = tid; i < 256; i += 128) s_hist[i] = 0;
  __syncthreads();
  const int W = jb.w, H = jb.h, x0 = 16 * X, y0 = 8 * Y;
  if (x0 < W && y0 < H) {
    const int nx = min(16, W - x0);
    for (int i = 0; i < 8 && y0 + i < H; i++) {
      const uint8_t* row = jb.l0 + (size_t)(y0 + i) * jb.l0_pitch + x0;
      if (nx == 16) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(row));
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 16; k++) atomicAdd(&s_hist[(w[k >> 2] >> (8 * (k & 3))) & 255u], 1u);
      } else {
        for (int k = 0; k < nx; k++) atomicAdd(&s_hist[row[k]], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < 256; i += 128)
    if (s_hist[i]) atomicAdd(&jb.hist[i], s_hist[i]);
}

__global__ void __launch_bounds__(128, 10) pyramid_kernel(const PyrJob* __restrict__ jobs) {
  const PyrJob jb = jobs[blockIdx.z];
  pyramid_tile(jb, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

// Per-frame level-0 histograms of the jobs whose `hist` is set (same grid as
// pyramid_kernel; launched only when histograms are wanted).
__global__ void __launch_bounds__(128) histogram_kernel(const PyrJob* __restrict__ jobs) {
  __shared__ uint32_t s_hist[256];
  const PyrJob& jb = jobs[blockIdx.z];
  if (!jb.hist) return;   // CTA-uniform
  histogram_tile(jb, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y, s_hist,
                 threadIdx.y * blockDim.x + threadIdx.x);
}

cudaError_t launch_pyramid(const PyrJob* d_jobs, int njobs, int max_w, int max_h, bool histograms, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 blk(32, 4);
  dim3 grd(((max_w + 15) / 16 + blk.x - 1) / blk.x, ((max_h + 7) / 8 + blk.y - 1) / blk.y, njobs);
  pyramid_kernel<<<grd, blk, 0, st>>>(d_jobs);
  if (histograms) histogram_kernel<<<grd, blk, 0, st>>>(d_jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small transfers between device memory and page-locked host memory, done by
// the SMs (the GPU addresses page-locked memory directly): per-wave descriptors
// and results that must not queue behind bulk frame copies on the copy engines
// ---------------------------------------------------------------------------

__global__ void copy_words_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_copy_words(const void* src, void* dst, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  const size_t n = (bytes + 15) / 16;
  const size_t blocks = (n + 255) / 256;
  copy_words_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(static_cast<const uint4*>(src),
                                                                                static_cast<uint4*>(dst), n);
  return cudaGetLastError();
}

cudaError_t launch_downsample(const DownJob* d_jobs, int njobs, int max_dst_h, int max_dst_w, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 blk(32, 8);
  dim3 grd((max_dst_w / 4 + 1 + blk.x - 1) / blk.x, (max_dst_h + blk.y - 1) / blk.y, njobs);
  downsample_kernel<<<grd, blk, 0, st>>>(d_jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fused pair kernel
// ---------------------------------------------------------------------------

template <int R, int TBX, int TBY>
struct PairShape {
  static constexpr int G = (2 * R + 4) / 4;       // vx groups of 4 candidates
  static constexpr int NB = TBX * TBY;            // blocks per tile
  static constexpr int NA = NB * G;               // threads busy in the coarse phase
  // whole warps, and at least 10 per 32 blocks so that the refinement tasks
  // (blocks x 5 dx x 4 columns at level 0, x 2 columns at level 1) fill 2 and 1 rounds
  static constexpr int NT0 = (NA + 31) / 32 * 32;
  static constexpr int NT = NT0 > NB * 10 ? NT0 : NB * 10;
  static constexpr int WROWS = TBY * kCoarseSide + 2 * R;
  static constexpr int WWORDS = TBX + G;
  static constexpr int NW = (NT + 31) / 32;
};

template <int R, int TBX, int TBY>
__global__ void __launch_bounds__(PairShape<R, TBX, TBY>::NT, 3)
pair_kernel(const PairBatch b) {
  using S = PairShape<R, TBX, TBY>;
  constexpr int NB = S::NB, NT = S::NT, WROWS = S::WROWS, WWORDS = S::WWORDS;
  static_assert(R % 4 == 0 && R <= 31, "coarse radius");

  // inputs of a tile, double-buffered: the next tile's are copied (cp.async)
  // while the current one computes
  __shared__ __align__(16) uint32_t s_jwin[2][WROWS * WWORDS];
  __shared__ __align__(16) uint32_t s_iw[2][TBY * kCoarseSide * TBX];
  __shared__ uint32_t s_best32[NB];
  __shared__ unsigned long long s_best64[NB];
  __shared__ int s_vx[NB], s_vy[NB];
  __shared__ unsigned long long s_red[S::NW][kRecWords];
  __shared__ PairJob s_job[2];
  // refinement windows: level side 16 with radius 2 is the largest fast case
  __shared__ __align__(16) uint32_t s_win[NB * kRefineWinWords];
  // I tiles of levels 0 and 1 (fast path: 3 levels, radius 2), staged asynchronously
  __shared__ __align__(16) uint32_t s_i0[2][TBY * 16 * TBX * 4];
  __shared__ __align__(16) uint32_t s_i1[2][TBY * 8 * TBX * 2];

  const int tid = threadIdx.x;
  const int L = b.cfg.levels;
  const int B0 = kCoarseSide << (L - 1);
  const int lam = b.cfg.lambda;
  const int rr = b.cfg.refine;
  const int side = 2 * rr + 1, ncand = side * side;

  const bool fast = (L == 3 && rr == 2);
  auto load_job = [&](int item, int slot) {
    int lo = 0, hi = b.njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.jobs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    static_assert(sizeof(PairJob) % 4 == 0, "job copy");
    const int* src = reinterpret_cast<const int*>(b.jobs + lo);
    int* dst = reinterpret_cast<int*>(&s_job[slot]);
    for (int i = tid; i < (int)(sizeof(PairJob) / 4); i += NT) dst[i] = src[i];
  };
  auto tile_of = [&](const PairJob& jb, int item, int& bx0, int& by0) {
    const int local = item - jb.item_begin;
    bx0 = (local % jb.tiles_x) * TBX;
    by0 = (local / jb.tiles_x) * TBY;
  };
  // asynchronous copies of a tile's inputs: the coarse search window (words
  // inside the coarsest level; the others are filled clamp-to-edge before use),
  // the coarse block rows and, for the default estimator, the level-0 and
  // level-1 I tiles
  auto prefetch = [&](int item, int slot) {
    const PairJob& jb = s_job[slot];
    int bx0, by0;
    tile_of(jb, item, bx0, by0);
    const Plane J2 = jb.J[L - 1], I2 = jb.I[L - 1];
    const int Xw0 = bx0 * kCoarseSide - R, Yw0 = by0 * kCoarseSide - R;
    for (int c = tid; c < WROWS * WWORDS; c += NT) {
      const int wy = c / WWORDS, wx = c - wy * WWORDS;
      const int y = Yw0 + wy, x = Xw0 + 4 * wx;
      if (y >= 0 && y < J2.h && x >= 0 && x + 3 <= J2.w - 1)
        cp_async4(&s_jwin[slot][c], J2.p + (size_t)y * J2.pitch + x);
    }
    for (int c = tid; c < TBY * kCoarseSide * TBX; c += NT) {
      const int r = c / TBX, k = c - r * TBX;
      if (bx0 + k < jb.nbx && by0 + r / kCoarseSide < jb.nby)
        cp_async4(&s_iw[slot][c], I2.p + (size_t)(by0 * kCoarseSide + r) * I2.pitch + (bx0 + k) * kCoarseSide);
    }
    if (fast) {
      for (int c = tid; c < TBY * 16 * TBX; c += NT) {
        const int r = c / TBX, k = c - r * TBX;
        if (bx0 + k < jb.nbx && by0 + r / 16 < jb.nby)
          cp_async16(&s_i0[slot][c * 4], jb.I[0].p + (size_t)(by0 * 16 + r) * jb.I[0].pitch + (bx0 + k) * 16);
      }
      for (int c = tid; c < TBY * 8 * TBX; c += NT) {
        const int r = c / TBX, k = c - r * TBX;
        if (bx0 + k < jb.nbx && by0 + r / 8 < jb.nby)
          cp_async8(&s_i1[slot][c * 2], jb.I[1].p + (size_t)(by0 * 8 + r) * jb.I[1].pitch + (bx0 + k) * 8);
      }
    }
    cp_async_commit();
  };

  int slot = 0;
  if ((int)blockIdx.x < b.nitems) {
    load_job(blockIdx.x, 0);
    __syncthreads();
    prefetch(blockIdx.x, 0);
  }
  for (int item = blockIdx.x; item < b.nitems; item += gridDim.x, slot ^= 1) {
    const int next = item + gridDim.x;
    if (next < b.nitems) load_job(next, slot ^ 1);
    __syncthreads();
    if (next < b.nitems) {
      prefetch(next, slot ^ 1);
      cp_async_wait_group1();
    } else {
      cp_async_wait_all();
    }
    const PairJob& jb = s_job[slot];
    int bx0, by0;
    tile_of(jb, item, bx0, by0);
    const int nbx = jb.nbx, nby = jb.nby;
    uint32_t* const jwin = s_jwin[slot];
    const uint32_t* const iwin = s_iw[slot];
    const uint32_t* const ti0 = s_i0[slot];
    const uint32_t* const ti1 = s_i1[slot];

    // ---- phase A: exhaustive search on the coarsest level --------------------
    {
      const Plane J2 = jb.J[L - 1];
      const int Xw0 = bx0 * kCoarseSide - R, Yw0 = by0 * kCoarseSide - R;
      if (Xw0 < 0 || Yw0 < 0 || Xw0 + 4 * WWORDS > J2.w || Yw0 + WROWS > J2.h) {
        // window words outside the coarsest level: clamp-to-edge
        for (int c = tid; c < WROWS * WWORDS; c += NT) {
          const int wy = c / WWORDS, wx = c - wy * WWORDS;
          const int y = Yw0 + wy, x = Xw0 + 4 * wx;
          if (!(y >= 0 && y < J2.h && x >= 0 && x + 3 <= J2.w - 1))
            jwin[c] = load4_clamped(J2.p + (size_t)clampi(y, 0, J2.h - 1) * J2.pitch, x, J2.w);
        }
      }
      for (int i = tid; i < NB; i += NT) s_best32[i] = 0xFFFFFFFFu;
      __syncthreads();

      coarse_phase<R, TBX, TBY, NT, false>(jwin, iwin, bx0, by0, nbx, nby, lam, b.cfg.key_mul, s_best32, s_vx, s_vy,
                                             tid);
    }

    // ---- phase B: refinement at levels L-2 .. 0 -------------------------------
    uint32_t part[6] = {0, 0, 0, 0, 0, 0};
    if (fast) {
      refine_level<8, 2, NT, NB, TBX, false>(jb.J[1], ti1, bx0, by0, nbx, nby, lam, s_vx, s_vy, s_win, part, tid);
      refine_level<16, 2, NT, NB, TBX, true>(jb.J[0], ti0, bx0, by0, nbx, nby, lam, s_vx, s_vy, s_win, part, tid);
    } else {
      for (int l = L - 2; l >= 0; l--) {
        const Plane Il = jb.I[l], Jl = jb.J[l];
        const int s = B0 >> l;
        const int lim_w = min(Jl.w, Jl.pitch);
        for (int i = tid; i < NB; i += NT) s_best64[i] = ~0ull;
        __syncthreads();
        for (int t = tid; t < NB * ncand; t += NT) {
          const int bl = t / ncand, c = t - bl * ncand;
          const int bxl = bl % TBX, byl = bl / TBX;
          const int bx = bx0 + bxl, by = by0 + byl;
          if (bx >= nbx || by >= nby) continue;
          const int vx = 2 * s_vx[bl] + (c % side) - rr;
          const int vy = 2 * s_vy[bl] + (c / side) - rr;
          const int x0 = bx * s, y0 = by * s;
          const int xj = x0 + vx;
          const bool fastj = (xj >= 0) && (xj + s + 3 <= lim_w - 1) && (y0 + vy >= 0) && (y0 + vy + s - 1 <= Jl.h - 1);
          uint32_t sad = 0;
          for (int y = 0; y < s; y++) {
            const uint8_t* irow = Il.p + (size_t)(y0 + y) * Il.pitch + x0;
            const int yj = clampi(y0 + y + vy, 0, Jl.h - 1);
            const uint8_t* jrow = Jl.p + (size_t)yj * Jl.pitch;
            for (int x = 0; x < s; x += 4) {
              const uint32_t iv = __ldg(reinterpret_cast<const uint32_t*>(irow + x));
              const uint32_t jv = fastj ? load4_unaligned(jrow, xj + x) : load4_clamped(jrow, xj + x, Jl.w);
              sad = sad4(iv, jv, sad);
            }
          }
          const int n1 = abs(vx) + abs(vy);
          const unsigned long long key = ((unsigned long long)(sad + (uint32_t)(lam * n1)) << 32) |
                                         ((unsigned long long)n1 << 20) | ((unsigned long long)(vy + 512) << 10) |
                                         (unsigned long long)(vx + 512);
          atomicMin(&s_best64[bl], key);
        }
        __syncthreads();
        for (int i = tid; i < NB; i += NT) {
          const unsigned long long k = s_best64[i];
          if (k != ~0ull) {
            s_vx[i] = (int)(k & 1023ull) - 512;
            s_vy[i] = (int)((k >> 10) & 1023ull) - 512;
          }
        }
        __syncthreads();
      }
    }

    __syncthreads();   // every block's vector is read below
    sums_phase<TBX, TBY, NT>(b, jb, bx0, by0, B0, fast, part, s_vx, s_vy, s_red, tid);
  }
}

// ---------------------------------------------------------------------------
// dispatch over the compiled (radius, tile) variants
// ---------------------------------------------------------------------------

#define VA_TILES(X, R) X(R, 8, 4) X(R, 4, 4) X(R, 8, 2) X(R, 16, 2) X(R, 4, 8)
#define VA_RADII(X) VA_TILES(X, 8) VA_TILES(X, 16) VA_TILES(X, 24)

bool pair_tile_supported(int radius, int tbx, int tby) {
#define VA_CASE(R_, X_, Y_) if (radius == R_ && tbx == X_ && tby == Y_) return true;
  VA_RADII(VA_CASE)
#undef VA_CASE
  return false;
}

int pair_threads(int radius, int tbx, int tby) {
#define VA_CASE(R_, X_, Y_) if (radius == R_ && tbx == X_ && tby == Y_) return PairShape<R_, X_, Y_>::NT;
  VA_RADII(VA_CASE)
#undef VA_CASE
  return 0;
}

int pair_blocks_per_sm(int radius, int tbx, int tby) {
  int n = 0;
#define VA_CASE(R_, X_, Y_)                                                                        \
  if (radius == R_ && tbx == X_ && tby == Y_) {                                                    \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_kernel<R_, X_, Y_>,                 \
                                                      PairShape<R_, X_, Y_>::NT, 0) != cudaSuccess) \
      n = 1;                                                                                       \
    return n;                                                                                      \
  }
  VA_RADII(VA_CASE)
#undef VA_CASE
  return 1;
}

cudaError_t launch_pairs(const PairBatch& b, int tbx, int tby, int grid, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
#define VA_CASE(R_, X_, Y_)                                                           \
  if (b.cfg.radius == R_ && tbx == X_ && tby == Y_) {                                 \
    pair_kernel<R_, X_, Y_><<<grid, PairShape<R_, X_, Y_>::NT, 0, st>>>(b);           \
    return cudaGetLastError();                                                        \
  }
  VA_RADII(VA_CASE)
#undef VA_CASE
  return cudaErrorInvalidValue;
}

}  // namespace va
