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
#include "va_kernels.cuh"

namespace va {

// ---------------------------------------------------------------------------
// packed-byte primitives
// ---------------------------------------------------------------------------

// c + sum over the 4 bytes of |a_k - b_k|
__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b, uint32_t c) {
#if defined(VA_SAD_DP4A)
  return __dp4a(__vabsdiffu4(a, b), 0x01010101u, c);
#elif defined(VA_SAD_VSAD)
  return __vsadu4(a, b) + c;
#else
  uint32_t d;
  asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
#endif
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// 4 bytes of row `row` starting at column x (any alignment), read clamp-to-edge.
__device__ __forceinline__ uint32_t load4_clamped(const uint8_t* row, int x, int w) {
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) v |= (uint32_t)row[clampi(x + k, 0, w - 1)] << (8 * k);
  return v;
}

// 4 bytes at column x of a row whose start is 4-byte aligned, any x alignment;
// the caller guarantees that bytes [x & ~3, (x & ~3) + 7] are readable.
__device__ __forceinline__ uint32_t load4_unaligned(const uint8_t* row, int x) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(row + (x & ~3));
  const uint32_t lo = __ldg(p), hi = __ldg(p + 1);
  return __funnelshift_r(lo, hi, 8 * (x & 3));
}

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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Refinement of every block of a tile at one pyramid level (block side S,
// radius RR), candidates v = 2*parent + d, |d| <= RR.
//  - each block's (S+2RR)-row search window in J is staged in shared memory
//    (clamp-to-edge);
//  - a thread owns one (block, dx, 4-pixel column q) with that I column in
//    registers (read from the tile staged in s_i) and slides down the window
//    rows, feeding the 2RR+1 dy candidates; the S/4 column partials are summed
//    with xor shuffles;
//  - a candidate's key is (cost << 8) | t with cost = SAD + lambda*|v|_1 and
//    t = (|v|_1 - min|v|_1)*25 + dy_i*5 + dx_i, which orders the block's 25
//    candidates exactly as (cost, |v|_1, vy, vx); the minimum goes to s_best.
// Afterwards s_vx/s_vy hold the level-l vectors.
template <int S, int RR, int NT, int NB, int TBX>
__device__ __forceinline__ void refine_level(const Plane Jl, const uint32_t* s_i, int bx0, int by0, int nbx, int nby,
                                             int lam, int* s_vx, int* s_vy, uint32_t* s_best, uint32_t* s_win,
                                             int tid) {
  static_assert(RR == 2, "relative candidate ranks assume radius 2");
  constexpr int NQ = S / 4, ND = 2 * RR + 1;
  constexpr int WR = S + 2 * RR, WW = (S + 2 * RR + 2) / 4 + 1;
  constexpr int IW = TBX * NQ;     // words per row of the staged I tile
  for (int task = tid; task < NB * WR; task += NT) {
    const int bl = task / WR, w = task - bl * WR;
    const int bx = bx0 + bl % TBX, by = by0 + bl / TBX;
    uint32_t* dst = s_win + task * WW;
    if (bx < nbx && by < nby) {
      const int xs = (bx * S + 2 * s_vx[bl] - RR) & ~3;
      const int yy = clampi(by * S + 2 * s_vy[bl] - RR + w, 0, Jl.h - 1);
      const uint8_t* row = Jl.p + (size_t)yy * Jl.pitch;
      if (xs >= 0 && xs + 4 * WW <= Jl.w) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(row + xs);
#pragma unroll
        for (int k = 0; k < WW; k++) dst[k] = __ldg(src + k);
      } else {
#pragma unroll
        for (int k = 0; k < WW; k++) dst[k] = load4_clamped(row, xs + 4 * k, Jl.w);
      }
    }
  }
  for (int i = tid; i < NB; i += NT) s_best[i] = 0xFFFFFFFFu;
  __syncthreads();
  // task = (block, 4-pixel column q): all ND x ND candidates of that column
  for (int base = 0; base < NB * NQ; base += NT) {
    const int it = base + tid;
    const int bl = it / NQ, q = it - bl * NQ;
    const int bxl = bl % TBX, byl = bl / TBX;
    const bool valid = it < NB * NQ && bx0 + bxl < nbx && by0 + byl < nby;
    uint32_t acc[ND][ND];     // [dx][dy]
#pragma unroll
    for (int a = 0; a < ND; a++)
#pragma unroll
      for (int d = 0; d < ND; d++) acc[a][d] = 0;
    int cx = 0, cy = 0;
    if (valid) {
      cx = 2 * s_vx[bl];
      cy = 2 * s_vy[bl];
      uint32_t icol[S];
      const uint32_t* ip = s_i + (byl * S) * IW + bxl * NQ + q;
#pragma unroll
      for (int i = 0; i < S; i++) icol[i] = ip[i * IW];
      const int xstart = (bx0 + bxl) * S + cx - RR;
      const int o = (xstart - (xstart & ~3)) + 4 * q;    // byte offset of dx = 0 in the window row
      const int wo = o >> 2, sh = (o & 3) * 8;
      const uint32_t* wp = s_win + bl * (WR * WW) + wo;
#pragma unroll
      for (int w = 0; w < WR; w++) {
        const uint32_t w0 = wp[w * WW], w1 = wp[w * WW + 1], w2 = wp[w * WW + 2];
        // the 5 dx alignments come from 3 consecutive words
        const uint64_t lo = ((uint64_t)w1 << 32) | w0;
        const uint64_t hi = ((uint64_t)w2 << 32) | w1;
        uint32_t jw[ND];
#pragma unroll
        for (int a = 0; a < ND; a++) {
          // byte offset o&3 + a within w0..w2
          const int bo = a;   // added to the runtime shift below
          jw[a] = (sh + 8 * bo < 32) ? (uint32_t)(lo >> (sh + 8 * bo)) : (uint32_t)(hi >> (sh + 8 * bo - 32));
        }
#pragma unroll
        for (int d = 0; d < ND; d++) {
          const int i = w - d;
          if (i >= 0 && i < S) {
#pragma unroll
            for (int a = 0; a < ND; a++) acc[a][d] = sad4(icol[i], jw[a], acc[a][d]);
          }
        }
      }
    }
#pragma unroll
    for (int off = NQ / 2; off >= 1; off >>= 1) {
#pragma unroll
      for (int a = 0; a < ND; a++)
#pragma unroll
        for (int d = 0; d < ND; d++) acc[a][d] += __shfl_xor_sync(0xFFFFFFFFu, acc[a][d], off);
    }
    // every column lane holds all sums: lane q finalises the dy rows d = q (mod NQ)
    uint32_t best = 0xFFFFFFFFu;
    if (valid) {
      const int n1min = max(abs(cx) - RR, 0) + max(abs(cy) - RR, 0);
#pragma unroll
      for (int d = 0; d < ND; d++) {
        if (d % NQ == q) {
          const int avy = abs(cy + d - RR);
#pragma unroll
          for (int a = 0; a < ND; a++) {
            const int n1 = abs(cx + a - RR) + avy;
            const uint32_t cost = acc[a][d] + (uint32_t)(lam * n1);
            const uint32_t t = (uint32_t)((n1 - n1min) * 25 + d * 5 + a);
            best = min(best, (cost << 8) | t);
          }
        }
      }
    }
#pragma unroll
    for (int off = NQ / 2; off >= 1; off >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, off));
    if (valid && q == 0) atomicMin(&s_best[bl], best);
  }
  __syncthreads();
  for (int i = tid; i < NB; i += NT) {
    const uint32_t k = s_best[i];
    if (k != 0xFFFFFFFFu) {
      const int t = (int)(k & 255u) % 25;
      s_vx[i] = 2 * s_vx[i] + (t % 5) - RR;
      s_vy[i] = 2 * s_vy[i] + (t / 5) - RR;
    }
  }
  __syncthreads();
}

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
  constexpr int G = S::G, NB = S::NB, NT = S::NT, WROWS = S::WROWS, WWORDS = S::WWORDS;
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
  __shared__ uint32_t s_win[NB * 20 * 6];
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

      const bool in_a = tid < S::NA;
      const int g = tid % G, bl = in_a ? tid / G : 0;
      const int bxl = bl % TBX, byl = bl / TBX;
      const bool active = in_a && (bx0 + bxl < nbx) && (by0 + byl < nby);
      const uint32_t i0 = iwin[(byl * 4 + 0) * TBX + bxl], i1 = iwin[(byl * 4 + 1) * TBX + bxl];
      const uint32_t i2 = iwin[(byl * 4 + 2) * TBX + bxl], i3 = iwin[(byl * 4 + 3) * TBX + bxl];
      const uint32_t lam18 = (uint32_t)lam << 18;
      // acc[j][c & 3] holds candidate c = dy - k (vy = c - R): it receives row k
      // of the block at window row dy, starts at k = 0 and completes at k = 3.
      uint32_t acc[4][4];
      uint32_t best[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        best[j] = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 4; k++) acc[j][k] = 0;
      }
      const uint32_t* wrow = jwin + (byl * 4) * WWORDS + bxl + g;
#pragma unroll
      for (int dy = 0; dy < 2 * R + 4; dy++) {
        const uint32_t wlo = wrow[dy * WWORDS], whi = wrow[dy * WWORDS + 1];
        uint32_t w[4];
        w[0] = wlo;
        w[1] = __funnelshift_r(wlo, whi, 8);
        w[2] = __funnelshift_r(wlo, whi, 16);
        w[3] = __funnelshift_r(wlo, whi, 24);
#pragma unroll
        for (int j = 0; j < 4; j++) {
          if (dy <= 2 * R) acc[j][dy & 3] = sad4(i0, w[j], 0u);
          if (dy >= 1 && dy - 1 <= 2 * R) acc[j][(dy - 1) & 3] = sad4(i1, w[j], acc[j][(dy - 1) & 3]);
          if (dy >= 2 && dy - 2 <= 2 * R) acc[j][(dy - 2) & 3] = sad4(i2, w[j], acc[j][(dy - 2) & 3]);
          if (dy >= 3) acc[j][(dy - 3) & 3] = sad4(i3, w[j], acc[j][(dy - 3) & 3]);
        }
        if (dy >= 3) {
          const int vy = dy - R - 3;
          const int avy = vy < 0 ? -vy : vy;
          const uint32_t bv = lam18 * (uint32_t)avy + (((uint32_t)avy << 12) | ((uint32_t)(vy + R) << 6));
#pragma unroll
          for (int j = 0; j < 4; j++) best[j] = min(best[j], (acc[j][(dy - 3) & 3] << 18) + bv);
        }
      }
      uint32_t tbest = 0xFFFFFFFFu;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int vx = -R + 4 * g + j;
        if (vx <= R) {
          const int avx = vx < 0 ? -vx : vx;
          const uint32_t a = (((uint32_t)(lam * avx)) << 18) + ((uint32_t)avx << 12) + (uint32_t)(vx + R);
          tbest = min(tbest, best[j] + a);
        }
      }
      if (active) atomicMin(&s_best32[bl], tbest);
      __syncthreads();
      for (int i = tid; i < NB; i += NT) {
        const uint32_t k = s_best32[i];
        s_vx[i] = (int)(k & 63u) - R;
        s_vy[i] = (int)((k >> 6) & 63u) - R;
      }
      __syncthreads();
    }

    // ---- phase B: refinement at levels L-2 .. 0 -------------------------------
    if (fast) {
      refine_level<8, 2, NT, NB, TBX>(jb.J[1], ti1, bx0, by0, nbx, nby, lam, s_vx, s_vy, s_best32, s_win, tid);
      refine_level<16, 2, NT, NB, TBX>(jb.J[0], ti0, bx0, by0, nbx, nby, lam, s_vx, s_vy, s_best32, s_win, tid);
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

    // ---- phase C: AMM sum and motion-compensated sums over the tile's pixels --
    {
      const Plane I0 = jb.I[0], J0 = jb.J[0];
      const int W = I0.w, H = I0.h;
      const int xs = bx0 * B0, ys = by0 * B0;
      const int xe = (bx0 + TBX >= nbx) ? W : (bx0 + TBX) * B0;
      const int ye = (by0 + TBY >= nby) ? H : (by0 + TBY) * B0;
      const int lim_w = min(J0.w, J0.pitch);
      uint32_t si = 0, sj = 0, sii = 0, sjj = 0, sij = 0, sab = 0;
      if (B0 == 16) {
        // columns of 16 pixels: TBX block columns plus a possible ragged strip
        constexpr int NCOL = TBX + 1, NGRP = NT / NCOL;
        const int col = tid % NCOL, grp = tid / NCOL;
        const int x = xs + 16 * col;
        if (grp < NGRP && x < xe) {
          const int bx = min(x >> 4, nbx - 1);
          const int nx = min(16, xe - x);          // pixels of this column (16 except a ragged edge)
          for (int y = ys + grp; y < ye; y += NGRP) {
            const int by = min(y >> 4, nby - 1);
            const int bl = (by - by0) * TBX + (bx - bx0);
            const int vx = s_vx[bl], vy = s_vy[bl];
            const uint8_t* irow = I0.p + (size_t)y * I0.pitch;
            const uint8_t* jrow = J0.p + (size_t)clampi(y + vy, 0, H - 1) * J0.pitch;
            const int xj = x + vx;
            uint32_t iv[4], jv[4];
            if (nx == 16) {
              uint4 q;
              if (fast && bx - bx0 < TBX && bx == (x >> 4) && y - ys < TBY * 16 && by == (y >> 4))
                q = *reinterpret_cast<const uint4*>(ti0 + ((y - ys) * TBX + (bx - bx0)) * 4);
              else
                q = __ldg(reinterpret_cast<const uint4*>(irow + x));
              iv[0] = q.x; iv[1] = q.y; iv[2] = q.z; iv[3] = q.w;
              if (xj >= 0 && xj + 19 <= lim_w - 1) {
                const uint32_t* p = reinterpret_cast<const uint32_t*>(jrow + (xj & ~3));
                const uint32_t a0 = __ldg(p), a1 = __ldg(p + 1), a2 = __ldg(p + 2), a3 = __ldg(p + 3), a4 = __ldg(p + 4);
                const int sh = 8 * (xj & 3);
                jv[0] = __funnelshift_r(a0, a1, sh);
                jv[1] = __funnelshift_r(a1, a2, sh);
                jv[2] = __funnelshift_r(a2, a3, sh);
                jv[3] = __funnelshift_r(a3, a4, sh);
              } else {
#pragma unroll
                for (int k = 0; k < 4; k++) jv[k] = load4_clamped(jrow, xj + 4 * k, W);
              }
            } else {
              // ragged right edge: bytes beyond W contribute zero to every sum
#pragma unroll
              for (int kw = 0; kw < 4; kw++) {
                uint32_t a = 0, c = 0;
#pragma unroll
                for (int kb = 0; kb < 4; kb++) {
                  const int k = 4 * kw + kb;
                  if (k < nx) {
                    a |= (uint32_t)irow[x + k] << (8 * kb);
                    c |= (uint32_t)jrow[clampi(xj + k, 0, W - 1)] << (8 * kb);
                  }
                }
                iv[kw] = a;
                jv[kw] = c;
              }
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
              si = __dp4a(iv[k], 0x01010101u, si);
              sj = __dp4a(jv[k], 0x01010101u, sj);
              sii = __dp4a(iv[k], iv[k], sii);
              sjj = __dp4a(jv[k], jv[k], sjj);
              sij = __dp4a(iv[k], jv[k], sij);
              sab = sad4(iv[k], jv[k], sab);
            }
          }
        }
      } else {
        const int nwx = (xe - xs + 3) >> 2;
        const int nrows = ye - ys;
        for (int idx = tid; idx < nrows * nwx; idx += NT) {
          const int ry = idx / nwx, wx = idx - ry * nwx;
          const int y = ys + ry, x = xs + 4 * wx;
          const int bx = min(x / B0, nbx - 1), by = min(y / B0, nby - 1);
          const int bl = (by - by0) * TBX + (bx - bx0);
          const int vx = s_vx[bl], vy = s_vy[bl];
          const uint8_t* irow = I0.p + (size_t)y * I0.pitch;
          const int yj = clampi(y + vy, 0, H - 1);
          const uint8_t* jrow = J0.p + (size_t)yj * J0.pitch;
          const int xj = x + vx;
          uint32_t iv, jv;
          if (x + 3 <= W - 1) {
            iv = __ldg(reinterpret_cast<const uint32_t*>(irow + x));
            jv = (xj >= 0 && xj + 7 <= lim_w - 1) ? load4_unaligned(jrow, xj) : load4_clamped(jrow, xj, J0.w);
          } else {
            iv = 0; jv = 0;
            for (int k = 0; x + k < W; k++) {
              iv |= (uint32_t)irow[x + k] << (8 * k);
              jv |= (uint32_t)jrow[clampi(xj + k, 0, W - 1)] << (8 * k);
            }
          }
          si = __dp4a(iv, 0x01010101u, si);
          sj = __dp4a(jv, 0x01010101u, sj);
          sii = __dp4a(iv, iv, sii);
          sjj = __dp4a(jv, jv, sjj);
          sij = __dp4a(iv, jv, sij);
          sab = sad4(iv, jv, sab);
        }
      }
      // AMM: one term per block of the tile, from the exact table
      uint32_t samm = 0;
      for (int i = tid; i < NB; i += NT) {
        const int bx = bx0 + i % TBX, by = by0 + i / TBX;
        if (bx < nbx && by < nby) {
          const int vx = s_vx[i], vy = s_vy[i];
          const int k = vx * vx + vy * vy;
          if (k <= b.qmax) samm += b.qtab[k];
          else atomicOr(b.status, 1);
          if (jb.vec) jb.vec[(size_t)by * nbx + bx] = make_short2((short)vx, (short)vy);
        }
      }
      unsigned long long v[kRecWords] = {si, sj, sii, sjj, sij, sab, samm};
#pragma unroll
      for (int k = 0; k < kRecWords; k++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], o);
      }
      const int warp = tid >> 5, lane = tid & 31;
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kRecWords; k++) s_red[warp][k] = v[k];
      }
      __syncthreads();
      if (tid < kRecWords) {
        unsigned long long a = 0;
        for (int w = 0; w < S::NW; w++) a += s_red[w][tid];
        atomicAdd(jb.rec + tid, a);
      }
      __syncthreads();
    }
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
