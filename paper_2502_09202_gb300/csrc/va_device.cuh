// Device-side building blocks shared by the pair kernels (va_kernels.cu).
#pragma once
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

// Exhaustive search of every block of a tile on the coarsest level (block
// side 4, radius R): a thread owns one block and 4 consecutive vx candidates
// and slides down the staged window rows; candidate keys are
// (cost << 18) | (|v|_1 << 12) | (vy + R) << 6 | (vx + R), i.e. the order
// (cost, |v|_1, vy, vx).  Expects s_best32 set to all ones and a barrier before
// the call; leaves the coarse vectors in s_vx/s_vy (after a barrier).
template <int R, int TBX, int TBY, int NT>
__device__ __forceinline__ void coarse_phase(const uint32_t* jwin, const uint32_t* iwin, int bx0, int by0, int nbx,
                                         int nby, int lam, uint32_t* s_best32, int* s_vx, int* s_vy, int tid) {
  constexpr int G = (2 * R + 4) / 4, NB = TBX * TBY, NA = NB * G, WWORDS = TBX + G;
  const bool in_a = tid < NA;
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

// Motion-compensated sums over the tile's pixels (the blocks' pixels and, for
// edge tiles, the border strips beyond the block grid, which use the nearest
// block's vector), the AMM term of every block, the optional motion dump, and
// the CTA reduction into the pair's accumulators.  Level-0 I rows come from the
// staged tile when `fast` (default estimator), otherwise from global memory.
template <int TBX, int TBY, int NT>
__device__ __forceinline__ void sums_phase(const PairBatch& b, const PairJob& jb, int bx0, int by0, int B0, bool fast,
                                           const uint32_t* ti0, const int* s_vx, const int* s_vy,
                                           unsigned long long (*s_red)[kRecWords], int tid) {
  constexpr int NB = TBX * TBY, NW = NT / 32;
  const int nbx = jb.nbx, nby = jb.nby;
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
    for (int w = 0; w < NW; w++) a += s_red[w][tid];
    atomicAdd(jb.rec + tid, a);
  }
  __syncthreads();
}

}  // namespace va
