// Device-side building blocks shared by the pair kernels (va_kernels.cu).
#pragma once
#include "va_kernels.cuh"

namespace va {

// ---------------------------------------------------------------------------
// barrier of the threads running a tile's code (the whole CTA)
// ---------------------------------------------------------------------------
struct CtaBarrier {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// ---------------------------------------------------------------------------
// packed-byte primitives
// ---------------------------------------------------------------------------

// c + sum over the 4 bytes of |a_k - b_k|.  PTX vabsdiff4 with accumulate is
// the fastest packed sequence measured on GB300 in register-only loops whose
// operands cannot be shared or hoisted (75 T |a-b|/s against 53 for the sum of
// absolute differences intrinsic plus an add and 47 for vabsdiff4 + dp4a; mixing
// sequences across chains gains nothing), and in the pair kernels (8.5 against
// 9.3 us per 1080p frame pair).  VA_SAD_VSAD builds the intrinsic variant.
__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b, uint32_t c) {
#if defined(VA_SAD_VSAD)
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

// Shared-memory window of one block at a refinement level of block side S
// (radius 2): WR rows of RW words copied in CB-byte pieces from the CB-byte
// boundary at or before the window's first byte (candidate dx = -2); RW * 4
// covers that offset (< CB) plus the S + 4 bytes the candidates reach.  Every
// block owns one region of kRefineWinWords words that both levels use, so a
// block's lanes never touch another block's window and the levels need no CTA
// barrier.  Regions start 4 banks apart (164 = 4 mod 32): the 8 blocks of a
// warp read their windows' rows from disjoint banks.
constexpr int kRefineWinWords = 164;
template <int S>
struct RefineWin;
template <>
struct RefineWin<16> {
  static constexpr int WR = 20, RW = 8, CB = 8;
};
template <>
struct RefineWin<8> {
  static constexpr int WR = 12, RW = 4, CB = 4;
};

// Lane layout of one block at a refinement level: LPB lanes per block, each
// with WPL consecutive 4-pixel words of a row and RT rows of the block.
template <int S, int LPB>
struct RefineLanes {
  static constexpr int NQ = S / 4;                       // words per block row
  static constexpr int WPL = (S == 16 && LPB == 2) ? 2 : 1;
  static constexpr int CL = NQ / WPL;                    // column lanes
  static constexpr int H = LPB / CL;                     // row slices
  static constexpr int RT = S / H;                       // rows per lane
  static_assert(CL * WPL == NQ && CL * H == LPB, "lane layout");
};

// Refinement of every block of a tile at one pyramid level (block side S,
// radius RR), candidates v = 2*parent + d, |d| <= RR (Sec. III.A, coarse to
// fine block matching).  LPB lanes own a block (lanes LPB*bl .. LPB*bl+LPB-1):
//  - they copy the block's window of J into shared memory (cp.async, the
//    lanes of a row together; clamp-to-edge loads where the window leaves the
//    image horizontally, row indices clamped), so a level needs no CTA barrier;
//  - a lane covers WPL 4-pixel words of RT rows of the block, keeps those I
//    words in registers and slides down the window rows, feeding all 25
//    (dx, dy) candidates; the lanes' partial sums are added with xor shuffles;
//  - a candidate's key is (cost << 8) + rank with cost = SAD + lambda*|v|_1 and
//    rank = (|v|_1 - min|v|_1)*25 + dy_i*5 + dx_i, which orders the block's 25
//    candidates exactly as (cost, |v|_1, vy, vx).
// Afterwards s_vx/s_vy hold the level-l vectors (visible to the block's own
// lanes; other threads need a CTA barrier first).  With SUMS the lanes then
// add the motion-compensated sums of their pixels (I words in registers,
// warped J from the window) to part[] =
// {sum I, sum J, sum I^2, sum J^2, sum IJ, sum |I-J|}.
//
// PHASE 0 does the whole level, the parent vector of a block read from
// s_vx/s_vy.  PHASE 1 only issues the window copies and PHASE 2 only computes
// (the caller commits and waits in between), both with the parent passed in
// (pvx, pvy): a kernel can then issue the first level's copies together with
// its other loads and wait once.
// With IGLOBAL the I words come from the level's plane in global memory
// (Ig, one or two words per lane and row) instead of a staged tile s_i; they
// are loaded with the window copies and kept in registers (*icp carries them
// from PHASE 1 to PHASE 2).
struct ICols {
  uint32_t v[2][16];
};
template <int S, int RR, int NT, int NB, int TBX, bool SUMS, int PHASE = 0, int LPB = 4, bool IGLOBAL = false,
          int WINW = kRefineWinWords>
__device__ __forceinline__ void refine_level(const Plane Jl, const uint32_t* s_i, int bx0, int by0, int nbx, int nby,
                                             int lam, int* s_vx, int* s_vy, uint32_t* s_win, uint32_t (&part)[6],
                                             int tid, int pvx = 0, int pvy = 0, const Plane Ig = Plane{},
                                             ICols* icp = nullptr) {
  static_assert(RR == 2, "candidate ranks and window shapes assume radius 2");
  using Wn = RefineWin<S>;
  using Ln = RefineLanes<S, LPB>;
  constexpr int NQ = Ln::NQ, WPL = Ln::WPL, CL = Ln::CL, RT = Ln::RT;
  constexpr int IW = TBX * NQ;                       // words per row of the staged I tile
  static_assert(Wn::WR % LPB == 0, "rows split evenly over a block's lanes");
  static_assert(NT % 32 == 0 && NT >= NB * LPB && (NB * LPB) % 32 == 0, "one task per thread, whole warps");
  if ((tid & ~31) >= NB * LPB) return;   // warps without a block (warp-uniform)
  const int bl = tid / LPB, t = tid % LPB;
  const int q0 = (t % CL) * WPL, h = t / CL;
  const int bxl = bl % TBX, byl = bl / TBX;
  const bool valid = bx0 + bxl < nbx && by0 + byl < nby;
  const int cx = 2 * (PHASE == 0 ? s_vx[bl] : pvx), cy = 2 * (PHASE == 0 ? s_vy[bl] : pvy);
  const int xw = (bx0 + bxl) * S + cx - RR;   // image position of candidate (-RR, -RR)
  const int yw = (by0 + byl) * S + cy - RR;
  constexpr int CB = Wn::CB, CPR = 4 * Wn::RW / CB;   // bytes per copy, copies per window row
  static_assert(CPR % LPB == 0 || LPB % CPR == 0, "copies split evenly over a block's lanes");
  const int xa = xw & ~(CB - 1), s8 = 8 * (xw & 3);
  const int off = (xw - xa) >> 2;             // word of the window's first byte
  static_assert(Wn::WR * Wn::RW <= WINW, "window fits the block's region");
  uint32_t* const win = s_win + bl * WINW;

  // ---- staging ----------------------------------------------------------------
  // Lane t copies pieces t, t + LPB, ... of every window row (a warp
  // instruction reads contiguous bytes per block).  Inside the image the row
  // address advances by the pitch; rows above or below it are clamped; a
  // window leaving the image horizontally is read byte by byte, clamp-to-edge.
  if (PHASE != 2 && valid) {
    auto copy = [&](uint32_t* d, const uint8_t* g) {
      if constexpr (CB == 8) cp_async8(d, g);
      else cp_async4(d, g);
    };
    if (xa >= 0 && xa + 4 * Wn::RW <= Jl.w) {
      if (yw >= 0 && yw + Wn::WR <= Jl.h) {
        const uint8_t* row = Jl.p + (size_t)yw * Jl.pitch + xa;
#pragma unroll 4
        for (int r = 0; r < Wn::WR; r++) {
#pragma unroll
          for (int c = 0; c < CPR; c += LPB)
            if (c + t < CPR) copy(win + r * Wn::RW + (c + t) * (CB / 4), row + (c + t) * CB);
          row += Jl.pitch;
        }
      } else {
#pragma unroll 4
        for (int r = 0; r < Wn::WR; r++) {
          const uint8_t* row = Jl.p + (size_t)clampi(yw + r, 0, Jl.h - 1) * Jl.pitch + xa;
#pragma unroll
          for (int c = 0; c < CPR; c += LPB)
            if (c + t < CPR) copy(win + r * Wn::RW + (c + t) * (CB / 4), row + (c + t) * CB);
        }
      }
    } else {
#pragma unroll 1
      for (int k = 0; k < Wn::WR / LPB; k++) {
        const int r = t + LPB * k;
        const uint8_t* row = Jl.p + (size_t)clampi(yw + r, 0, Jl.h - 1) * Jl.pitch;
#pragma unroll 1
        for (int c = 0; c < Wn::RW; c++) win[r * Wn::RW + c] = load4_clamped(row, xa + 4 * c, Jl.w);
      }
    }
  }
  ICols ic_local;
  ICols& ic = *(PHASE == 0 ? &ic_local : icp);
  static_assert(!IGLOBAL || (WPL <= 2 && RT <= 16), "a lane's I words fit ICols");
  if constexpr (IGLOBAL && PHASE != 2) {
    // the lane's I words, in flight while the window copies land
    if (valid) {
      const uint8_t* ib = Ig.p + (size_t)((by0 + byl) * S + h * RT) * Ig.pitch + (bx0 + bxl) * S + 4 * q0;
#pragma unroll
      for (int i = 0; i < RT; i++) {
        if constexpr (WPL == 2) {
          const uint2 v = __ldg(reinterpret_cast<const uint2*>(ib));
          ic.v[0][i] = v.x;
          ic.v[1][i] = v.y;
        } else {
          ic.v[0][i] = __ldg(reinterpret_cast<const uint32_t*>(ib));
        }
        ib += Ig.pitch;
      }
    }
  }
  if constexpr (PHASE != 1) {   // the rest computes (PHASE 1 only copies)
    if constexpr (PHASE == 0) {
      cp_async_commit();
      cp_async_wait_all();
      __syncwarp();
    }

    // ---- candidates -------------------------------------------------------------
    uint32_t acc[5][5];   // [dx][dy]
#pragma unroll
    for (int a = 0; a < 5; a++)
#pragma unroll
      for (int d = 0; d < 5; d++) acc[a][d] = 0;
    if (valid) {
      uint32_t icol[WPL][RT];
      if constexpr (IGLOBAL) {
#pragma unroll
        for (int m = 0; m < WPL; m++)
#pragma unroll
          for (int i = 0; i < RT; i++) icol[m][i] = ic.v[m][i];
      } else {
        const uint32_t* ip = s_i + (byl * S + h * RT) * IW + bxl * NQ + q0;
#pragma unroll
        for (int m = 0; m < WPL; m++)
#pragma unroll
          for (int i = 0; i < RT; i++) icol[m][i] = ip[i * IW + m];
      }
      const uint32_t* wp = win + (h * RT) * Wn::RW + q0 + off;
#pragma unroll
      for (int w = 0; w < RT + 2 * RR; w++) {
        uint32_t wv[WPL + 2], u[WPL + 1];
#pragma unroll
        for (int k = 0; k < WPL + 2; k++) wv[k] = wp[w * Wn::RW + k];
#pragma unroll
        for (int k = 0; k <= WPL; k++) u[k] = __funnelshift_r(wv[k], wv[k + 1], s8);
#pragma unroll
        for (int m = 0; m < WPL; m++) {
          const uint32_t jw[5] = {u[m], __funnelshift_r(u[m], u[m + 1], 8), __funnelshift_r(u[m], u[m + 1], 16),
                                  __funnelshift_r(u[m], u[m + 1], 24), u[m + 1]};
#pragma unroll
          for (int d = 0; d < 5; d++) {
            const int i = w - d;
            if (i >= 0 && i < RT) {
#pragma unroll
              for (int a = 0; a < 5; a++) acc[a][d] = sad4(icol[m][i], jw[a], acc[a][d]);
            }
          }
        }
      }
    }
    // sum the lanes' partials: every candidate's SAD over the block is below
    // 2^16 (at most 256 pixels * 255), so two candidates share a 32-bit shuffle
    // and their halves never carry into each other
    uint32_t pk[13];
#pragma unroll
    for (int j = 0; j < 13; j++) {
      const int c0 = 2 * j, c1 = 2 * j + 1;
      pk[j] = acc[c0 % 5][c0 / 5] | (c1 < 25 ? acc[c1 % 5][c1 / 5] << 16 : 0u);
    }
#pragma unroll
    for (int xo = 1; xo < LPB; xo <<= 1) {
#pragma unroll
      for (int j = 0; j < 13; j++) pk[j] += __shfl_xor_sync(0xFFFFFFFFu, pk[j], xo);
    }
    uint32_t best = 0xFFFFFFFFu;
    if (valid) {
      // key = acc*256 + |v|_1*(256*lambda + 25) + 5*dy_i + dx_i - 25*min|v|_1,
      // split into a dx part and a dy part (exact in 32 bits: key < 2^25)
      const int n1min = max(abs(cx) - RR, 0) + max(abs(cy) - RR, 0);
      const uint32_t k1 = (uint32_t)lam * 256u + 25u;
      uint32_t kx[5], ky[5];
#pragma unroll
      for (int a = 0; a < 5; a++) kx[a] = (uint32_t)abs(cx + a - RR) * k1 + (uint32_t)a - 25u * (uint32_t)n1min;
#pragma unroll
      for (int d = 0; d < 5; d++) ky[d] = (uint32_t)abs(cy + d - RR) * k1 + 5u * (uint32_t)d;
      uint32_t key[25];
#pragma unroll
      for (int d = 0; d < 5; d++)
#pragma unroll
        for (int a = 0; a < 5; a++) {
          const int c = d * 5 + a;
          const uint32_t sad = (c & 1) ? pk[c >> 1] >> 16 : pk[c >> 1] & 0xFFFFu;
          key[c] = sad * 256u + kx[a] + ky[d];
        }
#pragma unroll
      for (int c = 0; c < 24; c += 2) best = __vimin3_u32(best, key[c], key[c + 1]);
      best = min(best, key[24]);
    }
    const int r = (int)(best & 255u) % 25;
    if (valid && t == 0) {
      s_vx[bl] = cx + r % 5 - RR;
      s_vy[bl] = cy + r / 5 - RR;
    }
    if constexpr (SUMS) {
      if (valid) {
        // pixel (4(q0+m) + c, i) of the block meets window byte (xw & 3) + 4(q0+m) + c + dx_i
        // of row i + dy_i
        const int o = (xw & 3) + r % 5, dyi = r / 5, sh = 8 * (o & 3);
        uint32_t si = 0, sj = 0, sii = 0, sjj = 0, sij = 0, sab = 0;
        const uint32_t* ip = IGLOBAL ? nullptr : s_i + (byl * S + h * RT) * IW + bxl * NQ + q0;
#pragma unroll
        for (int m = 0; m < WPL; m++) {
          const uint32_t* jp = win + (h * RT + dyi) * Wn::RW + q0 + m + off + (o >> 2);
#pragma unroll
          for (int i = 0; i < RT; i++) {
            // the lane's I words again: registers, or reread from the staged tile
            const uint32_t iv = IGLOBAL ? ic.v[m][i] : ip[i * IW + m];
            const uint32_t w0 = jp[i * Wn::RW], w1 = sh ? jp[i * Wn::RW + 1] : 0u;
            const uint32_t jv = __funnelshift_r(w0, w1, sh);
            si = __dp4a(iv, 0x01010101u, si);
            sj = __dp4a(jv, 0x01010101u, sj);
            sii = __dp4a(iv, iv, sii);
            sjj = __dp4a(jv, jv, sjj);
            sij = __dp4a(iv, jv, sij);
            sab = sad4(iv, jv, sab);
          }
        }
        part[0] += si; part[1] += sj; part[2] += sii; part[3] += sjj; part[4] += sij; part[5] += sab;
      }
    }
    __syncwarp();   // the next level's lanes read s_vx/s_vy and rewrite the window
  }
}

// Multiplier of the coarse candidate keys: key = cost * kCoarseKeyM + tb with
// tb = (|v|_1 << 12) | (vy + R) << 6 | (vx + R) < 2^18 < kCoarseKeyM, so keys
// order exactly as (cost, |v|_1, vy, vx), and tb = key mod kCoarseKeyM.  A
// multiplier that is not a power of two makes the key one integer multiply-add,
// which runs beside the SAD instructions instead of on their pipe.  Keys stay
// below 2^32 for cost <= 16*255 + 64*2*24.
constexpr uint32_t kCoarseKeyM = kCoarseKeyMul;

// Rows of the coarse search for one block and NJ consecutive vx candidates
// starting at vx0: slides down the staged window rows from `wrow` (the block's
// first row, word of vx0) and returns the smallest key.  With SHIFTED the
// window is staged as four copies, copy j (at +j * COPY words) holding the
// rows shifted by j bytes; otherwise the shifts are taken here.
template <int R, int NJ, int WWORDS, int COPY, bool SHIFTED>
__device__ __forceinline__ uint32_t coarse_rows(const uint32_t* wrow, uint32_t i0, uint32_t i1, uint32_t i2,
                                                uint32_t i3, int vx0, uint32_t lamM, uint32_t keyM) {
  // acc[j][c & 3] holds candidate c = dy - k (vy = c - R): it receives row k
  // of the block at window row dy, starts at k = 0 and completes at k = 3.
  uint32_t acc[NJ][4];
  uint32_t best[NJ], pend[NJ];   // pend: the previous row's keys, folded in pairs by a 3-input minimum
#pragma unroll
  for (int j = 0; j < NJ; j++) {
    best[j] = 0xFFFFFFFFu;
    pend[j] = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 4; k++) acc[j][k] = 0;
  }
#pragma unroll
  for (int dy = 0; dy < 2 * R + 4; dy++) {
    uint32_t w[NJ];
    if constexpr (SHIFTED || NJ == 1) {
#pragma unroll
      for (int j = 0; j < NJ; j++) w[j] = wrow[j * COPY + dy * WWORDS];
    } else {
      const uint32_t wlo = wrow[dy * WWORDS], whi = wrow[dy * WWORDS + 1];
#pragma unroll
      for (int j = 0; j < NJ; j++) w[j] = j ? __funnelshift_r(wlo, whi, 8 * j) : wlo;
    }
#pragma unroll
    for (int j = 0; j < NJ; j++) {
      if (dy <= 2 * R) acc[j][dy & 3] = sad4(i0, w[j], 0u);
      if (dy >= 1 && dy - 1 <= 2 * R) acc[j][(dy - 1) & 3] = sad4(i1, w[j], acc[j][(dy - 1) & 3]);
      if (dy >= 2 && dy - 2 <= 2 * R) acc[j][(dy - 2) & 3] = sad4(i2, w[j], acc[j][(dy - 2) & 3]);
      if (dy >= 3) acc[j][(dy - 3) & 3] = sad4(i3, w[j], acc[j][(dy - 3) & 3]);
    }
    if (dy >= 3) {
      const int vy = dy - R - 3;
      const int avy = vy < 0 ? -vy : vy;
      const uint32_t bv = lamM * (uint32_t)avy + (((uint32_t)avy << 12) | ((uint32_t)(vy + R) << 6));
#pragma unroll
      for (int j = 0; j < NJ; j++) {
        const uint32_t key = acc[j][(dy - 3) & 3] * keyM + bv;
        if (((dy - 3) & 1) == 0 && dy < 2 * R + 3) pend[j] = key;
        else best[j] = __vimin3_u32(best[j], pend[j], key);
      }
    }
  }
  uint32_t tbest = 0xFFFFFFFFu;
#pragma unroll
  for (int j = 0; j < NJ; j++) {
    const int vx = vx0 + j;
    const int avx = vx < 0 ? -vx : vx;
    const uint32_t a = lamM * (uint32_t)avx + ((uint32_t)avx << 12) + (uint32_t)(vx + R);
    tbest = min(tbest, best[j] + a);
  }
  return tbest;
}

// Exhaustive search of every block of a tile on the coarsest level (block
// side 4, radius R): threads [0, NB*R/2) own one block and 4 consecutive vx
// candidates each (vx = -R .. R-1), threads [NB*R/2, NB*R/2 + NB) one block
// and the last column vx = +R (a whole warp or warps: the split is a multiple
// of 32 threads).  Window layout as in coarse_rows.  Expects s_best32 set to
// all ones and a barrier before the call; leaves the coarse vectors in
// s_vx/s_vy (after a barrier).
template <int R, int TBX, int TBY, int NT, bool SHIFTED>
__device__ __forceinline__ void coarse_phase(const uint32_t* jwin, const uint32_t* iwin, int bx0, int by0, int nbx,
                                             int nby, int lam, uint32_t keyM, uint32_t* s_best32, int* s_vx, int* s_vy,
                                             int tid) {
  constexpr int GQ = R / 2, NB = TBX * TBY, NG = NB * GQ, WWORDS = TBX + GQ + 1;
  constexpr int COPY = (TBY * 4 + 2 * R) * WWORDS;
  static_assert(R % 4 == 0 && NG % 32 == 0 && NT >= NG + NB, "coarse thread layout");
  const bool grouped = tid < NG, last = tid >= NG && tid < NG + NB;
  const int g = grouped ? tid % GQ : GQ;
  const int bl = grouped ? tid / GQ : (last ? tid - NG : 0);
  const int bxl = bl % TBX, byl = bl / TBX;
  const bool active = (grouped || last) && (bx0 + bxl < nbx) && (by0 + byl < nby);
  const uint32_t i0 = iwin[(byl * 4 + 0) * TBX + bxl], i1 = iwin[(byl * 4 + 1) * TBX + bxl];
  const uint32_t i2 = iwin[(byl * 4 + 2) * TBX + bxl], i3 = iwin[(byl * 4 + 3) * TBX + bxl];
  const uint32_t lamM = (uint32_t)lam * keyM;
  const uint32_t* wrow = jwin + (byl * 4) * WWORDS + bxl + g;
  uint32_t tbest = 0xFFFFFFFFu;
  if (grouped)   // warp-uniform
    tbest = coarse_rows<R, 4, WWORDS, COPY, SHIFTED>(wrow, i0, i1, i2, i3, -R + 4 * g, lamM, keyM);
  else if (tid < ((NG + NB + 31) & ~31))
    tbest = coarse_rows<R, 1, WWORDS, COPY, SHIFTED>(wrow, i0, i1, i2, i3, R, lamM, keyM);
  if (active) atomicMin(&s_best32[bl], tbest);
  __syncthreads();
  for (int i = tid; i < NB; i += NT) {
    const uint32_t tb = s_best32[i] % kCoarseKeyM;
    s_vx[i] = (int)(tb & 63u) - R;
    s_vy[i] = (int)((tb >> 6) & 63u) - R;
  }
  __syncthreads();
}

// Phase C of a tile (Sec. III.A, SWR and AMM): the integer sums of the
// motion-compensated pair over the tile's pixels (a pixel outside the full
// blocks takes the vector of the nearest block), the AMM term of every block,
// the optional motion dump, and the CTA reduction into the pair's accumulators.
// On the fast path part[] already holds each thread's share of the full-block
// pixels (added during the level-0 refinement) and only the strips beyond the
// last full block column/row are read here; otherwise every pixel of the tile
// is read here.
template <int TBX, int TBY, int NT, class Bar = CtaBarrier>
__device__ __forceinline__ void sums_phase(const PairBatch& b, const PairJob& jb, int bx0, int by0, int B0, bool fast,
                                           const uint32_t (&part)[6], const int* s_vx, const int* s_vy,
                                           unsigned long long (*s_red)[kRecWords], int tid, const Bar& bar = Bar{}) {
  constexpr int NB = TBX * TBY, NW = NT / 32;
  const int nbx = jb.nbx, nby = jb.nby;
  const Plane I0 = jb.I[0], J0 = jb.J[0];
  const int W = I0.w, H = I0.h;
  const int xs = bx0 * B0, ys = by0 * B0;
  const int xe = (bx0 + TBX >= nbx) ? W : (bx0 + TBX) * B0;
  const int ye = (by0 + TBY >= nby) ? H : (by0 + TBY) * B0;
  const int lim_w = min(J0.w, J0.pitch);
  uint32_t si = part[0], sj = part[1], sii = part[2], sjj = part[3], sij = part[4], sab = part[5];
  // pixels of [x0, x1) x [y0, y1), 4-pixel words from x0 (a multiple of 4)
  auto region = [&](int x0, int x1, int y0, int y1) {
    const int nwx = (x1 - x0 + 3) >> 2;
    const int nrows = y1 - y0;
    for (int idx = tid; idx < nrows * nwx; idx += NT) {
      const int ry = idx / nwx, wx = idx - ry * nwx;
      const int y = y0 + ry, x = x0 + 4 * wx;
      const int bx = min(x / B0, nbx - 1), by = min(y / B0, nby - 1);
      const int bl = (by - by0) * TBX + (bx - bx0);
      const int vx = s_vx[bl], vy = s_vy[bl];
      const uint8_t* irow = I0.p + (size_t)y * I0.pitch;
      const int yj = clampi(y + vy, 0, H - 1);
      const uint8_t* jrow = J0.p + (size_t)yj * J0.pitch;
      const int xj = x + vx;
      uint32_t iv, jv;
      if (x + 3 <= x1 - 1) {
        iv = __ldg(reinterpret_cast<const uint32_t*>(irow + x));
        jv = (xj >= 0 && xj + 7 <= lim_w - 1) ? load4_unaligned(jrow, xj) : load4_clamped(jrow, xj, J0.w);
      } else {
        // ragged end of the row: bytes beyond x1 contribute zero to every sum
        iv = 0;
        jv = 0;
        for (int k = 0; x + k < x1; k++) {
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
  };
  if (fast) {
    const int xf = nbx * B0, yf = nby * B0;   // end of the full blocks
    if (xe > xf) region(max(xs, xf), xe, ys, ye);
    if (ye > yf) region(xs, min(xe, xf), max(ys, yf), ye);
  } else {
    region(xs, xe, ys, ye);
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
  // warp sums fit 32 bits: a thread sums fewer than 2,000 pixels (about 100
  // with the supported tiles) and at most one block's AMM term, and
  // 32 * 2000 * 255^2 < 2^32, 32 * floor(sqrt(2 * 102^2) * 2^16) < 2^32 (102 px:
  // the reach with coarse radius 24); the CTA and pair totals are 64-bit
  uint32_t v[kRecWords] = {si, sj, sii, sjj, sij, sab, samm};
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
  bar.sync();
  if (tid < kRecWords) {
    unsigned long long a = 0;
    for (int w = 0; w < NW; w++) a += s_red[w][tid];
    atomicAdd(jb.rec + tid, a);
  }
  bar.sync();
}

}  // namespace va
