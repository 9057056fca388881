// The default estimator (3 pyramid levels, level-0 blocks of 16, refinement
// radius 2) as two kernels that the engine pipelines over chunks of a wave on
// two streams, so that the ALU-bound coarse search of one chunk runs beside the
// latency-bound refinement and correlation sums of the previous one:
//   coarse_kernel  one CTA per (pair, tile): exhaustive coarse search, vectors
//                  written to the pair's coarse-vector array;
//   refine_kernel  one CTA per (pair, tile): both refinement levels, the AMM
//                  term and the motion-compensated sums.
// Arithmetic and candidate order are those of the fused pair kernel.
#include "va_device.cuh"

#ifndef VA_COARSE_MINB
#define VA_COARSE_MINB 7
#endif
#ifndef VA_REFINE_LPB
#define VA_REFINE_LPB 4      // lanes per block in the refinement kernel (2 or 4)
#endif
#ifndef VA_REFINE_REGS
#define VA_REFINE_REGS (VA_REFINE_LPB == 2 ? 80 : 64)   // register budget per thread
#endif

namespace va {
namespace {

template <int R, int TBX, int TBY>
struct CoarseShape {
  static constexpr int G = (2 * R + 4) / 4;
  static constexpr int NB = TBX * TBY;
  static constexpr int NT = (NB * G + 31) / 32 * 32;
  static constexpr int WROWS = TBY * kCoarseSide + 2 * R;
  static constexpr int WWORDS = TBX + G;
  static constexpr int MINB = VA_COARSE_MINB * 288 / NT > 0 ? VA_COARSE_MINB * 288 / NT : 1;  // resident CTAs per SM
};

template <int TBX, int TBY>
struct RefineShape {
  static constexpr int NB = TBX * TBY;
  static constexpr int LPB = VA_REFINE_LPB;
  static constexpr int NT = NB * LPB < 32 ? 32 : NB * LPB;   // LPB lanes per block
  static constexpr int MINB0 = 65536 / (VA_REFINE_REGS * NT);
  static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 > 32 ? 32 : MINB0);   // resident CTAs per SM at the budget
};

// Copies the job holding `item` to shared memory: thread t checks jobs t,
// t + NT, ... at once (item_begin[j] <= item < item_begin[j + 1]; exactly one
// job matches, also with empty jobs), so the lookup costs one round trip to L2 whatever the
// number of jobs.  Called by every thread of `bar`; ends with a barrier.
template <int NT, class Bar>
__device__ __forceinline__ void copy_job(const PairBatch& b, int item, PairJob* dst, int* s_jidx, int tid,
                                         const Bar& bar) {
  for (int j = tid; j < b.njobs; j += NT) {
    const int beg = b.jobs[j].item_begin;
    const int next = j + 1 < b.njobs ? b.jobs[j + 1].item_begin : 0x7FFFFFFF;
    if ((j == 0 || beg <= item) && item < next) *s_jidx = j;   // item_begin is nondecreasing: one match
  }
  bar.sync();
  const int* src = reinterpret_cast<const int*>(b.jobs + *s_jidx);
  for (int i = tid; i < (int)(sizeof(PairJob) / 4); i += NT) reinterpret_cast<int*>(dst)[i] = src[i];
  bar.sync();
}

// Shared memory of one coarse tile and of one refinement tile.
template <int R, int TBX, int TBY>
struct CoarseSmem {
  using S = CoarseShape<R, TBX, TBY>;
  uint32_t jwin[4 * S::WROWS * S::WWORDS];   // the window shifted by 0..3 bytes
  uint32_t iw[TBY * kCoarseSide * TBX];
  uint32_t best32[S::NB];
  int vx[S::NB], vy[S::NB];
  PairJob job;
  int jidx;
};
template <int TBX, int TBY>
struct RefineSmem {
  using S = RefineShape<TBX, TBY>;
  alignas(16) uint32_t i1[TBY * 8 * TBX * 2];
  alignas(16) uint32_t win[S::NB * kRefineWinWords];
  int vx[S::NB], vy[S::NB];
  unsigned long long red[S::NT / 32][kRecWords];
  PairJob job;
  int jidx;
};

// Exhaustive coarse search of one tile by NT threads (the whole CTA, NT >= the
// shape's thread count); vectors written to the pair's coarse-vector array.
template <int R, int TBX, int TBY, int NT>
__device__ __forceinline__ void coarse_tile(const PairBatch& b, int item, CoarseSmem<R, TBX, TBY>& sm, int tid) {
  using S = CoarseShape<R, TBX, TBY>;
  constexpr int NB = S::NB, WROWS = S::WROWS, WWORDS = S::WWORDS;
  static_assert(NT >= S::NT, "enough threads for the coarse layout");
  copy_job<NT>(b, item, &sm.job, &sm.jidx, tid, CtaBarrier{});
  const PairJob& jb = sm.job;
  const int local = item - jb.item_begin;
  const int bx0 = (local % jb.tiles_x) * TBX, by0 = (local / jb.tiles_x) * TBY;
  const int nbx = jb.nbx, nby = jb.nby;
  const Plane J2 = jb.J[2], I2 = jb.I[2];
  const int Xw0 = bx0 * kCoarseSide - R, Yw0 = by0 * kCoarseSide - R;
  for (int c = tid; c < WROWS * WWORDS; c += NT) {
    const int wy = c / WWORDS, wx = c - wy * WWORDS;
    const int y = clampi(Yw0 + wy, 0, J2.h - 1), x = Xw0 + 4 * wx;
    const uint8_t* row = J2.p + (size_t)y * J2.pitch;
    uint32_t w0, w1;
    if (x >= 0 && x + 7 <= J2.w - 1) {
      w0 = __ldg(reinterpret_cast<const uint32_t*>(row + x));
      w1 = __ldg(reinterpret_cast<const uint32_t*>(row + x + 4));
    } else {
      w0 = load4_clamped(row, x, J2.w);
      w1 = load4_clamped(row, x + 4, J2.w);
    }
    sm.jwin[c] = w0;
    sm.jwin[WROWS * WWORDS + c] = __funnelshift_r(w0, w1, 8);
    sm.jwin[2 * WROWS * WWORDS + c] = __funnelshift_r(w0, w1, 16);
    sm.jwin[3 * WROWS * WWORDS + c] = __funnelshift_r(w0, w1, 24);
  }
  for (int c = tid; c < TBY * kCoarseSide * TBX; c += NT) {
    const int r = c / TBX, k = c - r * TBX;
    sm.iw[c] = (bx0 + k < nbx && by0 + r / kCoarseSide < nby)
                   ? __ldg(reinterpret_cast<const uint32_t*>(I2.p + (size_t)(by0 * kCoarseSide + r) * I2.pitch +
                                                             (bx0 + k) * kCoarseSide))
                   : 0u;
  }
  for (int i = tid; i < NB; i += NT) sm.best32[i] = 0xFFFFFFFFu;
  __syncthreads();
  coarse_phase<R, TBX, TBY, NT, true>(sm.jwin, sm.iw, bx0, by0, nbx, nby, b.cfg.lambda, b.cfg.key_mul, sm.best32,
                                       sm.vx, sm.vy, tid);
  for (int i = tid; i < NB; i += NT) {
    const int bx = bx0 + i % TBX, by = by0 + i / TBX;
    if (bx < nbx && by < nby) jb.cvec[(size_t)by * nbx + bx] = make_short2((short)sm.vx[i], (short)sm.vy[i]);
  }
}

// Both refinement levels, the AMM term and the motion-compensated sums of one
// tile by the shape's NT threads, which synchronise through `bar`.
template <int TBX, int TBY, class Bar>
__device__ __forceinline__ void refine_tile(const PairBatch& b, int item, RefineSmem<TBX, TBY>& sm, int tid,
                                            const Bar& bar) {
  using S = RefineShape<TBX, TBY>;
  constexpr int NB = S::NB, NT = S::NT, LPB = S::LPB;
  copy_job<NT>(b, item, &sm.job, &sm.jidx, tid, bar);
  const PairJob& jb = sm.job;
  const int local = item - jb.item_begin;
  const int bx0 = (local % jb.tiles_x) * TBX, by0 = (local / jb.tiles_x) * TBY;
  const int nbx = jb.nbx, nby = jb.nby;
  for (int c = tid; c < TBY * 8 * TBX; c += NT) {
    const int r = c / TBX, k = c - r * TBX;
    if (bx0 + k < nbx && by0 + r / 8 < nby)
      cp_async8(&sm.i1[c * 2], jb.I[1].p + (size_t)(by0 * 8 + r) * jb.I[1].pitch + (bx0 + k) * 8);
  }
  // each lane reads its block's coarse vector and issues its level-1 window
  // copies now, so that the tile's loads all land behind one wait
  const int lam = b.cfg.lambda;
  uint32_t part[6] = {0, 0, 0, 0, 0, 0};
  short2 pv = make_short2(0, 0);
  {
    const int bl = tid / LPB, bx = bx0 + bl % TBX, by = by0 + bl / TBX;
    if (bl < NB && bx < nbx && by < nby) pv = jb.cvec[(size_t)by * nbx + bx];
  }
  refine_level<8, 2, NT, NB, TBX, false, 1, LPB>(jb.J[1], sm.i1, bx0, by0, nbx, nby, lam, sm.vx, sm.vy, sm.win,
                                                 part, tid, pv.x, pv.y);
  cp_async_commit();
  cp_async_wait_all();
  bar.sync();
  refine_level<8, 2, NT, NB, TBX, false, 2, LPB>(jb.J[1], sm.i1, bx0, by0, nbx, nby, lam, sm.vx, sm.vy, sm.win,
                                                 part, tid, pv.x, pv.y);
  // level 0 reads its I words from global memory (no staged tile)
  refine_level<16, 2, NT, NB, TBX, true, 0, LPB, true>(jb.J[0], nullptr, bx0, by0, nbx, nby, lam, sm.vx, sm.vy,
                                                       sm.win, part, tid, 0, 0, jb.I[0]);
  bar.sync();   // every block's vector is read below
  sums_phase<TBX, TBY, NT>(b, jb, bx0, by0, 16, true, part, sm.vx, sm.vy, sm.red, tid, bar);
}

template <int R, int TBX, int TBY>
__global__ void __launch_bounds__(CoarseShape<R, TBX, TBY>::NT, CoarseShape<R, TBX, TBY>::MINB) coarse_kernel(const PairBatch b) {
  __shared__ CoarseSmem<R, TBX, TBY> sm;
  coarse_tile<R, TBX, TBY, CoarseShape<R, TBX, TBY>::NT>(b, blockIdx.x, sm, threadIdx.x);
}

template <int TBX, int TBY>
__global__ void __launch_bounds__(RefineShape<TBX, TBY>::NT, RefineShape<TBX, TBY>::MINB) refine_kernel(const PairBatch b) {
  __shared__ RefineSmem<TBX, TBY> sm;
  refine_tile<TBX, TBY>(b, blockIdx.x, sm, threadIdx.x, CtaBarrier{});
}

}  // namespace

#define VA_SPLIT_TILES(X, R) X(R, 8, 4) X(R, 4, 4) X(R, 8, 2) X(R, 16, 2) X(R, 4, 8)
#define VA_SPLIT_RADII(X) VA_SPLIT_TILES(X, 8) VA_SPLIT_TILES(X, 16) VA_SPLIT_TILES(X, 24)

bool split_applies(const PairBatch& b) { return b.cfg.levels == 3 && b.cfg.refine == 2; }

cudaError_t launch_coarse(const PairBatch& b, int tbx, int tby, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
#define VA_CASE(R_, X_, Y_)                                                                  \
  if (b.cfg.radius == R_ && tbx == X_ && tby == Y_) {                                        \
    coarse_kernel<R_, X_, Y_><<<b.nitems, CoarseShape<R_, X_, Y_>::NT, 0, st>>>(b);          \
    return cudaGetLastError();                                                               \
  }
  VA_SPLIT_RADII(VA_CASE)
#undef VA_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_refine(const PairBatch& b, int tbx, int tby, cudaStream_t st) {
  if (b.nitems <= 0) return cudaSuccess;
#define VA_CASE(X_, Y_)                                                              \
  if (tbx == X_ && tby == Y_) {                                                      \
    refine_kernel<X_, Y_><<<b.nitems, RefineShape<X_, Y_>::NT, 0, st>>>(b);          \
    return cudaGetLastError();                                                       \
  }
  VA_CASE(8, 4) VA_CASE(4, 4) VA_CASE(8, 2) VA_CASE(16, 2) VA_CASE(4, 8)
#undef VA_CASE
  return cudaErrorInvalidValue;
}

}  // namespace va
