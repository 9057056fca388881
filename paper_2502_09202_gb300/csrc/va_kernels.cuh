// Device-side data structures shared by the kernels and the host engine.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace va {

constexpr int kMaxLevels = 4;
constexpr int kCoarseSide = 4;     // block side at the coarsest pyramid level
constexpr int kRecWords = 7;       // sum i, sum j, sum i^2, sum j^2, sum i*j, sum |i-j|, S_amm

// One 8-bit image plane (or a row-strided view of one, e.g. a field).
struct Plane {
  const uint8_t* p;
  int pitch;   // bytes between consecutive rows of this view
  int w, h;
};

// One downsampling step: dst = box-filter of src, dims floor(w/2) x floor(h/2).
struct DownJob {
  Plane src;
  uint8_t* dst;
  int dst_pitch;
};

// Levels 1 and 2 of a frame and of both its fields from one read of level 0
// (rows 2y, 2y+1 -> frame level 1; rows 4y, 4y+2 -> upper field; 4y+1, 4y+3 ->
// lower field; level 2 from the rounded level-1 values).  out[] = frame L1,
// frame L2, upper L1, upper L2, lower L1, lower L2; the level-2 entries are
// null when the pyramid has two levels.
struct PyrJob {
  const uint8_t* l0;
  uint8_t* out[6];
  int pitch[6];
  int l0_pitch;
  int w, h;         // level-0 size (h even)
  uint32_t* hist;   // 256 bins the frame's level-0 values are added to, or null
};

// One pair measure: I against J (both views have the same dims per level).
struct PairJob {
  Plane I[kMaxLevels];
  Plane J[kMaxLevels];
  int nbx, nby;              // level-0 block grid
  int tiles_x, tiles_y;      // tile grid over the block grid
  int item_begin;            // index of this job's first tile in the batch
  unsigned long long* rec;   // kRecWords accumulators (zeroed before the launch)
  short2* vec;               // optional level-0 motion field dump (nby*nbx), or null
  short2* cvec;              // coarse vectors (nby*nbx) between the split kernels, or null
};

// Multiplier of the coarse candidate keys (see coarse_rows in va_device.cuh);
// the kernels read it from their launch parameters, so that the key stays one
// integer multiply-add instead of the shift-and-add sequence a compile-time
// 2^18 + 1 turns into on the integer ALU pipe the packed SADs use.
constexpr uint32_t kCoarseKeyMul = (1u << 18) + 1u;

struct SearchCfg {
  int levels;    // L; level-0 block side is kCoarseSide << (L-1)
  int radius;    // coarse exhaustive radius R (multiple of 4)
  int refine;    // refinement radius r
  int lambda;    // motion cost per pixel of |vx|+|vy|
  uint32_t key_mul = kCoarseKeyMul;   // always kCoarseKeyMul
};

struct PairBatch {
  const PairJob* jobs;
  int njobs;
  int nitems;                // total tiles over all jobs
  const uint32_t* qtab;      // Q(k) = floor(sqrt(k) * 2^16), k = 0..qmax
  int qmax;
  SearchCfg cfg;
  int* status;               // error word: nonzero when a device-side check failed
};

// Host launchers (defined in va_kernels.cu).
// Copies ceil(bytes/16) 16-byte words with a kernel; src and dst are 16-byte
// aligned device or page-locked host buffers of at least that many words.
cudaError_t launch_copy_words(const void* src, void* dst, size_t bytes, cudaStream_t st);
// pyramid_kernel, then histogram_kernel when `histograms` (jobs with hist set)
cudaError_t launch_pyramid(const PyrJob* d_jobs, int njobs, int max_w, int max_h, bool histograms, cudaStream_t st);
cudaError_t launch_downsample(const DownJob* d_jobs, int njobs, int max_dst_h, int max_dst_w,
                              cudaStream_t st);
cudaError_t launch_pairs(const PairBatch& b, int tbx, int tby, int grid, cudaStream_t st);
bool pair_tile_supported(int radius, int tbx, int tby);
int pair_threads(int radius, int tbx, int tby);
int pair_blocks_per_sm(int radius, int tbx, int tby);
// the default estimator as two kernels (va_split.cu): coarse search, then
// refinement + sums; each launch runs one CTA per (pair, tile)
bool split_applies(const PairBatch& b);
cudaError_t launch_coarse(const PairBatch& b, int tbx, int tby, cudaStream_t st);
cudaError_t launch_refine(const PairBatch& b, int tbx, int tby, cudaStream_t st);

}  // namespace va
