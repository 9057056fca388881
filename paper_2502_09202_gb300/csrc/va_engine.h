// Runtime of the analyser: per-clip device windows, the measure cache and GPU
// waves that batch the work of every active clip into one set of launches.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <deque>
#include <memory>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/analyser.h"
#include "va_detect.h"
#include "va_kernels.cuh"

namespace va {

double now_seconds();
int validate_params(const analyser_params& p, std::string& why);
int min_window(const analyser_params& p);   // smallest rolling window the detectors can work in
int validate_size(int width, int height, const analyser_params& p, std::string& why);

// Level geometry of one clip.
struct Geometry {
  int W = 0, H = 0, L = 0, B0 = 0;
  int fw[kMaxLevels], fh[kMaxLevels], fp[kMaxLevels];   // frame levels (fp[0] = ring pitch)
  int gw[kMaxLevels], gh[kMaxLevels], gp[kMaxLevels];   // field levels
  size_t off_f[kMaxLevels], off_u[kMaxLevels], off_l[kMaxLevels];  // offsets within a slot (levels >= 1)
  size_t slot_bytes = 0;                 // pyramid levels >= 1 of one slot
  size_t l0_bytes = 0;                   // level 0 of one slot (0 when frames stay in caller memory)
  void init(int width, int height, int levels, bool own_l0 = true);
  size_t l0_region(int cap) const;       // bytes of the level-0 array of `cap` slots
};

// One clip being analysed.
struct Clip {
  long long id = 0;
  Geometry geo;
  double fps = 25.0;
  analyser_params p{};
  int tbx = 8, tby = 4;              // tile of the pair kernel (autotuned per resolution)
  // device window
  int cap = 0;                       // slots
  uint8_t* d_ring = nullptr;         // level-0 array, then cap * slot_bytes of pyramids
  uint32_t* d_hist = nullptr;        // cap * 256 bins of the slots' level-0 histograms (want_histogram)
  uint8_t* pyr = nullptr;            // start of the pyramid array
  std::vector<const uint8_t*> l0;    // level-0 frame of each slot
  std::vector<int> l0_pitch;
  bool external_l0 = false;          // slots point at caller device frames
  // progress
  int pushed = 0;        // frames [0, pushed) delivered (resident on the device)
  int uploaded = 0;      // frames [0, uploaded) handed to the copy stream (>= pushed on the chunked path)
  std::deque<std::pair<int, cudaEvent_t>> up_chunks;   // (end frame, completion event) of chunked copies
  int pyr_done = 0;      // frames [0, pyr_done) have pyramids
  int evicted = 0;       // frames [0, evicted) no longer resident
  int aon_next = 0;      // next always-on pair (t, t+1) not yet requested
  bool finished = false;
  MeasureStore store;
  Detector det;
  std::vector<uint64_t> pending;     // requests for the next wave
  std::unordered_set<uint64_t> inflight;
  std::vector<int16_t> motion;       // level-0 fields of (t, t+1) when want_motion
  std::vector<analyser_frame_hist> hist;   // per frame when want_histogram
  int status = ANALYSER_OK;
  std::string message;
  // host frame source (server path)
  const uint8_t* host_frames = nullptr;
  long long host_pitch = 0;
  int host_nframes = 0;
  // timing (server path)
  double t_submit = 0.0, t_done = -1.0;
  // stateless measure calls: no detector, requested pairs only
  bool stateless_ = false;
  bool want_vec_ = false;
  std::vector<std::pair<uint64_t, std::vector<short2>>> vec_out_;
  bool done() const { return det.done(); }
  int slot_of(int f) const { return f % cap; }
  size_t device_bytes() const { return geo.l0_region(cap) + (size_t)cap * geo.slot_bytes; }
};

// Results kept for the C ABI.
struct ResultsBuf {
  std::vector<int> cuts, dissolves, keyframes;
  std::vector<analyser_shot> shots;
  std::vector<analyser_measure> measures;
  std::vector<int16_t> motion;
  std::vector<analyser_frame_hist> hist;
  analyser_results_t r{};
};
void build_results(const Clip& c, ResultsBuf& out);

class Engine {
 public:
  explicit Engine(const analyser_params& p);
  ~Engine();
  int init(std::string& why);

  // clip management
  int add_clip(Clip* c, std::string& why, bool enlist = true);  // allocates the clip's ring
  void remove_clip(Clip* c);
  static size_t ring_bytes(const Geometry& g, int cap);

  // copy host frames into a clip's free slots; returns frames taken
  // reference device frames
  int attach_device(Clip* c, const uint8_t* frames, long long pitch, long long stride, int nframes);

  // One wave over all clips: pyramids of new frames, every requested pair,
  // readback, detector advance, eviction.  Returns the number of pairs run
  // (0 = nothing to do), or a negative error.
  int wave();
  // the same in two halves, so that host work (e.g. copying the next frames on
  // the copy stream) can overlap the GPU work of a wave
  int wave_launch();
  int wave_complete();
  bool wave_inflight() const { return inflight_; }
  int free_slots(const Clip* c) const { return c->cap - (std::max(c->pushed, c->uploaded) - c->evicted); }
  // Chunked host upload: copies up to `nframes` frames into free slots, `chunk`
  // frames per copy, each copy with its own event; the frames count as pushed
  // only once poll_uploads() has seen their copy complete, so waves never wait
  // on the GPU for copies still in flight.  Returns frames issued or -1.
  int upload_async(Clip* c, const uint8_t* frames, long long pitch, int nframes, int chunk);
  // Marks completed chunks as pushed (blocking on the oldest one when `wait`);
  // returns the number of frames that became resident or -1.
  int poll_uploads(Clip* c, bool wait);

  // stateless measure for tests and timing
  int measure_pairs(int width, int height, const uint8_t* frames, long long pitch, long long stride, int nframes,
                    const int* kinds, const int* ia, const int* ib, int npairs, int64_t* records, int16_t* motion,
                    cudaStream_t st, std::string& why);

  // waits for an event / all work queued on a stream, against params.wait_timeout_ms
  // when it is set (cudaErrorTimeout when the deadline passes first)
  cudaError_t wait_event(cudaEvent_t ev);
  cudaError_t wait_stream(cudaStream_t st);

  // tile choice for a resolution (autotuned once per engine and size)
  void choose_tile(int width, int height, int* tbx, int* tby);

  analyser_params p;
  std::vector<Clip*> clips;
  cudaStream_t stream = nullptr;    // kernels and record read-back
  cudaStream_t cstream = nullptr;   // host-to-device frame copies
  long long n_pairs = 0, n_waves = 0, n_launches = 0;
  long long n_pair_launches = 0, n_pyr_launches = 0;
  double pair_ms = 0.0, pyr_ms = 0.0, absdiff_ops = 0.0, pyr_bytes = 0.0;
  long long h2d_bytes = 0, d2h_bytes = 0;
  double host_gather_ms = 0, host_wait_ms = 0, host_results_ms = 0, host_setup_ms = 0, host_copy_wait_ms = 0;
  void profile(analyser_profile_t* out) const;
  int status = ANALYSER_OK;
  std::string message;
  bool autotune = true;
  int max_chunks = 4;        // chunks of a large wave (coarse of chunk c+1 beside refinement of chunk c)

 private:
  int ensure_capacity(int npairs, int ndown, int npyr);
  int run_alone(Clip* c);
  int setup_pair_job(const Clip& c, uint64_t key, PairJob& pj, int item_begin, unsigned long long* rec,
                     short2* vec);

  // device tables
  const uint32_t* d_qtab = nullptr;   // shared, owned by the resource cache
  int qmax = 0;
  int* d_status = nullptr;
  int* h_status = nullptr;
  cudaEvent_t ev_[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t rstream = nullptr;   // refinement kernels of the split path
  cudaEvent_t ev_chunk_ = nullptr, ev_join_ = nullptr, ev_wait_ = nullptr;
  short2* d_cvec = nullptr;         // coarse vectors between the split kernels
  size_t cap_cvec = 0;
  // wave in flight (between wave_launch and wave_complete)
  bool inflight_ = false;
  int fl_npairs_ = 0, fl_ndown_ = 0;
  size_t fl_vec_total_ = 0;
  bool fl_groups_ = false;
  double fl_t1_ = 0.0;
  int sm_count = 0;
  // wave buffers
  int cap_pairs = 0, cap_down = 0, cap_pyr = 0;
  PairJob* d_pjobs = nullptr;
  PairJob* h_pjobs = nullptr;
  DownJob* d_djobs = nullptr;
  DownJob* h_djobs = nullptr;
  PyrJob* d_pyjobs = nullptr;
  PyrJob* h_pyjobs = nullptr;
  uint32_t* h_hist = nullptr;        // page-locked bins of a wave's new frames
  int cap_hist = 0;
  struct HistRun { Clip* clip; int frame0, slot0, n, off; };   // n consecutive frames/slots at row `off` of h_hist
  std::vector<HistRun> hist_runs_;
  std::vector<PyrJob> pyr_;   // this wave's fused pyramid jobs
  unsigned long long* d_rec = nullptr;
  unsigned long long* h_rec = nullptr;
  short2* d_vec = nullptr;
  size_t cap_vec = 0;
  std::vector<short2> h_vec;
  // per wave bookkeeping
  struct WavePair { Clip* clip; uint64_t key; size_t vec_off; int tbx, tby; };
  std::vector<WavePair> wp_;
  std::vector<std::pair<int, int>> tune_keys_;
  std::vector<std::pair<int, int>> tune_vals_;
};

}  // namespace va
