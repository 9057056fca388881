// Host-side detectors: shot boundaries (Sec. III.B), sampling structure
// (Sec. III.C) and dynamic keyframes (Sec. III.D), as a resumable state
// machine over pair measures that arrive from the GPU in waves.
//
// Every floating-point expression that feeds a decision is written as a fixed
// sequence of IEEE double operations; this file is compiled with
// -ffp-contract=off so no multiply-add is fused.
#pragma once
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "../../include/analyser.h"

namespace va {

enum PairKind { kFrame = 0, kUpperLower = 1, kLowerUpper = 2, kUpperUpper = 3, kLowerLower = 4 };
constexpr int kPairKinds = 5;

inline uint64_t pair_key(int kind, int a, int b) {
  return ((uint64_t)kind << 60) | ((uint64_t)(uint32_t)a << 30) | (uint64_t)(uint32_t)b;
}
inline int key_kind(uint64_t k) { return (int)(k >> 60); }
inline int key_a(uint64_t k) { return (int)((k >> 30) & 0x3FFFFFFFu); }
inline int key_b(uint64_t k) { return (int)(k & 0x3FFFFFFFu); }

struct Measure {
  int64_t s[7];   // sum i, sum j, sum i^2, sum j^2, sum i*j, sum |i-j|, S_amm
  int64_t n, nb;
  double ncc, swr, amm, act;
  bool used;      // fetched by a detector rule (reported in the results)
};

// Exact FP64 finalisation of one record (NCC, SWR, AMM, ACT).
void finalise_measure(Measure& m);

// Source of measures: returns null when the pair has not been computed yet.
struct MeasureStore {
  std::unordered_map<uint64_t, Measure> map;
  Measure* find(int kind, int a, int b) {
    auto it = map.find(pair_key(kind, a, b));
    return it == map.end() ? nullptr : &it->second;
  }
};

struct ShotOut {
  int first, last, label, field_order, phase, analysed;
};

class Detector {
 public:
  // kNeedVotes is internal: the shot detector waits for the sampling detector's
  // verdict on the current shot (run() reports it as kNeedPairs)
  enum Status { kProgress = 0, kNeedPairs = 1, kNeedFrames = 2, kDone = 3, kNeedVotes = 4 };

  Detector() = default;
  void reset(const analyser_params& p, int64_t nb);

  // Advance as far as the available measures and frames allow.
  //   avail    frames 0..avail-1 exist (pushed)
  //   finished no frame beyond avail-1 will ever come
  // Missing pair measures are appended to `need` (each at most once per call).
  Status run(MeasureStore& store, int avail, bool finished, std::vector<uint64_t>& need);

  // Oldest frame any future rule can still touch.
  int keep_from() const;

  bool done() const { return done_; }

  // results (valid once done())
  std::vector<int> cuts, dissolves, keyframes;
  std::vector<ShotOut> shots;
  int clip_label = ANALYSER_UNKNOWN, clip_fo = ANALYSER_FO_NONE, clip_phase = -1;

 private:
  enum { kRepNone = 0, kRepUpper = 1, kRepLower = 2 };
  struct Vote { int t; double a0, a1, a2; };   // AMM of v0, v1, v2
  struct Shot {
    int first = 0, last = -1;
    std::vector<int> eligible;     // frames t with t+1 in the shot, in order
    size_t next_eligible = 0;      // first eligible frame not yet examined
    std::vector<Vote> analysed;
    std::vector<int> reps;         // repeated-field flag of voters 1, 2, ...
    int voters_seen = 0;           // voters among the eligible frames (decided by S_amm alone)
    bool has_verdict = false;      // structure decided after samp_max_frames votes
    ShotOut verdict{};
  };
  Status shot_step(MeasureStore& store, int avail, bool finished, std::vector<uint64_t>& need);
  Status sampling_step(MeasureStore& store, Shot& sh, std::vector<uint64_t>& need, bool& voted);
  int deep_check(MeasureStore& store, int t, int T, bool finished, int avail, std::vector<uint64_t>& need,
                 Status& st);
  int deep_check_pulldown(MeasureStore& store, int t, int T, bool finished, int avail, std::vector<uint64_t>& need,
                          Status& st);
  bool wants_reps(const Shot& sh, size_t voter) const;
  void classify(const Shot& sh, ShotOut& out) const;
  void finish_clip();

  void use(Measure* m) const {   // a rule read m (a speculative copy reads without reporting)
    if (!spec_) m->used = true;
  }

  analyser_params p_{};
  bool spec_ = false;            // a speculative copy that only collects pair requests
  int spec_quiet_ = -1;          // (speculative copy) last frame a pending deep check could take
  int64_t static_thr_ = 0;
  int t_ = 0;                    // shot detector position (frame under test)
  int T_ = -1;                   // clip length once known
  std::vector<double> hist_;
  double S_ = 0.0;
  std::vector<Shot> open_;       // shots whose sampling is not complete (front = oldest)
  std::vector<ShotOut> closed_out_;
  bool done_ = false;
};

}  // namespace va
