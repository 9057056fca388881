// Detectors of Sec. III.B-D as a resumable state machine (see va_detect.h).
//
// Readings of what the paper leaves open (thresholds and window sizes are
// parameters, defaults in analyser_default_params):
//   fast check (III.B): with at least `jback` predecessors of t in the shot,
//     t is a candidate iff a_t > max(fast_tau, fast_lambda * m_t) (a jump) or
//     a_t > max(fast_tau, fast_rise * m_t) and a_t < a_{t+1} < a_{t+2} (a ramp
//     starts; needs frame t+3, false at the clip end), m_t the lower median of
//     the last <= fast_window values a_s of the shot.
//   deep check (III.B): for K = 1..kmax in order, with
//     p = max{ACT(t,t-j) : 1 <= j <= jback} and
//     "x significantly smaller than y" as deep_rho*x + deep_tau < y, K is valid iff
//     p << ACT(t,t+K), p << ACT(t,t+K+1) and a_{t+K} << ACT(t,t+K);
//     the smallest valid K wins (K = 1: hardcut at t+1; K >= 2: dissolve (t,K),
//     new shot from t+K).
//   sampling structure (III.C): the first samp_max_frames frames t of a shot
//     with t+1 in the shot and S_amm(t,t+1) >= ceil(static_amm_px*65536*nb)
//     vote with v0, v1, v2: combed iff v0 > comb_ratio * max(v1,v2); 3:2 phase
//     match of the combed pattern; otherwise interlaced iff most frames are
//     combed and the lower median B of beta = v1/v2 is off 1 by unequal_ratio
//     (B > 1: upper field first).
//   keyframes (III.D): first frame of each shot, then S += a_{t-1} and a
//     keyframe whenever S > kf_theta (S reset to 0).
#include "va_detect.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace va {

void finalise_measure(Measure& m) {
  const int64_t n = m.n, si = m.s[0], sj = m.s[1];
  // exact integer moments; |n*sum(ij)| < 2^63 for n <= 11.8M pixels of 8 bits
  const __int128 c = (__int128)n * m.s[4] - (__int128)si * sj;
  const __int128 vi = (__int128)n * m.s[2] - (__int128)si * si;
  const __int128 vj = (__int128)n * m.s[3] - (__int128)sj * sj;
  double ncc;
  if (vi == 0 && vj == 0) ncc = 1.0;
  else if (vi == 0 || vj == 0) ncc = 0.0;
  else {
    const double dc = (double)(int64_t)c, dvi = (double)(int64_t)vi, dvj = (double)(int64_t)vj;
    const double prod = dvi * dvj;
    ncc = dc / std::sqrt(prod);
  }
  const double om = 1.0 - ncc;
  m.ncc = ncc;
  m.swr = om > 0.0 ? om : 0.0;
  const double denom = (double)m.nb * 65536.0;
  m.amm = (double)m.s[6] / denom;
  const double prod2 = m.amm * m.swr;
  m.act = std::sqrt(prod2);
}

static double lower_median(const std::vector<double>& v, size_t from) {
  std::vector<double> s(v.begin() + (long)from, v.end());
  std::sort(s.begin(), s.end());
  return s[(s.size() - 1) / 2];
}

void Detector::reset(const analyser_params& p, int64_t nb) {
  p_ = p;
  const double thr = p.static_amm_px * 65536.0 * (double)nb;
  static_thr_ = (int64_t)std::ceil(thr);
  t_ = 0;
  T_ = -1;
  hist_.clear();
  S_ = 0.0;
  open_.clear();
  closed_out_.clear();
  cuts.clear();
  dissolves.clear();
  keyframes.clear();
  shots.clear();
  done_ = false;
  Shot first;
  first.first = 0;
  open_.push_back(first);
  keyframes.push_back(0);
}

int Detector::keep_from() const {
  int k = t_ - p_.kmax - 1;
  for (const Shot& sh : open_) {
    // only shots that still need votes keep their next eligible frame resident
    if (sh.analysed.size() < (size_t)p_.samp_max_frames && sh.next_eligible < sh.eligible.size())
      k = std::min(k, sh.eligible[sh.next_eligible]);
  }
  return std::max(k, 0);
}

// Pairs a deep check at t for span K reads.
static void deep_pairs(int t, int K, int s0, int jback, std::vector<uint64_t>& out) {
  for (int j = 1; j <= jback; j++)
    if (t - j >= s0) out.push_back(pair_key(kFrame, t, t - j));
  out.push_back(pair_key(kFrame, t, t + K));
  out.push_back(pair_key(kFrame, t, t + K + 1));
  out.push_back(pair_key(kFrame, t + K, t + K + 1));
}

int Detector::deep_check(MeasureStore& store, int t, int T, bool finished, int avail, std::vector<uint64_t>& need,
                         Status& st) {
  const int s0 = open_.back().first;
  st = kProgress;
  for (int K = 1; K <= p_.kmax; K++) {
    if (T >= 0 && t + K + 1 > T - 1) return 0;
    if (t + K + 1 >= avail) {
      st = finished ? kProgress : kNeedFrames;
      if (finished) return 0;
      return 0;
    }
    std::vector<uint64_t> keys;
    deep_pairs(t, K, s0, p_.jback, keys);
    bool missing = false;
    for (uint64_t k : keys) {
      if (!store.find(key_kind(k), key_a(k), key_b(k))) {
        missing = true;
        need.push_back(k);
      }
    }
    if (missing) {
      // ask for the later hypotheses' pairs in the same wave (they are only
      // reported once a rule reads them)
      for (int K2 = K + 1; K2 <= p_.kmax && t + K2 + 1 < avail; K2++) {
        std::vector<uint64_t> more;
        deep_pairs(t, K2, s0, p_.jback, more);
        for (uint64_t k : more)
          if (!store.find(key_kind(k), key_a(k), key_b(k))) need.push_back(k);
      }
      st = kNeedPairs;
      return 0;
    }
    double ref = 0.0;
    bool have_ref = false;
    for (int j = 1; j <= p_.jback; j++) {
      if (t - j < s0) continue;
      Measure* m = store.find(kFrame, t, t - j);
      m->used = true;
      if (!have_ref || m->act > ref) ref = m->act;
      have_ref = true;
    }
    Measure* fk = store.find(kFrame, t, t + K);
    Measure* fk1 = store.find(kFrame, t, t + K + 1);
    Measure* af = store.find(kFrame, t + K, t + K + 1);
    fk->used = fk1->used = af->used = true;
    const double base = p_.deep_rho * ref + p_.deep_tau;
    const double after = p_.deep_rho * af->act + p_.deep_tau;
    if (base < fk->act && base < fk1->act && after < fk->act) return K;
  }
  return 0;
}

Detector::Status Detector::shot_step(MeasureStore& store, int avail, bool finished, std::vector<uint64_t>& need) {
  Shot& cur = open_.back();
  if (T_ >= 0 && t_ >= T_ - 1) {
    if (cur.last < 0) cur.last = std::max(T_ - 1, cur.first);
    return kDone;
  }
  if (t_ + 1 >= avail) return kNeedFrames;
  Measure* a = store.find(kFrame, t_, t_ + 1);
  if (!a) {
    need.push_back(pair_key(kFrame, t_, t_ + 1));
    return kNeedPairs;
  }
  a->used = true;
  const double at = a->act;
  if ((int)hist_.size() >= p_.jback) {
    const size_t from = hist_.size() > (size_t)p_.fast_window ? hist_.size() - (size_t)p_.fast_window : 0;
    const double m = lower_median(hist_, from);
    const double lm = p_.fast_lambda * m;
    const double thr = p_.fast_tau >= lm ? p_.fast_tau : lm;
    bool cand = at > thr;
    if (!cand) {
      const double lr = p_.fast_rise * m;
      const double thr_r = p_.fast_tau >= lr ? p_.fast_tau : lr;
      const bool end_known = T_ >= 0;
      if (at > thr_r && !(end_known && t_ + 3 > T_ - 1)) {
        if (t_ + 3 >= avail) return kNeedFrames;
        Measure* a1 = store.find(kFrame, t_ + 1, t_ + 2);
        Measure* a2 = store.find(kFrame, t_ + 2, t_ + 3);
        if (!a1 || !a2) {
          if (!a1) need.push_back(pair_key(kFrame, t_ + 1, t_ + 2));
          if (!a2) need.push_back(pair_key(kFrame, t_ + 2, t_ + 3));
          return kNeedPairs;
        }
        cand = at < a1->act && a1->act < a2->act;
      }
    }
    if (cand) {
      Status st;
      const int K = deep_check(store, t_, T_, finished, avail, need, st);
      if (st != kProgress) return st;
      if (K > 0) {
        cur.last = t_;
        if (K == 1) cuts.push_back(t_ + 1);
        else { dissolves.push_back(t_); dissolves.push_back(K); }
        t_ += K;
        Shot nx;
        nx.first = t_;
        open_.push_back(nx);
        keyframes.push_back(t_);
        hist_.clear();
        S_ = 0.0;
        return kProgress;
      }
    }
  }
  hist_.push_back(at);
  cur.eligible.push_back(t_);
  S_ += at;
  if (S_ > p_.kf_theta) {
    keyframes.push_back(t_ + 1);
    S_ = 0.0;
  }
  t_ += 1;
  return kProgress;
}

Detector::Status Detector::sampling_step(MeasureStore& store, Shot& sh, std::vector<uint64_t>& need) {
  // Examine eligible frames in order; request the triples of every frame that
  // will vote (decided by S_amm alone) in one go.
  while (sh.analysed.size() < (size_t)p_.samp_max_frames && sh.next_eligible < sh.eligible.size()) {
    const int t = sh.eligible[sh.next_eligible];
    Measure* a = store.find(kFrame, t, t + 1);
    if (a->s[6] < static_thr_) {
      sh.next_eligible++;
      continue;
    }
    Measure* v0 = store.find(kUpperLower, t, t);
    Measure* v1 = store.find(kUpperLower, t, t + 1);
    Measure* v2 = store.find(kLowerUpper, t, t + 1);
    if (v0 && v1 && v2) {
      v0->used = v1->used = v2->used = true;
      sh.analysed.push_back({t, v0->act, v1->act, v2->act});
      sh.next_eligible++;
      continue;
    }
    // request this frame and every later eligible frame that will also vote
    size_t want = (size_t)p_.samp_max_frames - sh.analysed.size();
    for (size_t i = sh.next_eligible; i < sh.eligible.size() && want > 0; i++) {
      const int u = sh.eligible[i];
      if (store.find(kFrame, u, u + 1)->s[6] < static_thr_) continue;
      want--;
      if (!store.find(kUpperLower, u, u)) need.push_back(pair_key(kUpperLower, u, u));
      if (!store.find(kUpperLower, u, u + 1)) need.push_back(pair_key(kUpperLower, u, u + 1));
      if (!store.find(kLowerUpper, u, u + 1)) need.push_back(pair_key(kLowerUpper, u, u + 1));
    }
    return kNeedPairs;
  }
  return kProgress;
}

void Detector::classify(const Shot& sh, ShotOut& out) const {
  out.first = sh.first;
  out.last = sh.last;
  out.analysed = (int)sh.analysed.size();
  out.label = ANALYSER_UNKNOWN;
  out.field_order = ANALYSER_FO_NONE;
  out.phase = -1;
  const int n = (int)sh.analysed.size();
  if (n == 0) return;
  std::vector<char> combed(n);
  int ncombed = 0;
  for (int i = 0; i < n; i++) {
    const Sample& s = sh.analysed[i];
    const double mx = s.v1 >= s.v2 ? s.v1 : s.v2;
    const double c = p_.comb_ratio * mx;
    combed[i] = s.v0 > c;
    ncombed += combed[i] ? 1 : 0;
  }
  int best_phi = -1, best = -1;
  for (int phi = 0; phi < 5; phi++) {
    int match = 0;
    for (int i = 0; i < n; i++) {
      const int pos = ((sh.analysed[i].t - phi) % 5 + 5) % 5;
      const bool expect = pos == 2 || pos == 3;
      if ((combed[i] != 0) == expect) match++;
    }
    if (match > best) { best = match; best_phi = phi; }
  }
  const double need = p_.pulldown_match * (double)n;
  if ((double)best >= need) {
    out.label = ANALYSER_PULLDOWN;
    out.phase = best_phi;
    return;
  }
  std::vector<double> betas(n);
  for (int i = 0; i < n; i++) {
    const Sample& s = sh.analysed[i];
    betas[i] = s.v2 > 0.0 ? s.v1 / s.v2 : std::numeric_limits<double>::infinity();
  }
  std::sort(betas.begin(), betas.end());
  const double B = betas[(n - 1) / 2];
  const double ub = p_.unequal_ratio * B;
  if (2 * ncombed > n && (B > p_.unequal_ratio || ub < 1.0)) {
    out.label = ANALYSER_INTERLACED;
    out.field_order = B > 1.0 ? ANALYSER_FO_TFF : ANALYSER_FO_BFF;
    return;
  }
  out.label = ANALYSER_PROGRESSIVE;
}

void Detector::finish_clip() {
  shots = closed_out_;
  long long w[4] = {0, 0, 0, 0};
  long long fo_tff = 0, fo_bff = 0;
  int phase = -1, phase_n = 0;
  for (const ShotOut& s : shots) {
    if (s.label >= 1 && s.label <= 3) w[s.label] += s.analysed;
    if (s.label == ANALYSER_INTERLACED) {
      if (s.field_order == ANALYSER_FO_TFF) fo_tff += s.analysed;
      if (s.field_order == ANALYSER_FO_BFF) fo_bff += s.analysed;
    }
    if (s.label == ANALYSER_PULLDOWN && s.analysed > phase_n) { phase = s.phase; phase_n = s.analysed; }
  }
  clip_label = ANALYSER_UNKNOWN;
  long long best = 0;
  for (int lab = ANALYSER_PROGRESSIVE; lab <= ANALYSER_PULLDOWN; lab++)
    if (w[lab] > best) { best = w[lab]; clip_label = lab; }
  clip_fo = ANALYSER_FO_NONE;
  if (clip_label == ANALYSER_INTERLACED) {
    if (fo_tff > 0 && fo_tff >= fo_bff) clip_fo = ANALYSER_FO_TFF;
    else if (fo_bff > 0) clip_fo = ANALYSER_FO_BFF;
  }
  clip_phase = clip_label == ANALYSER_PULLDOWN ? phase : -1;
  done_ = true;
}

Detector::Status Detector::run(MeasureStore& store, int avail, bool finished, std::vector<uint64_t>& need) {
  if (done_) return kDone;
  if (finished) T_ = avail;
  if (T_ == 0) {
    open_.clear();
    keyframes.clear();
    finish_clip();
    return kDone;
  }
  Status shot_st;
  for (;;) {
    shot_st = shot_step(store, avail, finished, need);
    if (shot_st != kProgress) break;
  }
  bool sampling_waits = false;
  for (Shot& sh : open_) {
    if (sampling_step(store, sh, need) == kNeedPairs) sampling_waits = true;
  }
  // close shots (in order) whose boundaries and votes are final
  while (!open_.empty()) {
    Shot& sh = open_.front();
    const bool ended = sh.last >= 0;
    const bool votes_done = sh.analysed.size() >= (size_t)p_.samp_max_frames || sh.next_eligible >= sh.eligible.size();
    if (!(ended && votes_done)) break;
    if (open_.size() == 1 && shot_st != kDone) break;   // the current shot may still grow
    ShotOut o;
    classify(sh, o);
    closed_out_.push_back(o);
    open_.erase(open_.begin());
  }
  if (shot_st == kDone && open_.empty()) {
    finish_clip();
    return kDone;
  }
  if (!need.empty() || sampling_waits) return kNeedPairs;
  if (shot_st == kNeedPairs) return kNeedPairs;
  return shot_st == kDone ? kNeedPairs : kNeedFrames;
}

}  // namespace va
