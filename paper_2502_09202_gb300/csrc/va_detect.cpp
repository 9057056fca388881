// Detectors of Sec. III.B-D as a resumable state machine (see va_detect.h).
//
// Readings of what the paper leaves open (thresholds and window sizes are
// parameters, defaults in analyser_default_params):
//   fast check (III.B), generic: with at least `jback` predecessors of t in
//     the shot, t is a candidate iff a_t > max(fast_tau, fast_lambda * m_t)
//     (a jump) or a_t > max(fast_tau, fast_rise * m_t) and a_t < a_{t+1} <
//     a_{t+2} (a ramp starts; needs frame t+3, false at the clip end), m_t the
//     lower median of the last <= fast_window values a_s of the shot.
//   deep check (III.B), generic: for K = 1..kmax in order, with
//     p = max{ACT(t,t-j) : 1 <= j <= jback} and x << y as deep_rho*x +
//     deep_tau < y:
//       (a) p << ACT(t,t+K), p << ACT(t,t+K+1), a_{t+K} << ACT(t,t+K);
//       (b) ACT(t,t+K+1) <= (1 + done_eps) * ACT(t,t+K) (the transition is
//           complete at t+K);
//       (c) K >= 2: a_{t+K+d} <= steady_gamma * max of the next steady_frames
//           values, d = 0..steady_span-1 (the new shot is steady);
//     the first K meeting (a)-(c) wins, and a K >= 2 must also pass
//       (d) ACT(t,t+K) > lag_rho * ACT(t,t-K) when t-K is in the shot and
//       (e) ACT(t,t+K-1) >= blend_ratio * ACT(t,t+K),
//     or the check fails at t.  K = 1: hardcut at t+1; K >= 2: dissolve
//     (t,K), new shot from t+K.
//   3:2 pulldown shots (once their structure verdict is formed): candidates
//     only at (t - phase) mod 5 in {4, 0}, a_t > max(fast_tau, pd_rho * the
//     lower median of a_{t-5}, a_{t-10}, a_{t-15}); a hardcut at t+1 iff
//     a_t > pd_rho * a_{t-5}, a_{t+1} <= pd_gamma_new * a_{t-4} and
//     a_{t-1} <= pd_gamma_old * a_{t-6} (needs t-6 in the shot, frame t+2).
//   sampling structure (III.C): the first samp_max_frames frames t of a shot
//     with t+1 in the shot and S_amm(t,t+1) >= ceil(static_amm_px*65536*nb)
//     vote with the AMM parts A0, A1, A2 of v0, v1, v2; the first rep_probe
//     voters (all voters once one of those shows one) also read the
//     same-parity pairs for a repeated-field flag.  Pulldown iff every voter
//     has a flag and the best phase matches the 3:2 pattern (upper field
//     repeated at position 1, lower at 3) on >= pulldown_match of them;
//     otherwise interlaced iff most voters are combed (A0 > comb_ratio *
//     min(A1, A2)) and the lower median B of A1/A2 is off 1 by unequal_ratio
//     (B > 1: upper field first); otherwise progressive.  The verdict is
//     formed at the samp_max_frames-th vote and again when the shot ends.
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

// Pairs a generic deep check at t for span K reads before its first test.
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
  // ask for every later hypothesis' pairs in the same wave (they are only
  // reported once a rule reads them)
  auto request_from = [&](int K0) {
    for (int K2 = K0; K2 <= p_.kmax && t + K2 + 1 < avail; K2++) {
      std::vector<uint64_t> more;
      deep_pairs(t, K2, s0, p_.jback, more);
      for (uint64_t k : more)
        if (!store.find(key_kind(k), key_a(k), key_b(k))) need.push_back(k);
    }
    st = kNeedPairs;
    return 0;
  };
  auto a_of = [&](int u) { return store.find(kFrame, u, u + 1); };
  for (int K = 1; K <= p_.kmax; K++) {
    if (T >= 0 && t + K + 1 > T - 1) return 0;
    if (t + K + 1 >= avail) {
      if (!finished) st = kNeedFrames;
      return 0;
    }
    std::vector<uint64_t> keys;
    deep_pairs(t, K, s0, p_.jback, keys);
    for (uint64_t k : keys)
      if (!store.find(key_kind(k), key_a(k), key_b(k))) return request_from(K);
    double ref = 0.0;
    bool have_ref = false;
    for (int j = 1; j <= p_.jback; j++) {
      if (t - j < s0) continue;
      Measure* m = store.find(kFrame, t, t - j);
      use(m);
      if (!have_ref || m->act > ref) ref = m->act;
      have_ref = true;
    }
    Measure* fk = store.find(kFrame, t, t + K);
    Measure* fk1 = store.find(kFrame, t, t + K + 1);
    Measure* af = store.find(kFrame, t + K, t + K + 1);
    use(fk); use(fk1); use(af);
    const double x = fk->act, x1 = fk1->act;
    const double base = p_.deep_rho * ref + p_.deep_tau;
    const double after = p_.deep_rho * af->act + p_.deep_tau;
    if (!(base < x && base < x1 && after < x)) continue;                 // (a)
    const double done = (1.0 + p_.done_eps) * x;
    if (!(x1 <= done)) continue;                                          // (b)
    if (K >= 2) {
      // (c) frames up to t+K+steady_span+steady_frames, clipped at the clip end
      const int last_frame = t + K + p_.steady_span + p_.steady_frames;
      if (T < 0 && last_frame >= avail) {
        if (!finished) st = kNeedFrames;
        return 0;
      }
      bool steady = true;
      for (int d = 0; d < p_.steady_span && steady; d++) {
        if (T >= 0 && t + K + d + 1 > T - 1) break;
        Measure* cur = a_of(t + K + d);
        if (!cur) { need.push_back(pair_key(kFrame, t + K + d, t + K + d + 1)); st = kNeedPairs; return 0; }
        double mx = 0.0;
        bool any = false;
        for (int i = 1; i <= p_.steady_frames; i++) {
          const int u = t + K + d + i;
          if (T >= 0 && u + 1 > T - 1) continue;
          Measure* m = a_of(u);
          if (!m) { need.push_back(pair_key(kFrame, u, u + 1)); st = kNeedPairs; return 0; }
          if (!any || m->act > mx) mx = m->act;
          any = true;
        }
        const double lim = p_.steady_gamma * mx;
        if (any && cur->act > lim) steady = false;
      }
      if (!steady) continue;
      if (t - K >= s0) {                                                   // (d)
        Measure* lag = store.find(kFrame, t, t - K);
        if (!lag) {   // read only once (a)-(c) hold: not requested ahead
          need.push_back(pair_key(kFrame, t, t - K));
          st = kNeedPairs;
          return 0;
        }
        use(lag);
        const double lr = p_.lag_rho * lag->act;
        if (!(x > lr)) return 0;
      }
      Measure* prev = store.find(kFrame, t, t + K - 1);                    // (e), read by hypothesis K-1
      use(prev);
      const double br = p_.blend_ratio * x;
      if (!(prev->act >= br)) return 0;
    }
    return K;
  }
  return 0;
}

int Detector::deep_check_pulldown(MeasureStore& store, int t, int T, bool finished, int avail,
                                  std::vector<uint64_t>& need, Status& st) {
  const int s0 = open_.back().first;
  st = kProgress;
  if (t - 6 < s0 || (T >= 0 && t + 2 > T - 1)) return 0;
  if (t + 2 >= avail) {
    if (!finished) st = kNeedFrames;
    return 0;
  }
  Measure* m[8];   // a_{t-6} .. a_{t+1}
  for (int i = 0; i < 8; i++) {
    m[i] = store.find(kFrame, t - 6 + i, t - 5 + i);
    if (!m[i]) { need.push_back(pair_key(kFrame, t - 6 + i, t - 5 + i)); st = kNeedPairs; }
  }
  if (st == kNeedPairs) return 0;
  auto a = [&](int u) { return m[u - (t - 6)]->act; };
  const double r0 = p_.pd_rho * a(t - 5);
  if (!(a(t) > r0)) return 0;
  const double r1 = p_.pd_gamma_new * a(t - 4);
  if (!(a(t + 1) <= r1)) return 0;
  const double r2 = p_.pd_gamma_old * a(t - 6);
  if (!(a(t - 1) <= r2)) return 0;
  return 1;
}

Detector::Status Detector::shot_step(MeasureStore& store, int avail, bool finished, std::vector<uint64_t>& need) {
  Shot& cur = open_.back();
  if (T_ >= 0 && t_ >= T_ - 1) {
    if (cur.last < 0) cur.last = std::max(T_ - 1, cur.first);
    return kDone;
  }
  // the structure verdict is formed once the shot has samp_max_frames votes;
  // the rules for 3:2 pulldown shots apply from the frame after the last voter
  if (!cur.has_verdict && p_.samp_max_frames > 0 && cur.voters_seen >= p_.samp_max_frames) {
    if (cur.analysed.size() < (size_t)p_.samp_max_frames) return kNeedVotes;
    classify(cur, cur.verdict);
    cur.has_verdict = true;
  }
  if (t_ + 1 >= avail) return kNeedFrames;
  Measure* a = store.find(kFrame, t_, t_ + 1);
  if (!a) {
    need.push_back(pair_key(kFrame, t_, t_ + 1));
    return kNeedPairs;
  }
  use(a);
  const double at = a->act;
  const bool pulldown = cur.has_verdict && cur.verdict.label == ANALYSER_PULLDOWN;
  bool cand = false;
  // a speculative copy that passed over a pending deep check tests no frame
  // that a boundary found there would take
  const bool quiet = spec_ && t_ <= spec_quiet_;
  if ((int)hist_.size() >= p_.jback && !quiet) {
    if (pulldown) {
      const int pos = ((t_ - cur.verdict.phase) % 5 + 5) % 5;
      if ((pos == 4 || pos == 0) && t_ - 5 >= cur.first) {
        std::vector<double> v;
        for (int k = 1; k <= 3; k++)
          if (t_ - 5 * k >= cur.first) v.push_back(store.find(kFrame, t_ - 5 * k, t_ - 5 * k + 1)->act);
        const double m5 = lower_median(v, 0);
        const double l5 = p_.pd_rho * m5;
        const double thr = p_.fast_tau >= l5 ? p_.fast_tau : l5;
        cand = at > thr;
      }
    } else {
      const size_t from = hist_.size() > (size_t)p_.fast_window ? hist_.size() - (size_t)p_.fast_window : 0;
      const double m = lower_median(hist_, from);
      const double lm = p_.fast_lambda * m;
      const double thr = p_.fast_tau >= lm ? p_.fast_tau : lm;
      cand = at > thr;
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
            if (!spec_) return kNeedPairs;
          } else {
            cand = at < a1->act && a1->act < a2->act;
          }
        }
      }
    }
    if (cand) {
      Status st;
      int K = pulldown ? deep_check_pulldown(store, t_, T_, finished, avail, need, st)
                       : deep_check(store, t_, T_, finished, avail, need, st);
      if (st == kNeedPairs && spec_) {
        K = 0;   // a speculative copy goes on as if there were no boundary at t
        st = kProgress;
        spec_quiet_ = t_ + p_.kmax;
      }
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
  if (cur.voters_seen < p_.samp_max_frames && a->s[6] >= static_thr_) cur.voters_seen++;
  S_ += at;
  if (S_ > p_.kf_theta) {
    keyframes.push_back(t_ + 1);
    S_ = 0.0;
  }
  t_ += 1;
  return kProgress;
}

bool Detector::wants_reps(const Shot& sh, size_t voter) const {
  // voter is 0-based; the first rep_probe voters always read the same-parity
  // pairs, later ones only once a probe voter showed a repeated field
  if (voter < (size_t)p_.rep_probe) return true;
  for (int i = 0; i < p_.rep_probe && i < (int)sh.reps.size(); i++)
    if (sh.reps[i] != kRepNone) return true;
  return false;
}

Detector::Status Detector::sampling_step(MeasureStore& store, Shot& sh, std::vector<uint64_t>& need, bool& voted) {
  // Examine eligible frames in order; request the pairs of every frame that
  // will vote (decided by S_amm alone) in one go.
  while (sh.analysed.size() < (size_t)p_.samp_max_frames && sh.next_eligible < sh.eligible.size()) {
    const int t = sh.eligible[sh.next_eligible];
    Measure* a = store.find(kFrame, t, t + 1);
    if (a->s[6] < static_thr_) {
      sh.next_eligible++;
      continue;
    }
    const bool reps = wants_reps(sh, sh.analysed.size());
    Measure* v0 = store.find(kUpperLower, t, t);
    Measure* v1 = store.find(kUpperLower, t, t + 1);
    Measure* v2 = store.find(kLowerUpper, t, t + 1);
    Measure* ru = reps ? store.find(kUpperUpper, t, t + 1) : nullptr;
    Measure* rl = reps ? store.find(kLowerLower, t, t + 1) : nullptr;
    if (v0 && v1 && v2 && (!reps || (ru && rl))) {
      use(v0); use(v1); use(v2);
      sh.analysed.push_back({t, v0->amm, v1->amm, v2->amm});
      if (reps) {
        use(ru); use(rl);
        const double tu = p_.rep_ratio * rl->act, tl = p_.rep_ratio * ru->act;
        sh.reps.push_back(ru->act < tu ? kRepUpper : (rl->act < tl ? kRepLower : kRepNone));
      }
      sh.next_eligible++;
      voted = true;
      continue;
    }
    // request this frame and every later eligible frame that will also vote;
    // the same-parity pairs where it is already known that they are read
    size_t want = (size_t)p_.samp_max_frames - sh.analysed.size();
    size_t voter = sh.analysed.size();
    for (size_t i = sh.next_eligible; i < sh.eligible.size() && want > 0; i++) {
      const int u = sh.eligible[i];
      if (store.find(kFrame, u, u + 1)->s[6] < static_thr_) continue;
      want--;
      if (!store.find(kUpperLower, u, u)) need.push_back(pair_key(kUpperLower, u, u));
      if (!store.find(kUpperLower, u, u + 1)) need.push_back(pair_key(kUpperLower, u, u + 1));
      if (!store.find(kLowerUpper, u, u + 1)) need.push_back(pair_key(kLowerUpper, u, u + 1));
      const bool known = voter < (size_t)p_.rep_probe || (sh.reps.size() >= (size_t)p_.rep_probe);
      if (known && wants_reps(sh, voter)) {
        if (!store.find(kUpperUpper, u, u + 1)) need.push_back(pair_key(kUpperUpper, u, u + 1));
        if (!store.find(kLowerLower, u, u + 1)) need.push_back(pair_key(kLowerLower, u, u + 1));
      }
      voter++;
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
  if ((int)sh.reps.size() == n) {
    int best_phi = -1, best = -1;
    for (int phi = 0; phi < 5; phi++) {
      int match = 0;
      for (int i = 0; i < n; i++) {
        const int pos = ((sh.analysed[i].t - phi) % 5 + 5) % 5;
        const int expect = pos == 1 ? kRepUpper : (pos == 3 ? kRepLower : kRepNone);
        if (sh.reps[i] == expect) match++;
      }
      if (match > best) { best = match; best_phi = phi; }
    }
    const double need = p_.pulldown_match * (double)n;
    if ((double)best >= need) {
      out.label = ANALYSER_PULLDOWN;
      out.phase = best_phi;
      return;
    }
  }
  int ncombed = 0;
  std::vector<double> betas(n);
  for (int i = 0; i < n; i++) {
    const Vote& v = sh.analysed[i];
    const double mn = v.a1 <= v.a2 ? v.a1 : v.a2;
    const double c = p_.comb_ratio * mn;
    ncombed += v.a0 > c ? 1 : 0;
    betas[i] = v.a2 > 0.0 ? v.a1 / v.a2 : std::numeric_limits<double>::infinity();
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
  bool sampling_waits = false;
  for (;;) {
    for (;;) {
      shot_st = shot_step(store, avail, finished, need);
      if (shot_st != kProgress) break;
    }
    sampling_waits = false;
    bool voted = false;
    for (Shot& sh : open_) {
      if (sampling_step(store, sh, need, voted) == kNeedPairs) sampling_waits = true;
    }
    // votes cast just now may complete the verdict the shot detector waits for
    if (shot_st == kNeedVotes && voted) continue;
    break;
  }
  if (shot_st == kNeedVotes) shot_st = kNeedPairs;
  // Prefetch: when the shot detector waits for pairs (a deep check, a ramp
  // test or the structure verdict), a copy of the detectors runs on over the
  // frames already available as if the pending test found no boundary, and
  // asks for the pairs it reads; the next wave computes them beside the
  // pending ones.  The copy marks nothing as read and is discarded, so the
  // decisions and the reported measure set are those of the real run.
  if (!spec_ && shot_st == kNeedPairs && p_.prefetch_frames > 0) {
    Detector sp = *this;
    sp.spec_ = true;
    const int horizon = std::min(avail, t_ + p_.prefetch_frames);
    for (int guard = 0; guard < 1000000 && sp.t_ < horizon - 1; guard++) {
      const Status st = sp.shot_step(store, horizon, finished && horizon == avail, need);
      if (st != kProgress) break;
    }
    bool unused = false;
    for (Shot& sh : sp.open_) sp.sampling_step(store, sh, need, unused);
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
