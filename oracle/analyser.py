"""Oracle detectors: shot boundaries, sampling structure, dynamic keyframes.

Test infrastructure only (see oracle/__init__.py).  A plain sequential reading
of Sec. III.B-D over a whole clip, computing each pair measure on demand and
caching it (the on-demand measure framework of Sec. III.A).  The product path
implements the same rules independently in C++; the readings of what the paper
leaves open are listed here with their parameters.

Measures: a_t = ACT(t, t+1) is computed for every t (Sec. III.A: always).
Everything else is requested only when a rule reads it; the reported measure
set is exactly the set of pairs some rule read.

Shot detector (Sec. III.B).  Frames t of the current shot (first frame s0)
are tested in order once the shot holds >= J predecessors of t.
  fast check, generic: t is a candidate iff
      a_t > max(tau_f, lambda_f * m_t)                                 (a jump), or
      a_t > max(tau_f, lambda_r * m_t) and a_t < a_{t+1} < a_{t+2}      (a ramp starts)
    with m_t the lower median of the last <= W values a_s of the shot before t
    (the ramp test needs frame t+3; at the clip end it is false).
  deep check, generic, for K = 1 .. Kmax in order (needs frame t+K+1):
      p = max{ ACT(t, t-j) : 1 <= j <= J, t-j >= s0 }  (0 without predecessors)
      x << y  :=  rho * x + tau_d < y
      (a) p << ACT(t, t+K), p << ACT(t, t+K+1), a_{t+K} << ACT(t, t+K)
          (the paper's test, a persistence test against one-frame flashes, and
          a stable frame t+K);
      (b) completion: ACT(t, t+K+1) <= (1 + eps) * ACT(t, t+K): frame t+K is
          already as far from t as frame t+K+1 (frames inside a transition are
          blends, nearer to t than the frames after it);
      and for a dissolve hypothesis K >= 2:
      (c) the new shot is steady from t+K on: for d = 0 .. span-1 (pairs that
          exist), a_{t+K+d} <= gamma * max{ a_{t+K+d+i} : 1 <= i <= M };
    the first K meeting (a)-(c) is taken; for K >= 2 it must then also pass
      (d) ACT(t, t+K) > lambda_lag * ACT(t, t-K) when t-K >= s0 (more change
          across the transition than over the same number of frames back in
          the shot: motion alone grows ACT with the frame distance), and
      (e) ACT(t, t+K-1) >= beta * ACT(t, t+K) (frame t+K-1 already mostly
          shows the new shot: a transition, not an abrupt change at t+K),
    or the check fails at t.  K = 1 is a hardcut (new shot starts at t+1),
    K >= 2 a dissolve (t, K) whose new shot starts at t+K; frames t+1..t+K-1
    belong to no shot.
  Shots whose sampling structure is 3:2 pulldown with phase phi (decided by
  the sampling detector once the shot has N_s votes, below) are tested at the
  two clean steps of each 5-frame unit only, (t - phi) mod 5 in {4, 0} (both
  frames of the pair show one film frame in both fields): the cadence makes
  every other frame pair an unfair comparison (Sec. III.C: the pulldown
  pattern depends on the position in the unit).  With a5(u) = a_{u-5}, the
  same step one unit earlier:
      candidate iff t-5 >= s0 and a_t > max(tau_f, rho_pd * m5_t), m5_t the
          lower median of { a_{t-5k} : k = 1..3, t-5k >= s0 };
      hardcut at t+1 iff t-6 >= s0, t+2 <= T-1 and
          a_t > rho_pd * a_{t-5}          (the step across the boundary),
          a_{t+1} <= gamma_new * a_{t-4} (t+1 opens a steady shot),
          a_{t-1} <= gamma_old * a_{t-6} (t is an ordinary frame, not a flash).
Sampling structure (Sec. III.C), per shot: the first <= N_s frames t with t+1
  in the shot and S_amm(t, t+1) >= ceil(eps_s * 65536 * nb) vote with
      v0 = (u_t, l_t), v1 = (u_t, l_{t+1}), v2 = (l_t, u_{t+1})
  (ACT of those pairs, and A0, A1, A2 their AMM parts: the motion magnitude
  between the fields).  The first P voters, and every later voter once one
  of those showed a repeated field, also read the same-parity pairs
  r_u = ACT(u_t, u_{t+1}), r_l = ACT(l_t, l_{t+1}): repeated upper field iff
  r_u < theta_r * r_l, repeated lower field iff r_l < theta_r * r_u.
      pulldown   iff every voter has r_u, r_l and, for the best phase phi
                 (smallest on ties), the voters whose flag matches the 3:2
                 pattern (upper repeated at (t-phi) mod 5 = 1, lower repeated
                 at 3, neither elsewhere) number >= theta_pd * n;
      combed     : A0 > theta_c * min(A1, A2) (fields of one frame are as far
                   apart in motion as adjacent fields of two frames);
      beta       : A1 / A2 (+inf when A2 = 0); B = lower median over the voters;
      interlaced iff 2 * #combed > n and (B > theta_b or theta_b * B < 1);
                 upper field first iff B > 1, lower field first iff B < 1
                 (Sec. III.C: beta > 1 means upper field first);
      otherwise progressive; no voter: unknown.
  The verdict is formed when the N_s-th vote is cast (the pulldown rules of
  the shot detector apply from the next frame) and again when the shot ends.
Dynamic keyframes (Sec. III.D): the first frame of every shot; then for each
  later frame t of the shot S += a_{t-1}; when S > theta_kf, t is a keyframe
  and S = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dfield
from typing import Callable

import numpy as np

from .measures import (FRAME, LOWER_LOWER, LOWER_UPPER, UPPER_LOWER, UPPER_UPPER, SearchParams, measure,
                       pair_images, pair_record, finalise)

UNKNOWN, PROGRESSIVE, INTERLACED, PULLDOWN = 0, 1, 2, 3
FO_NONE, FO_TFF, FO_BFF = 0, 1, 2
LABEL_NAMES = {UNKNOWN: "unknown", PROGRESSIVE: "progressive", INTERLACED: "interlaced", PULLDOWN: "pulldown"}
FO_NAMES = {FO_NONE: "none", FO_TFF: "tff", FO_BFF: "bff"}
REP_NONE, REP_UPPER, REP_LOWER = 0, 1, 2


@dataclass(frozen=True)
class Params:
    search: SearchParams = SearchParams()
    kmax: int = 8                 # largest dissolve span K tested (paper: 4; the dissolves to detect need 7)
    jback: int = 2                # J: predecessors in the shot needed before a fast check
    fast_window: int = 8          # W: history for the median
    fast_lambda: float = 2.0      # lambda_f
    fast_rise: float = 1.3        # lambda_r (ramp start)
    fast_tau: float = 0.5         # tau_f
    deep_rho: float = 2.0         # rho
    deep_tau: float = 0.5         # tau_d
    done_eps: float = 0.25        # eps (completion)
    steady_gamma: float = 1.2     # gamma (steady new shot)
    steady_frames: int = 4        # M
    steady_span: int = 2          # span
    lag_rho: float = 1.5          # lambda_lag
    blend_ratio: float = 0.6      # beta
    pd_rho: float = 1.4           # rho_pd
    pd_gamma_new: float = 2.5     # gamma_new
    pd_gamma_old: float = 1.4     # gamma_old
    samp_max_frames: int = 20     # N_s (paper: 15 to 20)
    static_amm_px: float = 0.5    # eps_s
    comb_ratio: float = 0.65      # theta_c
    unequal_ratio: float = 1.04   # theta_b
    rep_ratio: float = 0.25       # theta_r
    rep_probe: int = 5            # P: voters that always read the same-parity pairs
    pulldown_match: float = 0.8   # theta_pd
    kf_theta: float = 8.0         # theta_kf


def lower_median(values):
    s = sorted(values)
    return s[(len(s) - 1) // 2]


@dataclass
class _Shot:
    first: int
    last: int = -1
    analysed: list = dfield(default_factory=list)   # (t, A0, A1, A2) of every voter
    reps: list = dfield(default_factory=list)       # repeated-field flag of voters 1, 2, ...
    verdict: tuple | None = None                     # (label, field order, phase) after N_s votes


class OracleAnalyser:
    """Runs the detectors over frames 0..T-1 given by ``frame(t)``."""

    def __init__(self, frame: Callable[[int], np.ndarray], nframes: int, params: Params = Params(),
                 precomputed: dict | None = None):
        self.frame = frame
        self.T = nframes
        self.p = params
        self.cache: dict = dict(precomputed or {})
        self._frames: dict = {}
        self._read: set = set()

    # ---- measures -----------------------------------------------------------
    def _img(self, t):
        f = self._frames.get(t)
        if f is None:
            if len(self._frames) > 24:
                self._frames.pop(next(iter(self._frames)))
            f = self.frame(t)
            self._frames[t] = f
        return f

    def _measure(self, kind: int, a: int, b: int) -> dict:
        """The measure of one pair, computed from the frames (a subclass may
        serve measures from elsewhere)."""
        return measure(kind, self._img(a), self._img(b), self.p.search)

    def m(self, kind: int, a: int, b: int) -> dict:
        """A rule reads the measure of pair (kind, a, b): cached, and reported."""
        key = (kind, a, b)
        self._read.add(key)
        r = self.cache.get(key)
        if r is None:
            r = self._measure(kind, a, b)
            self.cache[key] = r
        return r

    def act(self, kind, a, b) -> float:
        return self.m(kind, a, b)["act"]

    def a(self, t) -> float:
        """a_t = ACT(t, t+1)."""
        return self.act(FRAME, t, t + 1)

    # ---- shot detector: deep checks -------------------------------------------
    def _deep_check(self, t: int, s0: int) -> int:
        p, T = self.p, self.T
        for K in range(1, p.kmax + 1):
            if t + K + 1 > T - 1:
                return 0
            back = [self.act(FRAME, t, t - j) for j in range(1, p.jback + 1) if t - j >= s0]
            ref = max(back) if back else 0.0
            x = self.act(FRAME, t, t + K)
            x1 = self.act(FRAME, t, t + K + 1)
            after = self.a(t + K)
            base = p.deep_rho * ref + p.deep_tau
            if not (base < x and base < x1 and p.deep_rho * after + p.deep_tau < x):     # (a)
                continue
            if not x1 <= (1.0 + p.done_eps) * x:                                       # (b)
                continue
            if K >= 2:
                steady = True                                                          # (c)
                for d in range(p.steady_span):
                    if t + K + d + 1 > T - 1:
                        break
                    nxt = [self.a(t + K + d + i) for i in range(1, p.steady_frames + 1) if t + K + d + i + 1 <= T - 1]
                    if nxt and self.a(t + K + d) > p.steady_gamma * max(nxt):
                        steady = False
                        break
                if not steady:
                    continue
                if t - K >= s0 and not x > p.lag_rho * self.act(FRAME, t, t - K):      # (d)
                    return 0
                if not self.act(FRAME, t, t + K - 1) >= p.blend_ratio * x:             # (e)
                    return 0
            return K
        return 0

    def _deep_check_pulldown(self, t: int, s0: int) -> int:
        p = self.p
        if t - 6 < s0 or t + 2 > self.T - 1:
            return 0
        if not self.a(t) > p.pd_rho * self.a(t - 5):
            return 0
        if not self.a(t + 1) <= p.pd_gamma_new * self.a(t - 4):
            return 0
        if not self.a(t - 1) <= p.pd_gamma_old * self.a(t - 6):
            return 0
        return 1

    # ---- sampling structure ------------------------------------------------------
    def _repeat_flag(self, t: int) -> int:
        ru = self.act(UPPER_UPPER, t, t + 1)
        rl = self.act(LOWER_LOWER, t, t + 1)
        if ru < self.p.rep_ratio * rl:
            return REP_UPPER
        if rl < self.p.rep_ratio * ru:
            return REP_LOWER
        return REP_NONE

    def _vote(self, shot: _Shot, t: int):
        p = self.p
        A0 = self.m(UPPER_LOWER, t, t)["amm"]
        A1 = self.m(UPPER_LOWER, t, t + 1)["amm"]
        A2 = self.m(LOWER_UPPER, t, t + 1)["amm"]
        shot.analysed.append((t, A0, A1, A2))
        k = len(shot.analysed)
        if k <= p.rep_probe or any(r != REP_NONE for r in shot.reps[:p.rep_probe]):
            shot.reps.append(self._repeat_flag(t))
        if k == p.samp_max_frames:
            shot.verdict = self._classify(shot)

    def _classify(self, shot: _Shot):
        p = self.p
        A = shot.analysed
        n = len(A)
        if n == 0:
            return UNKNOWN, FO_NONE, -1
        if len(shot.reps) == n:
            want = {1: REP_UPPER, 3: REP_LOWER}
            best_phi, best = -1, -1
            for phi in range(5):
                match = sum(1 for (t, *_), r in zip(A, shot.reps) if r == want.get((t - phi) % 5, REP_NONE))
                if match > best:
                    best_phi, best = phi, match
            if best >= p.pulldown_match * n:
                return PULLDOWN, FO_NONE, best_phi
        combed = [A0 > p.comb_ratio * min(A1, A2) for _, A0, A1, A2 in A]
        betas = [A1 / A2 if A2 > 0.0 else math.inf for _, A0, A1, A2 in A]
        B = lower_median(betas)
        if 2 * sum(combed) > n and (B > p.unequal_ratio or p.unequal_ratio * B < 1.0):
            fo = FO_TFF if B > 1.0 else FO_BFF
            return INTERLACED, fo, -1
        return PROGRESSIVE, FO_NONE, -1

    # ---- the clip -----------------------------------------------------------------
    def run(self) -> dict:
        p, T = self.p, self.T
        for t in range(T - 1):          # always-on pairs, in order
            self.m(FRAME, t, t + 1)
        cuts, dissolves, keyframes, shots = [], [], [], []
        if T <= 0:
            return self._results(cuts, dissolves, keyframes, shots)
        h, w = self._img(0).shape
        nb = (w // p.search.block) * (h // p.search.block)
        static_thr = math.ceil(p.static_amm_px * 65536.0 * float(nb))
        shot = _Shot(first=0)
        keyframes.append(0)
        hist: list[float] = []
        S = 0.0
        t = 0
        while t < T - 1:
            a_t = self.a(t)
            cand = False
            pulldown = shot.verdict is not None and shot.verdict[0] == PULLDOWN
            if len(hist) >= p.jback:
                if pulldown:
                    phi = shot.verdict[2]
                    if (t - phi) % 5 in (4, 0) and t - 5 >= shot.first:
                        m5 = lower_median([self.a(t - 5 * k) for k in (1, 2, 3) if t - 5 * k >= shot.first])
                        cand = a_t > max(p.fast_tau, p.pd_rho * m5)
                else:
                    m_t = lower_median(hist[-p.fast_window:])
                    cand = a_t > max(p.fast_tau, p.fast_lambda * m_t)
                    if not cand and t + 3 <= T - 1 and a_t > max(p.fast_tau, p.fast_rise * m_t):
                        a1 = self.a(t + 1)
                        a2 = self.a(t + 2)
                        cand = a_t < a1 < a2
            if cand:
                K = self._deep_check_pulldown(t, shot.first) if pulldown else self._deep_check(t, shot.first)
                if K:
                    shot.last = t
                    shots.append(shot)
                    if K == 1:
                        cuts.append(t + 1)
                    else:
                        dissolves.append((t, K))
                    t = t + K
                    shot = _Shot(first=t)
                    keyframes.append(t)
                    hist = []
                    S = 0.0
                    continue
            # no boundary after t: frame t+1 belongs to the shot
            hist.append(a_t)
            if len(shot.analysed) < p.samp_max_frames and self.m(FRAME, t, t + 1)["samm"] >= static_thr:
                self._vote(shot, t)
            S += a_t
            if S > p.kf_theta:
                keyframes.append(t + 1)
                S = 0.0
            t += 1
        shot.last = T - 1
        shots.append(shot)
        return self._results(cuts, dissolves, keyframes, shots)

    def _results(self, cuts, dissolves, keyframes, shots) -> dict:
        out_shots = []
        weight = {PROGRESSIVE: 0, INTERLACED: 0, PULLDOWN: 0}
        fo_w = {FO_TFF: 0, FO_BFF: 0}
        phase_best, phase_n = -1, 0
        for sh in shots:
            label, fo, phase = self._classify(sh)
            n = len(sh.analysed)
            out_shots.append({"first": sh.first, "last": sh.last, "label": label, "field_order": fo,
                              "phase": phase, "analysed": n})
            if label in weight:
                weight[label] += n
            if label == INTERLACED and fo in fo_w:
                fo_w[fo] += n
            if label == PULLDOWN and n > phase_n:
                phase_best, phase_n = phase, n
        clip_label = UNKNOWN
        best = 0
        for lab in (PROGRESSIVE, INTERLACED, PULLDOWN):
            if weight[lab] > best:
                clip_label, best = lab, weight[lab]
        clip_fo = FO_NONE
        if clip_label == INTERLACED:
            if fo_w[FO_TFF] > 0 and fo_w[FO_TFF] >= fo_w[FO_BFF]:
                clip_fo = FO_TFF
            elif fo_w[FO_BFF] > 0:
                clip_fo = FO_BFF
        return {
            "cuts": cuts, "dissolves": dissolves, "keyframes": keyframes, "shots": out_shots,
            "label": clip_label, "field_order": clip_fo,
            "pulldown_phase": phase_best if clip_label == PULLDOWN else -1,
            "measures": dict(sorted((k, v) for k, v in self.cache.items() if k in self._read)),
        }


# ---- parallel always-on pairs (the oracle's CPU baseline uses this) -----------

def _pair_job(args):
    spec, kind, a, b, search = args
    from paper_2502_09202_gb300.synth import Clip
    clip = Clip(spec)
    return (kind, a, b), measure(kind, clip.frame(a), clip.frame(b), search)


def _chunk_job(args):
    spec, start, stop, search = args
    from paper_2502_09202_gb300.synth import Clip
    clip = Clip(spec)
    out = {}
    prev = clip.frame(start)
    for t in range(start, stop):
        nxt = clip.frame(t + 1)
        out[(FRAME, t, t + 1)] = measure(FRAME, prev, nxt, search)
        prev = nxt
    return out


def always_on_parallel(spec, params: Params = Params(), workers: int = 8, chunk: int = 16) -> dict:
    """ACT(t, t+1) for every t of a synthetic clip, over a spawn-started process pool."""
    import multiprocessing as mp
    T = spec.nframes
    jobs = [(spec, s, min(s + chunk, T - 1), params.search) for s in range(0, T - 1, chunk)]
    out = {}
    if workers <= 1:
        for j in jobs:
            out.update(_chunk_job(j))
        return out
    with mp.get_context("spawn").Pool(workers) as pool:
        for d in pool.imap_unordered(_chunk_job, jobs):
            out.update(d)
    return out


def analyse_spec(spec, params: Params = Params(), workers: int = 0) -> dict:
    """Run the oracle over a synthetic clip (optionally with the always-on pairs in parallel)."""
    from paper_2502_09202_gb300.synth import Clip
    clip = Clip(spec)
    pre = always_on_parallel(spec, params, workers) if workers > 1 else None
    return OracleAnalyser(clip.frame, spec.nframes, params, precomputed=pre).run()


def analyse_frames(frames: np.ndarray, params: Params = Params()) -> dict:
    return OracleAnalyser(lambda t: frames[t], len(frames), params).run()
