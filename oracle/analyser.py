"""Oracle detectors: shot boundaries, sampling structure, dynamic keyframes.

Test infrastructure only (see oracle/__init__.py).  A plain sequential reading
of Sec. III.B-D over a whole clip, computing each pair measure on demand and
caching it (the on-demand measure framework of Sec. III.A).  The product path
implements the same rules independently in C++; the readings of what the paper
leaves open are listed with the parameters below.

Measures: a_t = ACT(t, t+1) is computed for every t (Sec. III.A: always).
Everything else is requested only when a rule needs it.

Shot detector (Sec. III.B)
  fast check at t: the shot holds >= J predecessors of t and either
      a_t > max(tau_f, lambda_f * m_t)                       (a jump), or
      a_t > max(tau_f, lambda_r * m_t) and a_t < a_{t+1} < a_{t+2}   (the start of a ramp)
      with m_t = lower median of the last <= W values a_s of the current shot
      before t (the ramp test needs frame t+3; at the clip end it is false).
  deep check at a candidate t, for K = 1 .. Kmax in order (needs frame t+K+1):
      p = max{ ACT(t, t-j) : 1 <= j <= J }   (predecessors in the shot)
      "x significantly smaller than y" := rho * x + tau_d < y
      K is valid iff p << ACT(t, t+K), p << ACT(t, t+K+1) and a_{t+K} << ACT(t, t+K)
      The smallest valid K wins: K = 1 is a hardcut (new shot starts at t+1),
      K >= 2 a dissolve (t, K) whose new shot starts at t+K; frames t+1..t+K-1
      belong to no shot.
Sampling structure (Sec. III.C), per shot, on the first <= N_s frames t of the
  shot with t+1 in the shot and S_amm(t, t+1) >= ceil(eps_s * 65536 * nb):
      v0 = ACT(u_t, l_t), v1 = ACT(u_t, l_{t+1}), v2 = ACT(l_t, u_{t+1})
      combed  : v0 > theta_p * max(v1, v2)
      beta    : v1 / v2 (+inf when v2 = 0); B = lower median of beta over the shot
  pulldown   iff for the best phase phi (smallest on ties) the frames with
             combed == ((t - phi) mod 5 in {2, 3}) number >= theta_pd * n
  interlaced iff 2 * #combed > n and (B > theta_b or theta_b * B < 1);
             upper field first iff B > 1, lower field first iff B < 1
  otherwise progressive; no analysed frame: unknown.
Dynamic keyframes (Sec. III.D): the first frame of every shot; then for each
  later frame t of the shot S += a_{t-1}; when S > theta_kf, t is a keyframe
  and S = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dfield
from typing import Callable

import numpy as np

from .measures import FRAME, LOWER_UPPER, UPPER_LOWER, SearchParams, measure, pair_images, pair_record, finalise

UNKNOWN, PROGRESSIVE, INTERLACED, PULLDOWN = 0, 1, 2, 3
FO_NONE, FO_TFF, FO_BFF = 0, 1, 2
LABEL_NAMES = {UNKNOWN: "unknown", PROGRESSIVE: "progressive", INTERLACED: "interlaced", PULLDOWN: "pulldown"}
FO_NAMES = {FO_NONE: "none", FO_TFF: "tff", FO_BFF: "bff"}


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
    samp_max_frames: int = 20     # N_s (paper: 15 to 20)
    static_amm_px: float = 0.5    # eps_s
    comb_ratio: float = 0.3       # theta_p
    unequal_ratio: float = 1.12   # theta_b
    pulldown_match: float = 0.8   # theta_pd
    kf_theta: float = 8.0         # theta_kf


def lower_median(values):
    s = sorted(values)
    return s[(len(s) - 1) // 2]


@dataclass
class _Shot:
    first: int
    last: int = -1
    analysed: list = dfield(default_factory=list)   # (t, v0, v1, v2)


class OracleAnalyser:
    """Runs the detectors over frames 0..T-1 given by ``frame(t)``."""

    def __init__(self, frame: Callable[[int], np.ndarray], nframes: int, params: Params = Params(),
                 precomputed: dict | None = None):
        self.frame = frame
        self.T = nframes
        self.p = params
        self.cache: dict = dict(precomputed or {})
        self._frames: dict = {}

    # ---- measures -----------------------------------------------------------
    def _img(self, t):
        f = self._frames.get(t)
        if f is None:
            if len(self._frames) > 24:
                self._frames.pop(next(iter(self._frames)))
            f = self.frame(t)
            self._frames[t] = f
        return f

    def m(self, kind: int, a: int, b: int) -> dict:
        key = (kind, a, b)
        r = self.cache.get(key)
        if r is None:
            r = measure(kind, self._img(a), self._img(b), self.p.search)
            self.cache[key] = r
        return r

    def act(self, kind, a, b) -> float:
        return self.m(kind, a, b)["act"]

    # ---- detectors ----------------------------------------------------------
    def _deep_check(self, t: int, s0: int) -> int:
        p = self.p
        for K in range(1, p.kmax + 1):
            if t + K + 1 > self.T - 1:
                break
            back = [self.act(FRAME, t, t - j) for j in range(1, p.jback + 1) if t - j >= s0]
            ref = max(back) if back else 0.0
            fwd_k = self.act(FRAME, t, t + K)
            fwd_k1 = self.act(FRAME, t, t + K + 1)
            after = self.act(FRAME, t + K, t + K + 1)
            if (p.deep_rho * ref + p.deep_tau < fwd_k and p.deep_rho * ref + p.deep_tau < fwd_k1
                    and p.deep_rho * after + p.deep_tau < fwd_k):
                return K
        return 0

    def _classify(self, shot: _Shot):
        p = self.p
        A = shot.analysed
        n = len(A)
        if n == 0:
            return UNKNOWN, FO_NONE, -1
        combed = [v0 > p.comb_ratio * max(v1, v2) for _, v0, v1, v2 in A]
        best_phi, best = -1, -1
        for phi in range(5):
            match = sum(1 for (t, *_), c in zip(A, combed) if c == (((t - phi) % 5) in (2, 3)))
            if match > best:
                best_phi, best = phi, match
        if best >= p.pulldown_match * n:
            return PULLDOWN, FO_NONE, best_phi
        betas = [v1 / v2 if v2 > 0.0 else math.inf for _, v0, v1, v2 in A]
        B = lower_median(betas)
        if 2 * sum(combed) > n and (B > p.unequal_ratio or p.unequal_ratio * B < 1.0):
            fo = FO_TFF if B > 1.0 else FO_BFF
            return INTERLACED, fo, -1
        return PROGRESSIVE, FO_NONE, -1

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
            a_t = self.act(FRAME, t, t + 1)
            cand = False
            if len(hist) >= p.jback:
                m_t = lower_median(hist[-p.fast_window:])
                thr = max(p.fast_tau, p.fast_lambda * m_t)
                cand = a_t > thr
                if not cand and t + 3 <= T - 1 and a_t > max(p.fast_tau, p.fast_rise * m_t):
                    a1 = self.act(FRAME, t + 1, t + 2)
                    a2 = self.act(FRAME, t + 2, t + 3)
                    cand = a_t < a1 < a2
            if cand:
                K = self._deep_check(t, shot.first)
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
                v0 = self.act(UPPER_LOWER, t, t)
                v1 = self.act(UPPER_LOWER, t, t + 1)
                v2 = self.act(LOWER_UPPER, t, t + 1)
                shot.analysed.append((t, v0, v1, v2))
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
            "measures": dict(sorted(self.cache.items())),
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
