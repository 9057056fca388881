"""Pins for the oracle's detectors (Sec. III.B-D) on scripted measures.

The detectors read pair measures only through ``OracleAnalyser.m``; here a
subclass serves hand-made ACT, AMM and S_amm values instead of computing them
from frames, and each expected outcome below is derived by hand from the rules
(fast check, deep check with its completion, steadiness, lag and blend tests,
the rules for 3:2 pulldown shots, keyframe accumulation, sampling structure),
not by running the oracle.  A dropped condition, a wrong index (t - j for
t + j, K for K + 1) or a swapped field pair changes an outcome.
"""
import math

import numpy as np
import pytest

from oracle import analyser as OA
from oracle.measures import FRAME, LOWER_LOWER, LOWER_UPPER, UPPER_LOWER, UPPER_UPPER

W = H = 32                                   # 4 blocks of 16 x 16
STATIC = math.ceil(0.5 * 65536 * 4)          # S_amm threshold for "not static"


class Scripted(OA.OracleAnalyser):
    """act(kind, a, b): ACT; samm(a, b): S_amm of frame pairs; amm(kind, a, b):
    AMM of field pairs (the motion part the structure rules read)."""

    def __init__(self, T, act, samm=None, amm=None, params=OA.Params()):
        super().__init__(lambda t: np.zeros((H, W), np.uint8), T, params)
        self._act = act
        self._samm = samm or (lambda a, b: 0)
        self._amm = amm or (lambda kind, a, b: 0.0)

    def _measure(self, kind, a, b):
        return {"act": float(self._act(kind, a, b)),
                "samm": int(self._samm(a, b)) if kind == FRAME else 0,
                "amm": float(self._amm(kind, a, b)) if kind != FRAME else 0.0}


def positions(p, g=0.0):
    """ACT between frames a != b of one kind = 1 + g |a - b| + 9 |p(a) - p(b)|:
    1.0 inside a shot (growing by g per frame of distance) and 10.0 across a
    hard change."""
    def act(kind, a, b):
        return 1.0 + g * abs(a - b) + 9.0 * abs(p(a) - p(b))
    return act


def requested(o):
    """Frame pairs other than the always-on (t, t+1) the detectors read."""
    return sorted((a, b) for (k, a, b) in o.run()["measures"] if k == FRAME and b != a + 1)


def test_hard_cut():
    # a_6 = 10 against a median of 1: candidate; K = 1: p = max(ACT(6,5), ACT(6,4)) = 1,
    # 2*1 + 0.5 < ACT(6,7) = ACT(6,8) = 10 and 2*a_7 + 0.5 < 10; complete: 10 <= 1.25 * 10
    o = Scripted(12, positions(lambda f: 0.0 if f <= 6 else 1.0))
    r = o.run()
    assert r["cuts"] == [7] and r["dissolves"] == []
    assert [(s["first"], s["last"]) for s in r["shots"]] == [(0, 6), (7, 11)]
    assert r["keyframes"] == [0, 7]
    assert requested(o) == [(6, 4), (6, 5), (6, 8)]
    assert r["label"] == OA.UNKNOWN            # every pair static: nothing analysed


def test_dissolve_end_needs_a_stable_frame():
    # positions 0 | 1/3, 2/3 | 1: K = 1 and K = 2 fail on a_{t+K} << ACT(t, t+K)
    # (2*4 + 0.5 = 8.5 is not below 4, resp. 7); K = 3: 2*1 + 0.5 < 10, complete
    # (10 <= 12.5), steady (a_13 = a_14 = 1 <= 1.2 * 1), lag: 10 > 1.5 * ACT(10,7) = 1.5,
    # blend: ACT(10,12) = 7 >= 0.6 * 10
    p = {11: 1 / 3, 12: 2 / 3}
    o = Scripted(20, positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.0)))
    r = o.run()
    assert r["cuts"] == [] and r["dissolves"] == [(10, 3)]
    assert [(s["first"], s["last"]) for s in r["shots"]] == [(0, 10), (13, 19)]
    # S = a_0 + ... + a_8 = 9 > 8 makes frame 9 a keyframe; the six frames of
    # the second shot add 6
    assert r["keyframes"] == [0, 9, 13]
    assert requested(o) == [(10, 7), (10, 8), (10, 9), (10, 12), (10, 13), (10, 14)]


def test_completion_rejects_a_cut_inside_a_transition():
    # positions 0 | 0.5, 0.66 | 1: at K = 1, p << ACT(10,11) = 5.5, p << ACT(10,12) = 6.94
    # and 2*a_11 + 0.5 = 5.38 < 5.5 all hold, but frame 12 is farther from 10 than frame 11
    # (6.94 > 1.25 * 5.5): not complete.  K = 2 fails 2*a_12 + 0.5 < 6.94 (a_12 = 4.06);
    # K = 3: ACT(10,13) = 10, complete, steady, lag 10 > 1.5, blend 6.94 >= 6
    p = {11: 0.5, 12: 0.66}
    r = Scripted(20, positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.0))).run()
    assert r["cuts"] == [] and r["dissolves"] == [(10, 3)]


def test_dissolve_needs_a_steady_new_shot():
    # positions 0 | 0.5 | 1, then the new shot keeps moving for one more frame
    # (p(13) = 1.1): K = 2 passes (a), completion (10.9 <= 12.5) but a_12 = 1.9 >
    # 1.2 * max(a_13..a_16) = 1.2; d = 1 is not reached.  K = 3: ACT(10,13) = 10.9,
    # x1 = ACT(10,14) = 10.9, a_13 = 1 << 10.9, steady, lag 10.9 > 1.5, blend:
    # ACT(10,12) = 10 >= 0.6 * 10.9
    p = {11: 0.5, 12: 1.0}
    o = Scripted(24, positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.1)))
    r = o.run()
    assert r["dissolves"] == [(10, 3)] and r["cuts"] == []


def test_ramp_start_is_a_candidate_below_the_jump_threshold():
    # positions 0 | 0.1, 0.35, 0.65 | 1: a_10 = 1.9 < 2 * median (no jump) but > 1.3 * median
    # and a_10 < a_11 = 3.25 < a_12 = 3.7: a candidate.  K = 1, 2, 3 fail (a); K = 4:
    # ACT(10,14) = 10, a_14 = 1, complete, steady, lag: 10 > 1.5 * ACT(10,6) = 1.5,
    # blend: ACT(10,13) = 6.85 >= 6
    steps = {11: 0.1, 12: 0.35, 13: 0.65}
    o = Scripted(20, positions(lambda f: 0.0 if f <= 10 else steps.get(f, 1.0)))
    r = o.run()
    assert r["dissolves"] == [(10, 4)] and r["cuts"] == []
    assert r["keyframes"] == [0, 9, 14]
    assert requested(o) == [(10, 6), (10, 8), (10, 9), (10, 12), (10, 13), (10, 14), (10, 15)]


def test_motion_across_many_frames_is_no_dissolve():
    # a one-frame flash at 11 (p = 1) in a shot whose ACT grows by 0.5 per frame of
    # distance: a_10 = 10.5 is a candidate.  K = 1 fails persistence (ACT(10,12) = 2 is
    # not above 2 * 2 + 0.5); K = 2..7 fail p << ACT(10,10+K) = 1 + 0.5K; K = 8 passes
    # (a)-(c) (5 > 4.5, 5.5 > 4.5, 2*1.5 + 0.5 < 5; 5.5 <= 6.25; steady), but the lag
    # test rejects it: ACT(10,18) = 5 is not above 1.5 * ACT(10,2) = 7.5
    o = Scripted(30, positions(lambda f: 1.0 if f == 11 else 0.0, g=0.5))
    r = o.run()
    assert r["cuts"] == [] and r["dissolves"] == []
    assert (FRAME, 10, 2) in r["measures"]


def test_an_abrupt_change_is_no_dissolve_from_an_earlier_frame():
    # ACT grows by 0.3 per frame of distance and the new shot starts at 16.  A deep
    # check at 10 finds K = 6 first (ACT(10,16) = 11.8 against 2 * 1.6 + 0.5; complete;
    # steady; lag 11.8 > 1.5 * 2.8), but frame 15 is no blend: ACT(10,15) = 2.5 < 0.6 * 11.8.
    # The run itself finds the hardcut at 16 from t = 15.
    act = positions(lambda f: 0.0 if f <= 15 else 1.0, g=0.3)
    o = Scripted(30, act)
    assert o._deep_check(10, 0) == 0
    r = Scripted(30, act).run()
    assert r["cuts"] == [16] and r["dissolves"] == []


def test_falling_activity_is_no_ramp():
    # same jump-free start, but a_11 < a_10: no candidate anywhere
    steps = {11: 0.5 / 9, 12: 0.6 / 9, 13: 0.7 / 9}
    o = Scripted(20, positions(lambda f: 0.0 if f <= 10 else steps.get(f, steps[13])))
    r = o.run()
    assert r["cuts"] == [] and r["dissolves"] == [] and requested(o) == []


def test_candidate_needs_j_predecessors():
    # a jump at t = 1 has one predecessor in the shot (J = 2): not checked
    o = Scripted(8, positions(lambda f: 0.0 if f <= 1 else 1.0))
    r = o.run()
    assert r["cuts"] == [] and requested(o) == []


def test_keyframes_every_third_frame_at_constant_activity():
    # a_t = 3 (no candidate: 3 < 2 * 3 and 3 < 1.3 * 3): S passes 8 after three
    # frames, so frames 3, 6, 9 are keyframes; a_9 + a_10 = 6 leaves 12 out
    o = Scripted(12, lambda k, a, b: 3.0)
    assert o.run()["keyframes"] == [0, 3, 6, 9]


# ---- sampling structure ---------------------------------------------------------

def _structure(A, rep=None, T=30):
    """Clip whose every adjacent pair moves (S_amm at the threshold), whose field
    pairs (u_t,l_t), (u_t,l_t+1), (l_t,u_t+1) have AMM A(t) = (A0, A1, A2) and whose
    same-parity pairs have ACT rep(t) = (ACT(u_t,u_t+1), ACT(l_t,l_t+1))."""
    rep = rep or (lambda t: (1.0, 1.0))

    def act(kind, a, b):
        if kind == FRAME:
            return 1.0
        if kind == UPPER_UPPER:
            return rep(a)[0]
        if kind == LOWER_LOWER:
            return rep(a)[1]
        return 1.0

    def amm(kind, a, b):
        A0, A1, A2 = A(a)
        if kind == UPPER_LOWER:
            return A0 if a == b else A1
        if kind == LOWER_UPPER:
            return A2
        return 1.0

    o = Scripted(T, act, samm=lambda a, b: STATIC, amm=amm)
    return o.run()


def test_structure_interlaced_upper_field_first():
    # combed: 1 > 0.65 * min(3, 1); B = 3 > 1.04
    r = _structure(lambda t: (1.0, 3.0, 1.0))
    assert (r["label"], r["field_order"]) == (OA.INTERLACED, OA.FO_TFF)
    assert r["shots"][0]["analysed"] == 20          # N_s frames of the shot


def test_structure_interlaced_lower_field_first():
    r = _structure(lambda t: (1.0, 1.0, 3.0))
    assert (r["label"], r["field_order"]) == (OA.INTERLACED, OA.FO_BFF)


def test_structure_combed_but_balanced_fields_is_not_interlaced():
    # every frame combed, but B = 1 is inside (1/theta_b, theta_b)
    assert _structure(lambda t: (1.0, 1.0, 1.0))["label"] == OA.PROGRESSIVE


def test_structure_unequal_fields_without_combing_is_progressive():
    # B = 2 is off 1, but A0 = 0.3 < 0.65 * min(2, 1): the fields of a frame do not move apart
    assert _structure(lambda t: (0.3, 2.0, 1.0))["label"] == OA.PROGRESSIVE


def test_structure_progressive():
    r = _structure(lambda t: (0.1, 1.0, 1.0))
    assert (r["label"], r["field_order"], r["pulldown_phase"]) == (OA.PROGRESSIVE, OA.FO_NONE, -1)


def _cadence(phase):
    """Same-parity ACT of a 3:2 cadence: the upper field repeats at (t - phase) mod 5 = 1,
    the lower at 3."""
    def rep(t):
        c = (t - phase) % 5
        return (0.0, 1.0) if c == 1 else ((1.0, 0.0) if c == 3 else (1.0, 1.0))
    return rep


@pytest.mark.parametrize("phase", [0, 1, 4])
def test_structure_pulldown_phase(phase):
    r = _structure(lambda t: (1.0, 1.0, 1.0), rep=_cadence(phase))
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, phase)
    # a repeated field among the first five voters: every voter reads both same-parity pairs
    same = sorted(a for (k, a, b) in r["measures"] if k == UPPER_UPPER)
    assert same == list(range(20))


def test_same_parity_pairs_only_for_the_probe_without_a_repeat():
    r = _structure(lambda t: (1.0, 3.0, 1.0))
    assert sorted(a for (k, a, b) in r["measures"] if k in (UPPER_UPPER, LOWER_LOWER)) == [0, 0, 1, 1, 2, 2, 3, 3, 4, 4]


# ---- 3:2 pulldown shots ----------------------------------------------------------------

def _telecined(T, cut, flash=None):
    """Phase-0 cadence: a_t = 3 at positions 1 and 3 (clean to combed and combed
    to clean frames), 1 elsewhere; a_{cut-1} = 3 across the boundary, other frame
    pairs 2 inside a shot and 10 across; an optional flash frame f raises
    a_{f-1} and a_f to 9.  Same-parity pairs repeat in the 3:2 pattern."""
    def act(kind, a, b):
        if kind == FRAME:
            if b == a + 1:
                if flash is not None and a in (flash - 1, flash):
                    return 9.0
                if a == cut - 1:
                    return 3.0
                return 3.0 if a % 5 in (1, 3) else 1.0
            return 10.0 if (a < cut) != (b < cut) else 2.0
        if kind in (UPPER_UPPER, LOWER_LOWER):
            return _cadence(0)(a)[0 if kind == UPPER_UPPER else 1]
        return 1.0

    def amm(kind, a, b):
        return 1.0
    return Scripted(T, act, samm=lambda a, b: STATIC, amm=amm)


def test_pulldown_shot_cut_at_a_clean_step():
    # 20 voters (frames 0..19) make the first shot pulldown, phase 0, from frame 20 on.
    # The cadence peaks at positions 1, 3 are not tested there; t = 39 (position 4):
    # a_39 = 3 > 1.4 * median(a_34, a_29, a_24) = 1.4, and 3 > 1.4 * a_34,
    # a_40 = 1 <= 2.5 * a_35, a_38 = 3 <= 1.4 * a_33 = 4.2: a hardcut at 40
    o = _telecined(60, 40)
    r = o.run()
    assert r["cuts"] == [40] and r["dissolves"] == []
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, 0)
    # no deep-check pair is read between the verdict (frame 20) and the cut
    assert [p for p in requested(o) if 20 <= p[0] <= 39] == []


def test_pulldown_flash_is_no_cut():
    # a flash at 29 (position 4): a_29 = 9 passes the step test against a_24 = 1, but
    # a_28 = 9 > 1.4 * a_23 = 4.2: frame 29 is no ordinary frame of the shot
    r = _telecined(40, 1000, flash=29).run()
    assert r["cuts"] == [] and r["dissolves"] == []
