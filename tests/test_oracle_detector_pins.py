"""Pins for the oracle's detectors (Sec. III.B-D) on scripted measures.

The detectors read pair measures only through ``OracleAnalyser.m``; here a
subclass serves hand-made ACT and S_amm values instead of computing them from
frames, and each expected outcome below is derived by hand from the rules as
the paper states them (fast check, deep check, keyframe accumulation, sampling
structure), not by running the oracle.  A dropped condition, a wrong index
(t - j for t + j, K for K + 1) or a swapped field pair changes an outcome.
"""
import math

import numpy as np
import pytest

from oracle import analyser as OA
from oracle.measures import FRAME, LOWER_UPPER, UPPER_LOWER

W = H = 32                                   # 4 blocks of 16 x 16
STATIC = math.ceil(0.5 * 65536 * 4)          # S_amm threshold for "not static"


class Scripted(OA.OracleAnalyser):
    def __init__(self, T, act, samm=None, params=OA.Params()):
        super().__init__(lambda t: np.zeros((H, W), np.uint8), T, params)
        self._act = act
        self._samm = samm or (lambda a, b: 0)

    def m(self, kind, a, b):
        key = (kind, a, b)
        r = self.cache.get(key)
        if r is None:
            r = {"act": float(self._act(kind, a, b)), "samm": int(self._samm(a, b)) if kind == FRAME else 0}
            self.cache[key] = r
        return r


def positions(p):
    """ACT between frames a != b of one kind = 1 + 9 |p(a) - p(b)|, i.e. 1.0
    inside a shot and 10.0 across a hard change."""
    def act(kind, a, b):
        return 1.0 + 9.0 * abs(p(a) - p(b))
    return act


def requested(o):
    """Frame pairs other than the always-on (t, t+1) the detectors asked for."""
    return sorted((a, b) for (k, a, b) in o.cache if k == FRAME and b != a + 1)


def test_hard_cut():
    # a_6 = 10 against a median of 1: candidate; K = 1 passes: p = max(ACT(6,5),
    # ACT(6,4)) = 1 and 2*1 + 0.5 < ACT(6,7) = ACT(6,8) = 10, 2*ACT(7,8) + 0.5 < 10
    o = Scripted(12, positions(lambda f: 0.0 if f <= 6 else 1.0))
    r = o.run()
    assert r["cuts"] == [7] and r["dissolves"] == []
    assert [(s["first"], s["last"]) for s in r["shots"]] == [(0, 6), (7, 11)]
    assert r["keyframes"] == [0, 7]
    assert requested(o) == [(6, 4), (6, 5), (6, 8)]
    assert r["label"] == OA.UNKNOWN            # every pair static: nothing analysed


def test_dissolve_needs_the_after_condition():
    # positions 0 | 1/3, 2/3 | 1: K = 1 and K = 2 fail only on a_{t+K} << ACT(t, t+K)
    # (2*4 + 0.5 = 8.5 is not below 4, resp. 7); K = 3 passes (2*1 + 0.5 < 10)
    p = {11: 1 / 3, 12: 2 / 3}
    o = Scripted(20, positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.0)))
    r = o.run()
    assert r["cuts"] == [] and r["dissolves"] == [(10, 3)]
    assert [(s["first"], s["last"]) for s in r["shots"]] == [(0, 10), (13, 19)]
    # S = a_0 + ... + a_8 = 9 > 8 makes frame 9 a keyframe; the six frames of
    # the second shot add 6
    assert r["keyframes"] == [0, 9, 13]
    assert requested(o) == [(10, 8), (10, 9), (10, 12), (10, 13), (10, 14)]


def test_ramp_start_is_a_candidate_below_the_jump_threshold():
    # a_10 = 1.5 < 2 * median (no jump) but > 1.3 * median and a_10 < a_11 < a_12:
    # a candidate; the deep check passes first at K = 4 (ACT(10,14) = 10, a_14 = 1)
    steps = {11: 0.5 / 9, 12: 1.3 / 9, 13: 2.4 / 9}
    o = Scripted(20, positions(lambda f: 0.0 if f <= 10 else steps.get(f, 1.0)))
    r = o.run()
    assert r["dissolves"] == [(10, 4)] and r["cuts"] == []
    assert r["keyframes"] == [0, 9, 14]


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


def _structure(v, T=30):
    """Clip whose every adjacent pair moves (S_amm at the threshold) and whose
    field measures are v(t) = (v0, v1, v2)."""
    def act(kind, a, b):
        if kind == FRAME:
            return 1.0
        v0, v1, v2 = v(a)
        if kind == UPPER_LOWER:
            return v0 if a == b else v1
        assert kind == LOWER_UPPER and b == a + 1
        return v2
    return Scripted(T, act, samm=lambda a, b: STATIC).run()


def test_structure_interlaced_upper_field_first():
    r = _structure(lambda t: (5.0, 6.0, 3.0))
    assert (r["label"], r["field_order"]) == (OA.INTERLACED, OA.FO_TFF)
    assert r["shots"][0]["analysed"] == 20          # N_s frames of the shot


def test_structure_interlaced_lower_field_first():
    r = _structure(lambda t: (5.0, 3.0, 6.0))
    assert (r["label"], r["field_order"]) == (OA.INTERLACED, OA.FO_BFF)


def test_structure_combed_but_balanced_fields_is_not_interlaced():
    # every frame combed, but B = 1 is inside (1/theta_b, theta_b)
    assert _structure(lambda t: (5.0, 3.0, 3.0))["label"] == OA.PROGRESSIVE


def test_structure_progressive():
    r = _structure(lambda t: (0.1, 1.0, 1.0))
    assert (r["label"], r["field_order"], r["pulldown_phase"]) == (OA.PROGRESSIVE, OA.FO_NONE, -1)


@pytest.mark.parametrize("phase", [0, 1, 4])
def test_structure_pulldown_phase(phase):
    # combed exactly on the two mixed frames of each 3:2 cycle, (t - phase) mod 5 in {2, 3}
    r = _structure(lambda t: (5.0 if (t - phase) % 5 in (2, 3) else 0.1, 1.0, 1.0))
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, phase)
