"""Host-side checks that need no GPU: the C ABI loads and exports what the header
declares, argument validation, and the library's own detectors (C++) driven by
oracle measures reproduce the oracle's decisions and FP64 values exactly; on
scripted records they also reach the decisions derived by hand from the rules."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import analyser as OA
from oracle import measures as OM
from paper_2502_09202_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "analyser.h")


@pytest.fixture(scope="module")
def native():
    from paper_2502_09202_gb300 import build
    build.build()
    from paper_2502_09202_gb300 import native as N
    return N


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long long)\s+\(?\*?\s*([a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_symbol(native):
    names = _declared_functions()
    assert len(names) >= 18, names
    for n in names:
        assert hasattr(native.lib, n), n
    assert set(names) == set(native.SIGNATURES), set(names) ^ set(native.SIGNATURES)


def test_struct_layouts_match_the_header(native, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "analyser.h"\nint main(){printf("%zu %zu %zu %zu",'
                   'sizeof(analyser_params),sizeof(analyser_measure),sizeof(analyser_shot),'
                   'sizeof(analyser_results_t));}\n')
    exe = tmp_path / "sz"
    import subprocess
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(native.Params), ctypes.sizeof(native.Measure),
                                     ctypes.sizeof(native.Shot), ctypes.sizeof(native.Results)]


def test_defaults_and_validation_without_a_gpu(native):
    p = native.default_params()
    assert (p.block, p.levels, p.radius_coarse, p.radius_refine, p.mv_cost, p.kmax) == (16, 3, 16, 2, 4, 8)
    h = ctypes.c_void_p()
    bad = [(63, 180), (320, 63), (320, 181), (5000, 4000)]
    for w, hh in bad:
        assert native.lib.analyser_create(w, hh, 25.0, ctypes.byref(p), ctypes.byref(h)) == native.ERR_INVALID_ARG
    q = native.default_params(levels=4)
    assert native.lib.analyser_create(320, 180, 25.0, ctypes.byref(q), ctypes.byref(h)) == native.ERR_INVALID_ARG
    q = native.default_params(radius_coarse=12)
    assert native.lib.analyser_create(320, 180, 25.0, ctypes.byref(q), ctypes.byref(h)) == native.ERR_INVALID_ARG
    q = native.default_params(tile_x=3, tile_y=3)
    assert native.lib.analyser_create(320, 180, 25.0, ctypes.byref(q), ctypes.byref(h)) == native.ERR_INVALID_ARG
    assert native.lib.analyser_create(320, 180, 0.0, ctypes.byref(p), ctypes.byref(h)) == native.ERR_INVALID_ARG
    assert native.lib.analyser_push_frames(None, None, 320, 1) == native.ERR_INVALID_ARG
    assert native.lib.analyser_finish(None) == native.ERR_INVALID_ARG
    native.lib.analyser_destroy(None)


def test_budget_below_need_is_refused_before_device_work(native):
    # the 1080p window of 96 frames needs ~330 MB: a 1 MB budget is refused with
    # ANALYSER_ERR_OOM from the sizes alone (no GPU here), an unset one is not
    # refused for that reason
    h = ctypes.c_void_p()
    p = native.default_params(mem_budget_bytes=1 << 20)
    assert native.lib.analyser_create(1920, 1080, 25.0, ctypes.byref(p), ctypes.byref(h)) == native.ERR_OOM
    assert not h.value
    p = native.default_params(wait_timeout_ms=-1.0)
    assert native.lib.analyser_create(1920, 1080, 25.0, ctypes.byref(p), ctypes.byref(h)) == native.ERR_INVALID_ARG
    p = native.default_params(window_frames=25)      # below 2*kmax + steady_span + steady_frames + 4
    assert native.lib.analyser_create(320, 180, 25.0, ctypes.byref(p), ctypes.byref(h)) == native.ERR_INVALID_ARG


def test_offline_handle_refuses_frames(native):
    from paper_2502_09202_gb300 import api
    frames = synth.Clip(synth.config_small()).frames(0, 6)
    o = OA.OracleAnalyser(lambda t: frames[t], 6)
    o.run()

    def get(kind, a, b):
        m = o.m(kind, a, b)
        return [m[k] for k in OM.REC_FIELDS]

    h = ctypes.c_void_p()
    p = native.default_params()
    fn = native.MEASURE_FN(lambda ctx, kind, a, b, rec: [rec.__setitem__(i, v) for i, v in enumerate(get(kind, a, b))]
                           and 0)
    assert native.lib.analyser_detect_offline(ctypes.byref(p), 320, 180, 6, fn, None, ctypes.byref(h)) == native.OK
    buf = np.zeros((180, 320), np.uint8)
    assert native.lib.analyser_push_frames(h, buf.ctypes.data, 320, 1) == native.ERR_STATE
    r = native.Results()
    assert native.lib.analyser_results(h, ctypes.byref(r)) == native.OK     # a refused push is not sticky here
    native.lib.analyser_destroy(h)


def _offline(frames, params=OA.Params(), **overrides):
    from paper_2502_09202_gb300 import api
    o = OA.OracleAnalyser(lambda t: frames[t], len(frames), params)
    ref = o.run()

    def get(kind, a, b):
        m = o.m(kind, a, b)
        return [m[k] for k in OM.REC_FIELDS]

    got = api.detect_offline(frames.shape[2], frames.shape[1], len(frames), get, **overrides)
    return got, ref


def _same(got, ref):
    for k in ("cuts", "dissolves", "keyframes", "shots", "label", "field_order", "pulldown_phase"):
        assert got[k] == ref[k], (k, got[k], ref[k])
    assert set(got["measures"]) == set(ref["measures"])
    for key, m in ref["measures"].items():
        for f, v in m.items():
            assert got["measures"][key][f] == v, (key, f)


def test_library_detectors_equal_oracle_on_small_clip(native):
    got, ref = _offline(synth.Clip(synth.config_small()).frames())
    _same(got, ref)
    assert ref["cuts"] == [20, 41] and ref["dissolves"] == [(50, 4)]


@pytest.mark.parametrize("maker", [
    lambda: synth.config_interlaced(nframes=120, width=320, height=180),
    lambda: synth.config_pulldown(nframes=100, width=320, height=180),
    lambda: synth.config_batched(nclips=1, length_range=(90, 90), resolutions=((256, 144),))[0],
])
@pytest.mark.parametrize("prefetch", [0, 64])
def test_library_detectors_equal_oracle_on_reduced_configs(native, maker, prefetch):
    """With prefetch the speculative copy asks for more pairs; neither a
    decision nor the reported measure set may change."""
    got, ref = _offline(synth.Clip(maker()).frames(), prefetch_frames=prefetch)
    _same(got, ref)


def test_offline_callback_errors_surface(native):
    from paper_2502_09202_gb300 import api

    def bad(kind, a, b):
        raise ValueError("no such pair")

    with pytest.raises(ValueError):
        api.detect_offline(320, 180, 5, bad)


# ---- the library's detectors on scripted records ---------------------------------
# A record with S_i = S_j = S_ij = 0 and S_ii = S_jj = 1 has C = 0 and Vi, Vj > 0,
# so NCC = 0 and SWR = 1, and S_amm = ACT^2 * 65536 * nb makes ACT = sqrt(AMM) the
# scripted value (and AMM = ACT^2, the motion part the structure rules read).  The
# expected decisions are derived by hand from the rules (Sec. III.B-D), as in the
# oracle's detector pins; the oracle run on the same records must agree on
# everything, the reported measure set included.

def _scripted_record(act, kind, a, b):
    n, nb = (64 * 64, 16) if kind == OM.FRAME else (64 * 32, 8)
    return [0, 0, 1, 1, 0, 0, int(round(act * act * 65536 * nb)), n, nb]


def _both(T, act):
    """Library and oracle decisions for a 64x64 clip of T frames whose pair
    (kind, a, b) has ACT = act(kind, a, b)."""
    from paper_2502_09202_gb300 import api

    def get(kind, a, b):
        return _scripted_record(act(kind, a, b), kind, a, b)

    got = api.detect_offline(64, 64, T, get)

    class Records(OA.OracleAnalyser):
        def _measure(self, kind, a, b):
            return OM.finalise(dict(zip(OM.REC_FIELDS, get(kind, a, b))))

    ref = Records(lambda t: np.zeros((64, 64), np.uint8), T).run()
    _same(got, ref)
    return got


def _positions(p, g=0.0, field_act=1.0):
    def act(kind, a, b):
        return 1.0 + g * abs(a - b) + 9.0 * abs(p(a) - p(b)) if kind == OM.FRAME else field_act
    return act


def _requested(r):
    return sorted((a, b) for (k, a, b) in r["measures"] if k == OM.FRAME and b != a + 1)


def test_library_hard_cut_on_scripted_records(native):
    r = _both(12, _positions(lambda f: 0.0 if f <= 6 else 1.0))
    assert r["cuts"] == [7] and r["dissolves"] == []
    assert r["keyframes"] == [0, 7]
    assert _requested(r) == [(6, 4), (6, 5), (6, 8)]


def test_library_dissolve_on_scripted_records(native):
    p = {11: 1 / 3, 12: 2 / 3}
    r = _both(20, _positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.0)))
    assert r["dissolves"] == [(10, 3)] and r["cuts"] == []
    assert r["keyframes"] == [0, 9, 13]
    assert _requested(r) == [(10, 7), (10, 8), (10, 9), (10, 12), (10, 13), (10, 14)]


def test_library_completion_and_steadiness_on_scripted_records(native):
    # frame 12 farther from 10 than frame 11: K = 1 incomplete, dissolve (10, 3)
    p = {11: 0.5, 12: 0.66}
    assert _both(20, _positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.0)))["dissolves"] == [(10, 3)]
    # the new shot still moves at 12: K = 2 not steady, dissolve (10, 3)
    p = {11: 0.5, 12: 1.0}
    assert _both(24, _positions(lambda f: 0.0 if f <= 10 else p.get(f, 1.1)))["dissolves"] == [(10, 3)]


def test_library_ramp_start_on_scripted_records(native):
    steps = {11: 0.1, 12: 0.35, 13: 0.65}
    r = _both(20, _positions(lambda f: 0.0 if f <= 10 else steps.get(f, 1.0)))
    assert r["dissolves"] == [(10, 4)] and r["cuts"] == []
    assert _requested(r) == [(10, 6), (10, 8), (10, 9), (10, 12), (10, 13), (10, 14), (10, 15)]


def test_library_lag_and_blend_tests_on_scripted_records(native):
    # a flash at 11 in a shot whose ACT grows by 0.45 per frame of distance: K = 8 passes
    # (a)-(c) but ACT(10,18) = 4.6 is not above 1.5 * ACT(10,2) = 6.9
    r = _both(30, _positions(lambda f: 1.0 if f == 11 else 0.0, g=0.45))
    assert r["cuts"] == [] and r["dissolves"] == [] and (OM.FRAME, 10, 2) in r["measures"]
    # an abrupt change at 16 after frames of growing distance: a hardcut, no dissolve
    r = _both(30, _positions(lambda f: 0.0 if f <= 15 else 1.0, g=0.3))
    assert r["cuts"] == [16] and r["dissolves"] == []


def test_library_keyframes_on_scripted_records(native):
    assert _both(12, lambda k, a, b: 3.0)["keyframes"] == [0, 3, 6, 9]


@pytest.mark.parametrize("v,label,fo", [
    ((1.0, 3.0, 1.0), OA.INTERLACED, OA.FO_TFF),
    ((1.0, 1.0, 3.0), OA.INTERLACED, OA.FO_BFF),
    ((1.0, 1.0, 1.0), OA.PROGRESSIVE, OA.FO_NONE),
    ((0.55, 1.4, 1.0), OA.PROGRESSIVE, OA.FO_NONE),
    ((0.1, 1.0, 1.0), OA.PROGRESSIVE, OA.FO_NONE),
])
def test_library_structure_on_scripted_records(native, v, label, fo):
    # field ACT v -> AMM v^2 (SWR = 1): (1, 9, 1) combed and B = 9: TFF; (1, 1, 9): BFF;
    # (1, 1, 1) combed but B = 1; (0.3025, 1.96, 1): B = 1.96 but A0 < 0.65 * 1; (0.01, 1, 1)
    def act(kind, a, b):
        if kind == OM.FRAME:
            return 1.0                      # AMM = 1 px: not static
        if kind == OM.UPPER_LOWER:
            return v[0] if a == b else v[1]
        if kind == OM.LOWER_UPPER:
            return v[2]
        return 1.0                          # same-parity pairs: no repeated field
    r = _both(30, act)
    assert (r["label"], r["field_order"]) == (label, fo)


@pytest.mark.parametrize("phase", [0, 2, 3])
def test_library_pulldown_phase_on_scripted_records(native, phase):
    def act(kind, a, b):
        c = (a - phase) % 5
        if kind == OM.UPPER_UPPER:
            return 0.0 if c == 1 else 1.0
        if kind == OM.LOWER_LOWER:
            return 0.0 if c == 3 else 1.0
        return 1.0
    r = _both(30, act)
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, phase)


def test_library_pulldown_shot_cut_on_scripted_records(native):
    # phase-0 cadence (peaks of 3 at positions 1 and 3), voters 0..19, a cut at 40
    # (a_39 = 3 against a_34 = 1) and a flash at 29 that the old-shot test rejects
    def act(kind, a, b):
        if kind == OM.FRAME:
            if b == a + 1:
                if a in (28, 29):
                    return 9.0
                if a == 39:
                    return 3.0
                return 3.0 if a % 5 in (1, 3) else 1.0
            return 10.0 if (a < 40) != (b < 40) else 2.0
        if kind == OM.UPPER_UPPER:
            return 0.0 if a % 5 == 1 else 1.0
        if kind == OM.LOWER_LOWER:
            return 0.0 if a % 5 == 3 else 1.0
        return 1.0
    r = _both(60, act)
    assert r["cuts"] == [40] and r["dissolves"] == []
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, 0)
    assert [p for p in _requested(r) if 20 <= p[0] <= 39] == []


def test_missing_library_fails_loudly(tmp_path):
    """Without the compiled library the package refuses to import: there is no
    CPU fallback behind the API."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_2502_09202_gb300")
    dst = tmp_path / "paper_2502_09202_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", "csrc"))
    for mod in ("native", "api"):
        p = subprocess.run([sys.executable, "-c", f"import paper_2502_09202_gb300.{mod}"], cwd=tmp_path,
                           capture_output=True, text=True, env={**os.environ, "PYTHONPATH": str(tmp_path)})
        assert p.returncode != 0 and "ImportError" in p.stderr and "libgb300va.so is missing" in p.stderr, p.stderr
