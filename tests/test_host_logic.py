"""Host-side checks that need no GPU: the C ABI loads and exports what the header
declares, argument validation, and the library's own detectors (C++) driven by
oracle measures reproduce the oracle's decisions and FP64 values exactly."""
import ctypes
import os
import re

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


def _offline(frames, params=OA.Params()):
    from paper_2502_09202_gb300 import api
    o = OA.OracleAnalyser(lambda t: frames[t], len(frames), params)
    ref = o.run()

    def get(kind, a, b):
        m = o.m(kind, a, b)
        return [m[k] for k in OM.REC_FIELDS]

    got = api.detect_offline(frames.shape[2], frames.shape[1], len(frames), get)
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
def test_library_detectors_equal_oracle_on_reduced_configs(native, maker):
    got, ref = _offline(synth.Clip(maker()).frames())
    _same(got, ref)


def test_offline_callback_errors_surface(native):
    from paper_2502_09202_gb300 import api

    def bad(kind, a, b):
        raise ValueError("no such pair")

    with pytest.raises(ValueError):
        api.detect_offline(320, 180, 5, bad)
