"""The two full-size single-clip workloads (1920x1080 interlaced, 1500 frames;
1920x1080 3:2 pulldown, 1800 frames) through the library on the GPU, frames
resident in device memory as in the benchmark, compared value by value with
the oracle's analysis stored by tests/golden/make_full_size_oracle.py: every
decision, the reported measure set and every integer and FP64 value of it.
The decisions must also be the generator's planted events."""
import gzip
import json
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from paper_2502_09202_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SPECS = {"interlaced_1080p": synth.config_interlaced, "pulldown_1080p": synth.config_pulldown}


def _chunk(args):
    spec, s, e = args
    return synth.Clip(spec).frames(s, e)


_FRAMES = {}


def _frames(spec):
    if spec.name in _FRAMES:
        return _FRAMES[spec.name]
    _FRAMES.clear()
    out = np.empty((spec.nframes, spec.height, spec.width), np.uint8)
    jobs = [(spec, s, min(s + 50, spec.nframes)) for s in range(0, spec.nframes, 50)]
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        for (_, s, e), arr in zip(jobs, ex.map(_chunk, jobs)):
            out[s:e] = arr
    _FRAMES[spec.name] = out
    return out


@pytest.mark.parametrize("name", sorted(SPECS))
@pytest.mark.parametrize("prefetch", [0, 256])
def test_full_size_workload_equals_the_stored_oracle_run(name, prefetch):
    """prefetch > 0: the speculative pair requests change the waves, not one
    decision or reported value."""
    from paper_2502_09202_gb300 import api
    with gzip.open(os.path.join(GOLDEN, f"oracle_{name}.json.gz"), "rt") as f:
        ref = json.load(f)
    spec = SPECS[name]()
    frames = _frames(spec)
    dev = torch.from_numpy(frames).cuda()
    with api.Analyser(spec.width, spec.height, spec.fps, window_frames=512, prefetch_frames=prefetch) as a:
        a.push_device(dev)
        a.finish()
        got = a.results()
    assert got["cuts"] == ref["cuts"]
    assert [list(d) for d in got["dissolves"]] == ref["dissolves"]
    for k in ("keyframes", "shots", "label", "field_order", "pulldown_phase"):
        assert got[k] == ref[k], k
    want = {(k, a, b): m for k, a, b, m in ref["measures"]}
    assert set(got["measures"]) == set(want)
    for key, m in want.items():
        g = got["measures"][key]
        for f, v in m.items():
            v = float.fromhex(v) if isinstance(v, str) else v
            assert g[f] == v, (key, f, g[f], v)
    truth = synth.Clip(spec).truth()
    assert got["cuts"] == truth["cuts"]
    assert [tuple(d) for d in got["dissolves"]] == [tuple(d) for d in truth["dissolves"]]
