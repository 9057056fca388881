"""The oracle's decisions against the events the generator planted (Sec. III.B-C
read on synthetic video): the interlaced and 3:2 pulldown workloads at reduced
size (640x360, 600 frames, the same events, motion and noise per pixel as the
full-size clips) and a 640x360 version of the batched workload.  These pin the
decision readings themselves, not only their agreement with the library."""
import os

import pytest

from oracle import analyser as OA
from paper_2502_09202_gb300 import synth

WORKERS = min(8, os.cpu_count() or 1)
STRUCT = {"progressive": (OA.PROGRESSIVE, OA.FO_NONE), "tff": (OA.INTERLACED, OA.FO_TFF),
          "bff": (OA.INTERLACED, OA.FO_BFF), "pulldown": (OA.PULLDOWN, OA.FO_NONE)}


def _events(r):
    return r["cuts"], [tuple(d) for d in r["dissolves"]]


def test_reduced_interlaced_workload_recovers_its_events():
    spec = synth.config_interlaced(nframes=600, width=640, height=360)
    truth = synth.Clip(spec).truth()
    r = OA.analyse_spec(spec, workers=WORKERS)
    # two 8-frame dissolves (K = 7), flashes at frames not reported as events
    assert _events(r) == (truth["cuts"], [tuple(d) for d in truth["dissolves"]])
    assert truth["dissolves"] and all(k == 7 for _, k in truth["dissolves"])
    assert (r["label"], r["field_order"]) == STRUCT["tff"]
    assert all(s["label"] == OA.INTERLACED and s["field_order"] == OA.FO_TFF for s in r["shots"])


def test_reduced_pulldown_workload_recovers_its_cuts_and_phase():
    spec = synth.config_pulldown(nframes=600, width=640, height=360)
    truth = synth.Clip(spec).truth()
    r = OA.analyse_spec(spec, workers=WORKERS)
    assert len(truth["cuts"]) == 4
    assert _events(r) == (truth["cuts"], [])
    assert (r["label"], r["pulldown_phase"]) == (OA.PULLDOWN, truth["pulldown_phase"])
    assert all(s["label"] == OA.PULLDOWN and s["phase"] == truth["pulldown_phase"] for s in r["shots"])


def test_reduced_batched_workload():
    """Twelve 640x360 clips of 90-160 frames drawn as in the batched workload.
    Every cut and dissolve of the progressive and interlaced clips is found and
    nothing else; pulldown clips get their cuts, structure and phase, while a
    dissolve inside 3:2 pulldown content is not detected (a stated limit of the
    readings); at most one clip may carry the wrong structure (slow interlaced
    content whose fields barely move apart reads as progressive)."""
    specs = synth.config_batched(nclips=12, length_range=(90, 160), resolutions=((640, 360),))
    wrong_structure = 0
    structures = set()
    for spec in specs:
        truth = synth.Clip(spec).truth()
        r = OA.analyse_spec(spec, workers=WORKERS)
        structures.add(truth["structure"])
        cuts, dis = _events(r)
        assert cuts == truth["cuts"], spec.name
        if truth["structure"] == "pulldown":
            assert dis == [], spec.name
            assert r["pulldown_phase"] == truth["pulldown_phase"], spec.name
        else:
            assert dis == [tuple(d) for d in truth["dissolves"]], spec.name
        wrong_structure += (r["label"], r["field_order"]) != STRUCT[truth["structure"]]
    assert structures == set(STRUCT)
    assert wrong_structure <= 1
