"""The seeded input generator plants what the input recipe says (CPU): frames
are pure functions of (spec, t); interlaced frames take their two fields from
consecutive field times in field order; 3:2 pulldown follows the AA BB BC CD DD
cadence from its phase; a dissolve is the stated integer blend; a flash adds
80 and clips.  Noise is off here so every frame can be rebuilt from the scene
renderer."""
import dataclasses

import numpy as np
import pytest

from paper_2502_09202_gb300 import synth


def _spec(structure, **kw):
    base = dataclasses.replace(synth.config_small(), width=96, height=64, nframes=24, sigma=0.0,
                               structure=structure, cuts=[], dissolves=[], flashes=[])
    return dataclasses.replace(base, **kw)


def _render(spec, key, tau):
    scene = synth.make_scene(spec.seed, key, spec.width, spec.height, spec.style)
    return synth.render(scene, tau, spec.width, spec.height).astype(np.int32)


def test_frames_are_pure_functions_of_spec_and_time():
    spec = synth.config_small()
    a, b = synth.Clip(spec), synth.Clip(spec)
    for t in (0, 33, 63):
        assert np.array_equal(a.frame(t), b.frame(t))
    assert np.array_equal(a.frames(10, 14), np.stack([b.frame(t) for t in range(10, 14)]))


@pytest.mark.parametrize("structure", [synth.TFF, synth.BFF])
def test_interlaced_fields_come_from_consecutive_field_times(structure):
    spec = _spec(structure)
    clip = synth.Clip(spec)
    for t in (0, 5, 11):
        f = clip.frame(t).astype(np.int32)
        first, second = _render(spec, 0, 2 * t), _render(spec, 0, 2 * t + 1)
        top, bottom = (first, second) if structure == synth.TFF else (second, first)
        assert np.array_equal(f[0::2], top[0::2]) and np.array_equal(f[1::2], bottom[1::2])


@pytest.mark.parametrize("phase", [0, 3])
def test_pulldown_cadence(phase):
    # video frame (t - phase) mod 5 = 0..4 shows film frames AA BB BC CD DD of its 4-frame group
    spec = _spec(synth.PULLDOWN, pulldown_phase=phase)
    clip = synth.Clip(spec)
    fields = {0: (0, 0), 1: (1, 1), 2: (1, 2), 3: (2, 3), 4: (3, 3)}
    for t in range(phase, phase + 10):
        c, u = (t - phase) % 5, (t - phase) // 5
        top, bottom = (4 * u + k for k in fields[c])
        f = clip.frame(t).astype(np.int32)
        assert np.array_equal(f[0::2], _render(spec, 0, top)[0::2])
        assert np.array_equal(f[1::2], _render(spec, 0, bottom)[1::2])
        assert (top != bottom) == (c in (2, 3))       # only the two mixed frames comb


def test_dissolve_is_the_stated_integer_blend_and_cut_switches_scene():
    L, s = 5, 8
    spec = _spec(synth.PROGRESSIVE, dissolves=[(s, L)], cuts=[16])
    clip = synth.Clip(spec)
    for t in range(s, s + L):
        i = t - s
        a, b = _render(spec, 0, t), _render(spec, 1, t)
        want = (a * (L - 1 - i) + b * i + (L - 1) // 2) // (L - 1)
        assert np.array_equal(clip.frame(t).astype(np.int32), want), t
    assert np.array_equal(clip.frame(15).astype(np.int32), _render(spec, 1, 15))
    assert np.array_equal(clip.frame(16).astype(np.int32), _render(spec, 2, 16))
    assert clip.truth()["dissolves"] == [(s, L - 1)] and clip.truth()["cuts"] == [16]


def test_flash_adds_eighty_and_clips():
    spec = _spec(synth.PROGRESSIVE, flashes=[7])
    clip = synth.Clip(spec)
    assert np.array_equal(clip.frame(7).astype(np.int32), np.clip(_render(spec, 0, 7) + 80, 0, 255))
    assert np.array_equal(clip.frame(6).astype(np.int32), _render(spec, 0, 6))
