"""analyser_measure_pair_noalloc: the pair measure for callers that must not
allocate device memory while they run (a host application that reserves all
device memory up front).  Its record must equal analyser_measure_pairs' for
the same frames, call after call, although every call reuses one fixed
scratch array.  Collected last so that a failure here stops a -x run only
after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2502_09202_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(frames):
    n, h, w = frames.shape
    pitch = (w + 63) // 64 * 64
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(frames).cuda()
    torch.cuda.synchronize()
    return buf


def _noalloc(N, p, w, h, kind, buf, a, b):
    rec = (ctypes.c_int64 * 7)()
    pitch = buf.stride(1)
    code = N.lib.analyser_measure_pair_noalloc(ctypes.byref(p), w, h, kind, buf[a].data_ptr(), buf[b].data_ptr(),
                                               pitch, rec, None)
    assert code == N.OK, code
    return [rec[i] for i in range(7)]


def test_noalloc_matches_measure_pairs_on_consecutive_calls():
    from paper_2502_09202_gb300 import api, native as N
    spec = synth.config_interlaced(nframes=4, width=640, height=360)
    frames = synth.Clip(spec).frames()
    buf = _dev(frames)
    view = buf[:, :, :spec.width]
    p = N.default_params()
    calls = [(0, 0, 1), (1, 2, 3), (2, 1, 2), (0, 3, 0), (3, 1, 2), (4, 0, 3)]
    want, _ = api.measure_pairs(view, [c[0] for c in calls], [c[1] for c in calls], [c[2] for c in calls])
    # one warm call loads the kernels; after it, no call may take device memory:
    # neither CUDA's free bytes nor the library's resource cache may change
    _noalloc(N, p, spec.width, spec.height, 0, buf, 0, 1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    cached0 = N.lib.analyser_cached_bytes()
    # two calls in a row (and four more): each equals the allocating entry point, exactly
    got = [_noalloc(N, p, spec.width, spec.height, kind, buf, a, b) for kind, a, b in calls]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert N.lib.analyser_cached_bytes() == cached0
    for k, (kind, a, b) in enumerate(calls):
        assert got[k] == [int(x) for x in want[k]], (kind, a, b)


def test_noalloc_keeps_the_callers_device_and_checks_the_pitch():
    from paper_2502_09202_gb300 import native as N
    frames = synth.Clip(synth.config_small()).frames(0, 2)
    buf = _dev(frames)
    p = N.default_params()
    before = torch.cuda.current_device()
    _noalloc(N, p, 320, 180, 0, buf, 0, 1)
    assert torch.cuda.current_device() == before
    rec = (ctypes.c_int64 * 7)()
    # a pitch whose doubled field pitch would not fit the kernels' int descriptors is refused
    code = N.lib.analyser_measure_pair_noalloc(ctypes.byref(p), 320, 180, 1, buf[0].data_ptr(), buf[1].data_ptr(),
                                               1 << 30, rec, None)
    assert code == N.ERR_INVALID_ARG


def test_noalloc_repeat_and_size_limit():
    from paper_2502_09202_gb300 import api, native as N
    frames = synth.Clip(synth.config_small()).frames(10, 12)
    buf = _dev(frames)
    p = N.default_params()
    first = _noalloc(N, p, 320, 180, 0, buf, 0, 1)
    second = _noalloc(N, p, 320, 180, 0, buf, 0, 1)
    want, _ = api.measure_pairs(buf[:, :, :320], [0], [0], [1])
    assert first == second == [int(x) for x in want[0]]
    # a size whose pyramids exceed the fixed scratch is refused before any GPU work
    rec = (ctypes.c_int64 * 7)()
    code = N.lib.analyser_measure_pair_noalloc(ctypes.byref(p), 4096, 2880, 0, buf[0].data_ptr(), buf[1].data_ptr(),
                                               4096, rec, None)
    assert code == N.ERR_INVALID_ARG
