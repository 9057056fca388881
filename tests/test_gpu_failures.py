"""Failure handling on the GPU path, all of it made on the host (no kernel is
made to fault or hang): a push after finish, results before the end of a clip,
a sticky error refusing later calls, a device-memory budget below the need,
and the host watchdog on GPU waits (params.wait_timeout_ms), which gives up on
a real wave that cannot be done in the time allowed and returns
ANALYSER_ERR_TIMEOUT while the work completes normally on the GPU."""
import ctypes

import numpy as np
import pytest

from paper_2502_09202_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_push_after_finish_is_a_sticky_state_error():
    from paper_2502_09202_gb300 import native as N
    frames = synth.Clip(synth.config_small()).frames(0, 8)
    p = N.default_params()
    h = ctypes.c_void_p()
    assert N.lib.analyser_create(320, 180, 25.0, ctypes.byref(p), ctypes.byref(h)) == N.OK
    assert N.lib.analyser_push_frames(h, frames.ctypes.data, 320, 8) == N.OK
    assert N.lib.analyser_finish(h) == N.OK
    r = N.Results()
    assert N.lib.analyser_results(h, ctypes.byref(r)) == N.OK and r.nframes == 8
    assert N.lib.analyser_push_frames(h, frames.ctypes.data, 320, 1) == N.ERR_STATE
    msg = ctypes.c_char_p()
    assert N.lib.analyser_last_error(h, ctypes.byref(msg)) == N.ERR_STATE
    assert b"after analyser_finish" in msg.value
    # the handle now refuses further work with the same code
    assert N.lib.analyser_results(h, ctypes.byref(r)) == N.ERR_STATE
    assert N.lib.analyser_finish(h) == N.ERR_STATE
    N.lib.analyser_destroy(h)


def test_results_before_the_end_are_refused_without_failing_the_handle():
    from paper_2502_09202_gb300 import api
    frames = synth.Clip(synth.config_small()).frames(0, 12)
    with api.Analyser(320, 180, 25.0) as a:
        with pytest.raises(api.AnalyserError) as e:
            a.results()                       # before any frame
        assert e.value.code == -5
        a.push(frames)
        with pytest.raises(api.AnalyserError):
            a.results()                       # before analyser_finish
        a.finish()
        assert a.results()["nframes"] == 12


def test_budget_below_need_gives_oom():
    from paper_2502_09202_gb300 import api, native as N
    with pytest.raises(api.AnalyserError) as e:
        api.Analyser(1920, 1080, 25.0, mem_budget_bytes=64 << 20)
    assert e.value.code == N.ERR_OOM
    srv = api.Server(budget_bytes=64 << 20)
    with pytest.raises(api.AnalyserError) as e:
        srv.submit(np.zeros((4, 1080, 1920), np.uint8))
    assert e.value.code == N.ERR_OOM
    srv.close()


def test_watchdog_gives_up_on_a_wave_and_the_handle_stays_safe():
    from paper_2502_09202_gb300 import api, native as N
    spec = synth.config_interlaced(nframes=96)
    frames = torch.from_numpy(synth.Clip(spec).frames()).cuda()
    torch.cuda.synchronize()
    # a 1080p wave of 96 frames takes far longer than a microsecond: the first wait gives up
    a = api.Analyser(1920, 1080, 25.0, wait_timeout_ms=1e-3)
    with pytest.raises(api.AnalyserError) as e:
        a.push_device(frames)
        a.finish()
    assert e.value.code == N.ERR_TIMEOUT
    msg = ctypes.c_char_p()
    assert N.lib.analyser_last_error(a._h, ctypes.byref(msg)) == N.ERR_TIMEOUT
    a.close()                                 # waits for the queued work before its buffers go back
    torch.cuda.synchronize()
    # the same clip with a generous deadline completes
    with api.Analyser(1920, 1080, 25.0, wait_timeout_ms=60000.0) as b:
        b.push_device(frames)
        b.finish()
        assert b.results()["nframes"] == 96
