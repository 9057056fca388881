"""GPU path vs oracle, through the C ABI: bit-exact motion vectors, integer sums,
FP64 measures and decisions."""
import numpy as np
import pytest

from oracle import analyser as OA
from oracle import measures as OM
from paper_2502_09202_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REC7 = ("si", "sj", "sii", "sjj", "sij", "sabs", "samm")


def _api():
    from paper_2502_09202_gb300 import api
    return api


def _dev(frames: np.ndarray, pad: int = 0):
    """Device copy (n, h, w) with rows padded to a multiple of 64 + pad bytes."""
    n, h, w = frames.shape
    pitch = (w + 63) // 64 * 64 + pad
    buf = torch.zeros((n, h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :, :w] = torch.from_numpy(frames).cuda()
    return buf[:, :, :w]


def _oracle_pair(kind, fa, fb, sp=OM.SearchParams()):
    I, J = OM.pair_images(kind, fa, fb)
    return OM.pair_record(I, J, sp, want_vec=True)


@pytest.mark.parametrize("w,h", [(200, 136), (333, 190), (640, 360), (1100, 258)])
def test_measure_pairs_bit_exact_random_content(w, h):
    """Pairs of every kind on sizes that span several tiles and ragged tails."""
    api = _api()
    clip = synth.Clip(synth.ClipSpec(w, h, 6, 25.0, synth.TFF, 5, 3.0,
                                     synth.SceneStyle(n_objects=(4, 6), obj_speed=12, cell=8, bg_kind="textured")))
    frames = clip.frames()
    kinds = [0, 0, 1, 1, 2, 0, 0, 3, 4]
    ia = [0, 1, 2, 3, 4, 5, 0, 1, 2]
    ib = [1, 2, 2, 4, 5, 0, 5, 2, 3]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7], (k, list(rec[k]), ref)
        assert np.array_equal(mot[k], vec), k


@pytest.mark.parametrize("tile", [(8, 4), (4, 4), (8, 2), (16, 2), (4, 8)])
def test_every_tile_shape_gives_identical_results(tile):
    api = _api()
    frames = synth.Clip(synth.config_small()).frames(18, 23)
    ia, ib = [0, 1, 2, 3, 0], [1, 2, 3, 4, 4]
    rec, mot = api.measure_pairs(_dev(frames), [0, 0, 0, 0, 2], ia, ib, want_motion=True,
                                 tile_x=tile[0], tile_y=tile[1])
    for k in range(5):
        ref, vec = _oracle_pair(2 if k == 4 else 0, frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7]
        assert np.array_equal(mot[k], vec)


@pytest.mark.parametrize("sx,sy", [(0, 0), (12, -8), (-40, 28), (64, 0)])
def test_known_shift_and_identity(sx, sy):
    api = _api()
    I, J = synth.shifted_pair(31, 256, 192, sx, sy)
    frames = np.stack([I, J])
    rec, mot = api.measure_pairs(_dev(frames), [0, 0], [0, 0], [1, 0], want_motion=True)
    ref, vec = _oracle_pair(0, I, J)
    assert list(rec[0]) == [ref[f] for f in REC7]
    assert np.array_equal(mot[0], vec)
    assert (mot[1] == 0).all() and rec[1][5] == 0           # identical pair: zero field, zero residual


def test_degenerate_flat_frames_and_extremes():
    api = _api()
    flat0 = np.zeros((96, 128), np.uint8)
    flat255 = np.full((96, 128), 255, np.uint8)
    tex = synth.random_frame(8, 128, 96)
    frames = np.stack([flat0, flat255, tex])
    kinds, ia, ib = [0, 0, 0, 1, 2], [0, 0, 2, 1, 2], [1, 2, 0, 2, 0]
    rec, mot = api.measure_pairs(_dev(frames, pad=16), kinds, ia, ib, want_motion=True)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7]
        assert np.array_equal(mot[k], vec)


def _compare_results(got, ref):
    for k in ("cuts", "dissolves", "keyframes", "shots", "label", "field_order", "pulldown_phase"):
        assert got[k] == ref[k], (k, got[k], ref[k])
    assert set(got["measures"]) == set(ref["measures"])
    for key, m in ref["measures"].items():
        g = got["measures"][key]
        for f, v in m.items():
            # integer sums and decisions bit-exact; FP64 values formed by the same
            # IEEE operations on both sides: identical (bound stated: 1e-9)
            assert g[f] == v, (key, f, g[f], v)


def test_small_clip_end_to_end_host_push():
    api = _api()
    spec = synth.config_small()
    frames = synth.Clip(spec).frames()
    with api.Analyser(spec.width, spec.height, spec.fps) as a:
        a.push(frames[:10])
        a.push(frames[10:37])
        a.push(frames[37:])
        a.finish()
        got = a.results()
    _compare_results(got, OA.analyse_frames(frames))


def test_small_clip_device_push_and_small_window():
    api = _api()
    spec = synth.config_small()
    frames = synth.Clip(spec).frames()
    with api.Analyser(spec.width, spec.height, spec.fps, window_frames=26) as a:
        a.push_device(_dev(frames))
        a.finish()
        got = a.results()
    _compare_results(got, OA.analyse_frames(frames))


def test_motion_dump_matches_oracle():
    api = _api()
    spec = synth.config_small()
    frames = synth.Clip(spec).frames(0, 12)
    with api.Analyser(spec.width, spec.height, spec.fps, want_motion=1) as a:
        a.push(frames)
        a.finish()
        got = a.results()
    for t in range(11):
        _, vec = _oracle_pair(0, frames[t], frames[t + 1])
        assert np.array_equal(got["motion"][t], vec), t


def test_empty_and_tiny_clips():
    api = _api()
    for n in (0, 1, 2, 3):
        frames = synth.Clip(synth.config_small()).frames(0, n)
        with api.Analyser(320, 180, 25.0) as a:
            if n:
                a.push(frames)
            a.finish()
            got = a.results()
        ref = OA.analyse_frames(frames) if n else OA.OracleAnalyser(lambda t: None, 0).run()
        _compare_results(got, ref)


def test_reduced_interlaced_and_pulldown_clips():
    """Configs 2 and 3 at reduced size (same structure and motion) end to end."""
    api = _api()
    for spec in (synth.config_interlaced(nframes=180, width=640, height=360),
                 synth.config_pulldown(nframes=160, width=640, height=360)):
        frames = synth.Clip(spec).frames()
        with api.Analyser(spec.width, spec.height, spec.fps) as a:
            a.push(frames)
            a.finish()
            got = a.results()
        _compare_results(got, OA.analyse_frames(frames))


def test_server_results_identical_alone_and_in_the_mix():
    api = _api()
    specs = [synth.config_small(), synth.config_interlaced(nframes=40, width=256, height=144),
             synth.config_pulldown(nframes=36, width=384, height=216)]
    clips = [synth.Clip(s).frames() for s in specs]
    alone = []
    for s, f in zip(specs, clips):
        with api.Analyser(s.width, s.height, s.fps) as a:
            a.push(f)
            a.finish()
            alone.append(a.results())
    srv = api.Server(budget_bytes=8 << 30)
    tickets = [srv.submit(f, s.fps) for s, f in zip(specs, clips)]
    srv.drain()
    for t, ref in zip(tickets, alone):
        _compare_results(srv.poll(t), ref)
        assert srv.latency(t) >= 0.0
    srv.close()


def test_full_size_1080p_sampled_pairs():
    """At the benchmark's 1080p size and launch configuration: sampled pairs of
    every kind, compared value by value with the oracle."""
    api = _api()
    spec = synth.config_interlaced()
    clip = synth.Clip(spec)
    ts = [0, 1, 2, 211, 212, 219]
    frames = np.stack([clip.frame(t) for t in ts])
    kinds, ia, ib = [0, 0, 1, 1, 2, 0], [0, 1, 0, 0, 0, 3], [1, 2, 0, 1, 1, 5]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7]
        assert np.array_equal(mot[k], vec)


def test_long_clip_streams_through_a_small_window():
    """A clip several windows long, pushed in uneven chunks: the window must keep
    advancing and the results must not depend on the chunking."""
    api = _api()
    spec = synth.config_interlaced(nframes=260, width=256, height=144)
    frames = synth.Clip(spec).frames()
    ref = OA.analyse_frames(frames)
    for chunks in ((260,), (7, 100, 1, 152)):
        with api.Analyser(spec.width, spec.height, spec.fps, window_frames=26) as a:
            s = 0
            for c in chunks:
                a.push(frames[s:s + c])
                s += c
            a.finish()
            _compare_results(a.results(), ref)


def test_long_clip_device_pushes_any_window():
    """Device pushes of a clip several windows long, whole and in uneven chunks,
    through windows below and above the size at which new frames join waves that
    still carry deep checks: the decisions must not depend on how the waves were
    composed."""
    api = _api()
    spec = synth.config_interlaced(nframes=260, width=256, height=144)
    frames = synth.Clip(spec).frames()
    ref = OA.analyse_frames(frames)
    dev = _dev(frames)
    for window in (26, 64, 128, 300):
        for chunks in ((260,), (7, 100, 1, 152)):
            with api.Analyser(spec.width, spec.height, spec.fps, window_frames=window) as a:
                s = 0
                for c in chunks:
                    a.push_device(dev[s:s + c])
                    s += c
                a.finish()
                _compare_results(a.results(), ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_split_and_fused_kernels_match_the_oracle(mode):
    """kernel_mode 0 runs the coarse and refinement kernels on two streams,
    kernel_mode 1 the fused kernel: both must equal the oracle."""
    api = _api()
    w, h = 333, 190
    clip = synth.Clip(synth.ClipSpec(w, h, 5, 25.0, synth.BFF, 9, 3.0,
                                     synth.SceneStyle(n_objects=(4, 6), obj_speed=10, cell=8, bg_kind="textured")))
    frames = clip.frames()
    kinds, ia, ib = [0, 1, 2, 0, 0, 1, 3, 4], [0, 1, 2, 3, 4, 4, 0, 3], [1, 2, 3, 4, 0, 4, 1, 4]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True, kernel_mode=mode)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7]
        assert np.array_equal(mot[k], vec)
    spec = synth.config_small()
    frames = synth.Clip(spec).frames()
    with api.Analyser(spec.width, spec.height, spec.fps, kernel_mode=mode) as a:
        a.push(frames)
        a.finish()
        _compare_results(a.results(), OA.analyse_frames(frames))


def test_chunked_wave_matches_the_oracle():
    """A call of 300 pairs runs as 4 chunks: the coarse kernel of chunk c+1
    beside the refinement kernel of chunk c on the second stream.  Every
    pair's record and motion field equal the oracle's, at a ragged size, pairs
    of every kind."""
    api = _api()
    w, h = 333, 190
    clip = synth.Clip(synth.ClipSpec(w, h, 12, 25.0, synth.TFF, 9, 3.0,
                                     synth.SceneStyle(n_objects=(4, 6), obj_speed=10, cell=8, bg_kind="textured")))
    frames = clip.frames()
    rng = np.random.default_rng(7)
    n = 300
    kinds = [int(k) for k in rng.integers(0, 5, n)]
    ia = [int(a) for a in rng.integers(0, 12, n)]
    ib = [int(b) for b in rng.integers(0, 12, n)]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True)
    for k in range(n):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7], k
        assert np.array_equal(mot[k], vec), k


def test_cached_buffers_reused_across_clips_and_trimmed():
    """Analysers and stateless calls created one after another run on buffers the
    previous ones returned to the resource cache (not cleared): results stay
    exact, and trimming returns the cached device memory."""
    api = _api()
    spec = synth.config_small()
    frames = synth.Clip(spec).frames()
    ref = OA.analyse_frames(frames)
    other = synth.Clip(synth.ClipSpec(333, 190, 5, 25.0, synth.TFF, 3, 3.0,
                                      synth.SceneStyle(n_objects=(4, 6), obj_speed=10, cell=8, bg_kind="textured")))
    of = other.frames()
    for rep in range(3):
        with api.Analyser(spec.width, spec.height, spec.fps) as a:
            a.push_device(_dev(frames))
            a.finish()
            _compare_results(a.results(), ref)
        rec, _ = api.measure_pairs(_dev(of), [0, 1], [0, 2], [1, 3])
        for k, (kind, i, j) in enumerate([(0, 0, 1), (1, 2, 3)]):
            r, _ = _oracle_pair(kind, of[i], of[j])
            assert list(rec[k]) == [r[f] for f in REC7], rep
    assert api.N.lib.analyser_cached_bytes() > 0
    assert api.trim_cache() > 0
    assert api.N.lib.analyser_cached_bytes() == 0


def test_frame_histograms_match_the_oracle():
    """Per-frame histogram measure (want_histogram): bins, mean, std, median and
    MAD of every frame equal the oracle's exactly; off by default."""
    api = _api()
    spec = synth.config_small()
    frames = synth.Clip(spec).frames()
    with api.Analyser(spec.width, spec.height, spec.fps, want_histogram=1, window_frames=26) as a:
        a.push(frames)
        a.finish()
        got = a.results()
    assert len(got["histograms"]) == len(frames)
    for t, h in enumerate(got["histograms"]):
        ref = OM.frame_histogram(frames[t])
        assert h["frame"] == t
        assert np.array_equal(h["bins"], ref["bins"]), t
        assert (h["mean"], h["std"], h["median"], h["mad"]) == (ref["mean"], ref["std"], ref["median"], ref["mad"]), t
    with api.Analyser(spec.width, spec.height, spec.fps) as a:
        a.push(frames[:8])
        a.finish()
        assert "histograms" not in a.results()


def test_largest_accepted_frame_size():
    """4096x2880 (11.8 M pixels, the largest the library accepts) with a ragged
    block grid in neither dimension; one frame pair and one field pair, value by
    value against the oracle, and one pixel more is refused."""
    api = _api()
    w, h = 4096, 2880
    spec = synth.ClipSpec(w, h, 3, 25.0, synth.TFF, 21, 3.0,
                          synth.SceneStyle(n_objects=(6, 8), obj_speed=14, cell=8, bg_kind="textured"))
    frames = synth.Clip(spec).frames()
    kinds, ia, ib = [0, 1], [0, 1], [1, 2]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]])
        assert list(rec[k]) == [ref[f] for f in REC7]
        assert np.array_equal(mot[k], vec)
    with pytest.raises(api.AnalyserError):
        api.Analyser(w + 2, h, 25.0)


@pytest.mark.parametrize("levels", [2, 3])
@pytest.mark.parametrize("radius", [8, 16, 24])
@pytest.mark.parametrize("refine", [0, 1, 2, 4])
@pytest.mark.parametrize("lam", [0, 4, 64])
def test_every_accepted_search_parameter_matches_the_oracle(levels, radius, refine, lam):
    """Every estimator parameter the C ABI accepts (levels 2-3, coarse radius
    8/16/24, refinement radius 0-4, motion cost 0-64), on pairs of every kind at a
    ragged size: records and motion fields element by element against the oracle.
    Radius 2 with 3 levels runs the split coarse/refinement kernels, everything
    else the fused kernel's general refinement."""
    api = _api()
    w, h = 232, 152
    spec = synth.config_interlaced(nframes=4, width=w, height=h)
    frames = synth.Clip(spec).frames()
    sp = OM.SearchParams(levels=levels, block=4 << (levels - 1), radius=radius, refine=refine, mv_cost=lam)
    kinds, ia, ib = [0, 1, 2, 3, 4, 0], [0, 1, 1, 2, 3, 3], [1, 1, 2, 3, 3, 0]
    rec, mot = api.measure_pairs(_dev(frames), kinds, ia, ib, want_motion=True, levels=levels,
                                 block=4 << (levels - 1), radius_coarse=radius, radius_refine=refine, mv_cost=lam)
    for k in range(len(kinds)):
        ref, vec = _oracle_pair(kinds[k], frames[ia[k]], frames[ib[k]], sp)
        assert list(rec[k]) == [ref[f] for f in REC7], (k, kinds[k])
        assert np.array_equal(mot[k], vec), (k, kinds[k])


def test_served_requests_match_the_oracle():
    """Requests drawn as in the served workload (Poisson arrivals, mixed
    structures, lengths 30-300, here at the two smallest sizes), submitted while
    others run and admitted under a budget that holds only some at a time: every
    result equals the oracle's analysis of the same clip, value by value."""
    api = _api()
    reqs = synth.config_served(nrequests=5, length_range=(30, 120), resolutions=((320, 180), (640, 360)))
    clips = [synth.Clip(s).frames() for _, s in reqs]
    srv = api.Server(budget_bytes=48 << 20)      # one 640x360 window (36 MB) at a time
    tickets = []
    for (_, s), f in zip(reqs, clips):
        tickets.append(srv.submit(f, s.fps))
        srv.step()
    srv.drain()
    for t, f in zip(tickets, clips):
        _compare_results(srv.poll(t), OA.analyse_frames(f))
    srv.close()


def test_batched_clips_match_the_oracle():
    """Three clips drawn as in the batched workload (mixed structures and
    lengths, two sizes) analysed together by one server (one tile shape for
    all, one coarse and one refinement launch per wave): every result equals
    the oracle's analysis of the same clip, value by value."""
    api = _api()
    specs = synth.config_batched(nclips=3, length_range=(60, 90), resolutions=((320, 180), (640, 360)))
    clips = [synth.Clip(s).frames() for s in specs]
    srv = api.Server(budget_bytes=8 << 30)
    tickets = [srv.submit(f, s.fps) for s, f in zip(specs, clips)]
    srv.drain()
    for t, f in zip(tickets, clips):
        _compare_results(srv.poll(t), OA.analyse_frames(f))
    srv.close()


def test_packed_sequence_rates_are_measured():
    """Each packed |a-b| sequence of the peak loop runs and gives a positive
    rate; sequence 0 is analyser_measure_sad_peak's; a sequence outside 0..4 is
    refused without device work."""
    import ctypes
    from paper_2502_09202_gb300 import native as N
    api = _api()
    rates = [api.sad_sequence_rate(q, 0) for q in range(5)]
    assert all(r > 0 for r in rates)
    v = ctypes.c_double()
    assert N.lib.analyser_measure_sad_sequence(0, 5, ctypes.byref(v)) == N.ERR_INVALID_ARG
    assert N.lib.analyser_measure_sad_sequence(0, 0, None) == N.ERR_INVALID_ARG
