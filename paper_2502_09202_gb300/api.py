"""Python face of the C ABI: Analyser, Server, measure_pairs, detect_offline.

Every computation runs in the CUDA library; this module converts arguments and
results.  PyTorch is used only to hand over device buffers and streams.
"""
from __future__ import annotations

import ctypes
from collections.abc import Mapping

import numpy as np

from . import native as N
from .native import AnalyserError, default_params

__all__ = ["Analyser", "Server", "measure_pairs", "detect_offline", "default_params", "AnalyserError",
           "results_to_dict", "sad_peak", "sad_sequence_rate", "MeasureTable", "trim_cache",
           "flow_params", "dense_flow", "flow_measure"]


def _check(code: int, where: str, handle=None):
    if code not in (N.OK, N.PENDING):
        msg = ""
        if handle is not None and where.startswith("analyser"):
            m = ctypes.c_char_p()
            N.lib.analyser_last_error(handle, ctypes.byref(m))
            msg = (m.value or b"").decode(errors="replace")
        raise AnalyserError(code, where, msg)
    return code


class MeasureTable(Mapping):
    """The measures of a clip keyed by (kind, a, b): a read-only mapping over one
    structured numpy array (``.array``, fields as in the C struct), copied from
    the library in one piece; a value is built as a dict when it is read."""

    FIELDS = ("si", "sj", "sii", "sjj", "sij", "sabs", "samm", "n", "nb", "ncc", "swr", "amm", "act")

    def __init__(self, array: np.ndarray):
        self.array = array
        self._index = None

    def _keys(self) -> dict:
        if self._index is None:
            a = self.array
            self._index = {k: i for i, k in enumerate(zip(a["kind"].tolist(), a["a"].tolist(), a["b"].tolist()))}
        return self._index

    def __getitem__(self, key):
        row = self.array[self._keys()[tuple(key)]]
        return {f: row[f].item() for f in self.FIELDS}

    def __iter__(self):
        return iter(self._keys())

    def __len__(self):
        return len(self.array)

    def __contains__(self, key):
        return tuple(key) in self._keys()


def _ints(ptr, n: int) -> list:
    return np.ctypeslib.as_array(ptr, shape=(n,)).tolist() if n > 0 else []


def results_to_dict(r: N.Results) -> dict:
    """Results in the layout the oracle returns (measures keyed by (kind, a, b))."""
    cuts = _ints(r.cuts, r.ncuts)
    d = _ints(r.dissolves, 2 * r.ndissolves)
    dis = [(d[2 * i], d[2 * i + 1]) for i in range(r.ndissolves)]
    shots = [{"first": s.first, "last": s.last, "label": s.label, "field_order": s.field_order,
              "phase": s.pulldown_phase, "analysed": s.analysed} for s in (r.shots[i] for i in range(r.nshots))]
    kf = _ints(r.keyframes, r.nkeyframes)
    if r.nmeasures > 0:
        meas = MeasureTable(np.ctypeslib.as_array(r.measures, shape=(r.nmeasures,)).copy())
    else:
        meas = MeasureTable(np.zeros(0, dtype=np.dtype(N.Measure)))
    out = {"cuts": cuts, "dissolves": dis, "keyframes": kf, "shots": shots, "label": r.label,
           "field_order": r.field_order, "pulldown_phase": r.pulldown_phase, "measures": meas,
           "nframes": r.nframes}
    if r.motion:
        n = max(r.nframes - 1, 0) * r.motion_h * r.motion_w * 2
        out["motion"] = np.ctypeslib.as_array(r.motion, shape=(n,)).reshape(-1, r.motion_h, r.motion_w, 2).copy()
    if r.nhist > 0:
        h = np.ctypeslib.as_array(r.hist, shape=(r.nhist,)).copy()
        out["histograms"] = [{"frame": int(x["frame"]), "bins": x["bins"].astype(np.int64), "mean": float(x["mean"]),
                              "std": float(x["std"]), "median": int(x["median"]), "mad": int(x["mad"])} for x in h]
    return out


class Analyser:
    """One clip: create, push frames (host or device), finish, results."""

    def __init__(self, width: int, height: int, fps: float = 25.0, params: N.Params | None = None, **overrides):
        self.params = params if params is not None else default_params(**overrides)
        self._h = ctypes.c_void_p()
        _check(N.lib.analyser_create(width, height, float(fps), ctypes.byref(self.params), ctypes.byref(self._h)),
               "analyser_create")
        self.width, self.height = width, height
        self._keep = []          # device buffers referenced by push_device

    def push(self, frames: np.ndarray):
        """Host frames: uint8 array (n, height, width) or (height, width)."""
        f = np.ascontiguousarray(frames, dtype=np.uint8)
        if f.ndim == 2:
            f = f[None]
        assert f.shape[1:] == (self.height, self.width), f.shape
        _check(N.lib.analyser_push_frames(self._h, f.ctypes.data, f.shape[2], f.shape[0]), "analyser_push_frames",
               self._h)

    def push_host_ptr(self, ptr: int, pitch: int, n: int):
        _check(N.lib.analyser_push_frames(self._h, ptr, pitch, n), "analyser_push_frames", self._h)

    def push_device(self, frames):
        """Device frames: a CUDA uint8 torch tensor (n, height, pitch>=width) kept alive until finish()."""
        assert frames.is_cuda and frames.dtype.itemsize == 1 and frames.dim() == 3
        pitch = frames.stride(1)
        stride = frames.stride(0)
        assert frames.stride(2) == 1
        self._keep.append(frames)
        _check(N.lib.analyser_push_frames_device(self._h, frames.data_ptr(), pitch, stride, frames.shape[0]),
               "analyser_push_frames_device", self._h)

    def finish(self):
        _check(N.lib.analyser_finish(self._h), "analyser_finish", self._h)

    def results(self) -> dict:
        r = N.Results()
        _check(N.lib.analyser_results(self._h, ctypes.byref(r)), "analyser_results", self._h)
        return results_to_dict(r)

    def stats(self) -> dict:
        p, w, l = N.c_ll(), N.c_ll(), N.c_ll()
        N.lib.analyser_stats(self._h, ctypes.byref(p), ctypes.byref(w), ctypes.byref(l))
        return {"pairs": p.value, "waves": w.value, "launches": l.value}

    def profile(self) -> dict:
        pr = N.Profile()
        N.lib.analyser_profile(self._h, ctypes.byref(pr))
        return pr.as_dict()

    def close(self):
        if self._h:
            N.lib.analyser_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def analyse(frames: np.ndarray, fps: float = 25.0, **overrides) -> dict:
    """Whole-clip convenience: host frames in, results out."""
    n, h, w = frames.shape
    with Analyser(w, h, fps, **overrides) as a:
        a.push(frames)
        a.finish()
        return a.results()


def flow_params(**overrides) -> N.FlowParams:
    p = N.FlowParams()
    N.lib.analyser_default_flow_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def dense_flow(frame_a, frame_b, out=None, stream=None, **overrides):
    """Dense sub-pixel flow (analyser_dense_flow) from frame a to frame b, both CUDA
    uint8 tensors (h, w) with unit column stride and the same row pitch.  Returns
    a CUDA float32 tensor (h, w, 2) of (u, v) per pixel (`out` if given)."""
    import torch
    assert frame_a.is_cuda and frame_b.is_cuda and frame_a.dim() == 2 and frame_a.shape == frame_b.shape
    assert frame_a.stride(1) == 1 and frame_b.stride(1) == 1 and frame_a.stride(0) == frame_b.stride(0)
    h, w = frame_a.shape
    if out is None:
        out = torch.empty((h, w, 2), dtype=torch.float32, device=frame_a.device)
    assert out.is_cuda and out.is_contiguous() and out.shape == (h, w, 2) and out.dtype == torch.float32
    p = flow_params(**overrides)
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(N.lib.analyser_dense_flow(ctypes.byref(p), w, h, frame_a.data_ptr(), frame_b.data_ptr(), frame_a.stride(0),
                                     out.data_ptr(), ctypes.c_void_p(st)), "analyser_dense_flow")
    return out


def flow_measure(frame_a, frame_b, stream=None, **overrides) -> dict:
    """Pair measures (amm, ncc, swr, act, sums) of frame a and frame b with the dense
    flow as the motion field (analyser_flow_measure); frames as for dense_flow."""
    import torch
    assert frame_a.is_cuda and frame_b.is_cuda and frame_a.dim() == 2 and frame_a.shape == frame_b.shape
    assert frame_a.stride(1) == 1 and frame_b.stride(1) == 1 and frame_a.stride(0) == frame_b.stride(0)
    h, w = frame_a.shape
    p = flow_params(**overrides)
    m = N.FlowMeasure()
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(N.lib.analyser_flow_measure(ctypes.byref(p), w, h, frame_a.data_ptr(), frame_b.data_ptr(),
                                       frame_a.stride(0), ctypes.byref(m), ctypes.c_void_p(st)), "analyser_flow_measure")
    return {"amm": m.amm, "ncc": m.ncc, "swr": m.swr, "act": m.act, "sums": list(m.sums), "n": int(h * w)}


def measure_pairs(frames, kinds, ia, ib, params: N.Params | None = None, want_motion: bool = False,
                  stream=None, **overrides):
    """Stateless measures of pairs of DEVICE frames: a CUDA uint8 tensor (n, h, w) whose rows
    may be padded (a view frames[:, :, :w] of a wider buffer; row pitch = stride(1)).

    Returns (records int64 (npairs, 7), motion int16 list or None)."""
    import torch
    assert frames.is_cuda and frames.dim() == 3 and frames.stride(2) == 1
    p = params if params is not None else default_params(**overrides)
    n, h, w = frames.shape[0], frames.shape[1], frames.shape[2]
    kinds = np.ascontiguousarray(kinds, dtype=np.int32)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    npairs = len(kinds)
    rec = np.zeros((npairs, 7), np.int64)
    B0 = p.block
    mot = None
    mot_ptr = None
    if want_motion:
        sizes = [(w // B0) * ((h if k == 0 else h // 2) // B0) * 2 for k in kinds]
        mot = np.zeros(sum(sizes), np.int16)
        mot_ptr = mot.ctypes.data_as(ctypes.POINTER(ctypes.c_int16))
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    code = N.lib.analyser_measure_pairs(
        ctypes.byref(p), w, h, frames.data_ptr(), frames.stride(1), frames.stride(0), n,
        kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        ib.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), npairs, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        mot_ptr, ctypes.c_void_p(st))
    _check(code, "analyser_measure_pairs")
    if want_motion:
        out, off = [], 0
        for k in kinds:
            hh = h if k == 0 else h // 2
            m = (w // B0) * (hh // B0) * 2
            out.append(mot[off:off + m].reshape(hh // B0, w // B0, 2))
            off += m
        return rec, out
    return rec, None


def trim_cache() -> int:
    """Return the library's cached device and page-locked buffers to CUDA; the
    device bytes that were cached."""
    n = int(N.lib.analyser_cached_bytes())
    N.lib.analyser_trim_cache()
    return n


def sad_peak(device: int = 0) -> float:
    """Measured packed-SAD throughput of this GPU, 10^12 |a-b| accumulates per second."""
    v = ctypes.c_double()
    _check(N.lib.analyser_measure_sad_peak(device, ctypes.byref(v)), "analyser_measure_sad_peak")
    return v.value


def sad_sequence_rate(sequence: int, device: int = 0) -> float:
    """|a-b| accumulates per second (T/s) of packed sequence `sequence` (0..4)
    in the peak loop: 0 vabsdiff4 with accumulate, 1 sum-of-absolute-differences
    plus add, 2 absolute differences plus dp4a, 3 max - min plus dp4a, 4 half and half of 0 and 2."""
    v = ctypes.c_double()
    _check(N.lib.analyser_measure_sad_sequence(device, sequence, ctypes.byref(v)), "analyser_measure_sad_sequence")
    return v.value


def detect_offline(width: int, height: int, nframes: int, get_record, params: N.Params | None = None,
                   **overrides) -> dict:
    """Run the library's detectors (host only, no GPU) on records from ``get_record(kind, a, b)``,
    which returns the 9 integers (si, sj, sii, sjj, sij, sabs, samm, n, nb)."""
    p = params if params is not None else default_params(**overrides)
    errors = []

    def cb(ctx, kind, a, b, rec):
        try:
            vals = get_record(kind, a, b)
            for i in range(9):
                rec[i] = int(vals[i])
            return 0
        except Exception as e:  # pragma: no cover - surfaced below
            errors.append(e)
            return 1

    fn = N.MEASURE_FN(cb)
    h = ctypes.c_void_p()
    code = N.lib.analyser_detect_offline(ctypes.byref(p), width, height, nframes, fn, None, ctypes.byref(h))
    if errors:
        raise errors[0]
    _check(code, "analyser_detect_offline")
    try:
        r = N.Results()
        _check(N.lib.analyser_results(h, ctypes.byref(r)), "analyser_results")
        return results_to_dict(r)
    finally:
        N.lib.analyser_destroy(h)


class Server:
    """Continuous batching of many clips on one GPU under a device-memory budget."""

    def __init__(self, budget_bytes: int, params: N.Params | None = None, **overrides):
        self.params = params if params is not None else default_params(**overrides)
        self._h = ctypes.c_void_p()
        _check(N.lib.server_create(ctypes.byref(self.params), int(budget_bytes), ctypes.byref(self._h)),
               "server_create")
        self._frames = {}

    def submit(self, frames: np.ndarray, fps: float = 25.0) -> int:
        f = np.ascontiguousarray(frames, dtype=np.uint8)
        t = N.c_ll()
        _check(N.lib.server_submit(self._h, f.shape[2], f.shape[1], float(fps), f.ctypes.data, f.shape[2],
                                   f.shape[0], ctypes.byref(t)), "server_submit")
        self._frames[t.value] = f      # the server reads it until the request is done
        return t.value

    def step(self) -> int:
        active = ctypes.c_int()
        _check(N.lib.server_step(self._h, ctypes.byref(active)), "server_step")
        return active.value

    def drain(self):
        _check(N.lib.server_drain(self._h), "server_drain")

    def poll(self, ticket: int):
        r = N.Results()
        code = _check(N.lib.server_poll(self._h, ticket, ctypes.byref(r)), "server_poll")
        if code == N.PENDING:
            return None
        return results_to_dict(r)

    def profile(self) -> dict:
        pr = N.Profile()
        N.lib.server_profile(self._h, ctypes.byref(pr))
        return pr.as_dict()

    def latency(self, ticket: int) -> float:
        s = ctypes.c_double()
        _check(N.lib.server_latency(self._h, ticket, ctypes.byref(s)), "server_latency")
        return s.value

    def release(self, ticket: int):
        _check(N.lib.server_release(self._h, ticket), "server_release")
        self._frames.pop(ticket, None)

    def close(self):
        if self._h:
            N.lib.server_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._frames.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
