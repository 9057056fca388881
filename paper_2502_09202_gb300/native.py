"""ctypes binding of include/analyser.h (argument marshalling only).

Loads the in-tree CUDA library ``libgb300va.so``.  There is no fallback: if
the library is missing, importing this module raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgb300va.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, PENDING = 0, -1, -2, -3, -4, -5, 1
UNKNOWN, PROGRESSIVE, INTERLACED, PULLDOWN = 0, 1, 2, 3
FO_NONE, FO_TFF, FO_BFF = 0, 1, 2
PAIR_FRAME, PAIR_UPPER_LOWER, PAIR_LOWER_UPPER = 0, 1, 2

c_int, c_double, c_ll, c_ull = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_ulonglong
c_i64 = ctypes.c_int64


class Params(ctypes.Structure):
    _fields_ = [
        ("block", c_int), ("levels", c_int), ("radius_coarse", c_int), ("radius_refine", c_int),
        ("mv_cost", c_int),
        ("kmax", c_int), ("jback", c_int), ("fast_window", c_int),
        ("fast_lambda", c_double), ("fast_rise", c_double), ("fast_tau", c_double), ("deep_rho", c_double), ("deep_tau", c_double),
        ("done_eps", c_double), ("steady_gamma", c_double), ("steady_frames", c_int), ("steady_span", c_int),
        ("lag_rho", c_double), ("blend_ratio", c_double),
        ("pd_rho", c_double), ("pd_gamma_new", c_double), ("pd_gamma_old", c_double),
        ("samp_max_frames", c_int),
        ("static_amm_px", c_double), ("comb_ratio", c_double), ("unequal_ratio", c_double),
        ("rep_ratio", c_double), ("rep_probe", c_int),
        ("pulldown_match", c_double),
        ("kf_theta", c_double),
        ("device", c_int), ("window_frames", c_int), ("mem_budget_bytes", c_ull), ("want_motion", c_int),
        ("tile_x", c_int), ("tile_y", c_int), ("time_kernels", c_int),
        ("step_frames", c_int), ("kernel_mode", c_int), ("want_histogram", c_int),
        ("prefetch_frames", c_int), ("wait_timeout_ms", c_double),
    ]


class Measure(ctypes.Structure):
    _fields_ = [("kind", c_int), ("a", c_int), ("b", c_int),
                ("si", c_i64), ("sj", c_i64), ("sii", c_i64), ("sjj", c_i64), ("sij", c_i64),
                ("sabs", c_i64), ("samm", c_i64), ("n", c_i64), ("nb", c_i64),
                ("ncc", c_double), ("swr", c_double), ("amm", c_double), ("act", c_double)]


class Shot(ctypes.Structure):
    _fields_ = [("first", c_int), ("last", c_int), ("label", c_int), ("field_order", c_int),
                ("pulldown_phase", c_int), ("analysed", c_int)]


class FrameHist(ctypes.Structure):
    _fields_ = [("frame", c_int), ("bins", ctypes.c_uint32 * 256), ("mean", c_double), ("std", c_double),
                ("median", c_int), ("mad", c_int)]


class Results(ctypes.Structure):
    _fields_ = [("nframes", c_int),
                ("ncuts", c_int), ("cuts", ctypes.POINTER(c_int)),
                ("ndissolves", c_int), ("dissolves", ctypes.POINTER(c_int)),
                ("nshots", c_int), ("shots", ctypes.POINTER(Shot)),
                ("label", c_int), ("field_order", c_int), ("pulldown_phase", c_int),
                ("nkeyframes", c_int), ("keyframes", ctypes.POINTER(c_int)),
                ("nmeasures", c_int), ("measures", ctypes.POINTER(Measure)),
                ("motion_w", c_int), ("motion_h", c_int), ("motion", ctypes.POINTER(ctypes.c_int16)),
                ("nhist", c_int), ("hist", ctypes.POINTER(FrameHist))]


class Profile(ctypes.Structure):
    _fields_ = [("pairs", c_ll), ("waves", c_ll), ("launches", c_ll), ("pair_launches", c_ll),
                ("pyramid_launches", c_ll), ("pair_kernel_ms", c_double), ("pyramid_kernel_ms", c_double),
                ("absdiff_ops", c_double), ("pyramid_bytes", c_double), ("h2d_bytes", c_ll), ("d2h_bytes", c_ll),
                ("host_gather_ms", c_double), ("host_wait_ms", c_double), ("host_results_ms", c_double),
                ("host_setup_ms", c_double), ("host_copy_wait_ms", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


MEASURE_FN = ctypes.CFUNCTYPE(c_int, ctypes.c_void_p, c_int, c_int, c_int, ctypes.POINTER(c_i64))

class FlowParams(ctypes.Structure):
    _fields_ = [("levels", c_int), ("patch", c_int), ("stride", c_int), ("iters", c_int), ("fp64", c_int),
                ("damp_rel", c_double), ("damp_abs", c_double)]


class FlowMeasure(ctypes.Structure):
    _fields_ = [("amm", c_double), ("ncc", c_double), ("swr", c_double), ("act", c_double),
                ("sums", c_double * 6)]


# every entry point of include/analyser.h: name -> (restype, argtypes)
P, VP = ctypes.POINTER, ctypes.c_void_p
SIGNATURES = {
    "analyser_default_params": (c_int, [P(Params)]),
    "analyser_create": (c_int, [c_int, c_int, c_double, P(Params), P(VP)]),
    "analyser_push_frames": (c_int, [VP, VP, c_ll, c_int]),
    "analyser_push_frames_device": (c_int, [VP, VP, c_ll, c_ll, c_int]),
    "analyser_finish": (c_int, [VP]),
    "analyser_results": (c_int, [VP, P(Results)]),
    "analyser_last_error": (c_int, [VP, P(ctypes.c_char_p)]),
    "analyser_stats": (c_int, [VP, P(c_ll), P(c_ll), P(c_ll)]),
    "analyser_profile": (c_int, [VP, P(Profile)]),
    "analyser_destroy": (None, [VP]),
    "analyser_measure_pairs": (c_int, [P(Params), c_int, c_int, VP, c_ll, c_ll, c_int, P(c_int), P(c_int),
                                       P(c_int), c_int, P(c_i64), P(ctypes.c_int16), VP]),
    "analyser_measure_pair_noalloc": (c_int, [P(Params), c_int, c_int, c_int, VP, VP, c_ll, P(c_i64), VP]),
    "analyser_detect_offline": (c_int, [P(Params), c_int, c_int, c_int, MEASURE_FN, VP, P(VP)]),
    "analyser_measure_sad_peak": (c_int, [c_int, P(c_double)]),
    "analyser_measure_sad_sequence": (c_int, [c_int, c_int, P(c_double)]),
    "analyser_default_flow_params": (None, [P(FlowParams)]),
    "analyser_dense_flow": (c_int, [P(FlowParams), c_int, c_int, VP, VP, c_ll, VP, VP]),
    "analyser_flow_measure": (c_int, [P(FlowParams), c_int, c_int, VP, VP, c_ll, P(FlowMeasure), VP]),
    "analyser_trim_cache": (None, []),
    "analyser_cached_bytes": (c_ll, []),
    "server_create": (c_int, [P(Params), c_ull, P(VP)]),
    "server_submit": (c_int, [VP, c_int, c_int, c_double, VP, c_ll, c_int, P(c_ll)]),
    "server_step": (c_int, [VP, P(c_int)]),
    "server_drain": (c_int, [VP]),
    "server_poll": (c_int, [VP, c_ll, P(Results)]),
    "server_profile": (c_int, [VP, P(Profile)]),
    "server_latency": (c_int, [VP, c_ll, P(c_double)]),
    "server_release": (c_int, [VP, c_ll]),
    "server_destroy": (None, [VP]),
}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library {LIB_PATH} is missing; build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class AnalyserError(RuntimeError):
    def __init__(self, code: int, where: str, message: str = ""):
        super().__init__(f"{where} failed with status {code}" + (f": {message}" if message else ""))
        self.code = code


def default_params(**overrides) -> Params:
    p = Params()
    lib.analyser_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p
