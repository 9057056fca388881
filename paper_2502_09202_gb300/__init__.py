"""GB300 video analyser: shot boundaries, sampling structure and dynamic keyframes
(arXiv 2502.09202) with the per-frame measures computed by hand-written CUDA for sm_103a.

    from paper_2502_09202_gb300 import Analyser
    with Analyser(1920, 1080, fps=25.0) as a:
        a.push(frames)            # uint8 (n, 1080, 1920), host memory
        a.finish()
        res = a.results()         # cuts, dissolves, shots, label, field order, keyframes, measures

The CUDA library is built in-tree by ``build.build()``; using the API without
it raises ImportError (there is no CPU fallback).  ``synth`` (the synthetic
video generator) imports without the library.
"""
_API = ("Analyser", "Server", "AnalyserError", "analyse", "default_params", "detect_offline", "measure_pairs")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
