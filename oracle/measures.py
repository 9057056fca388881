"""Oracle measures: ctypes wrapper over measures.c plus the FP64 finalisation.

Test infrastructure only (see oracle/__init__.py).

Pair kinds (the three ways the detectors pair frames, Sec. III.A and III.C, and
the two same-parity field pairs, an extension for repeated-field detection in
the spirit of Sec. III.C that the detectors do not use):
  FRAME (0)        I = frame a,            J = frame b
  UPPER_LOWER (1)  I = upper field of a,   J = lower field of b   (v0 = (1,t,t), v1 = (1,t,t+1))
  LOWER_UPPER (2)  I = lower field of a,   J = upper field of b   (v2 = (2,t,t+1))
  UPPER_UPPER (3)  I = upper field of a,   J = upper field of b
  LOWER_LOWER (4)  I = lower field of a,   J = lower field of b
The upper field is the even rows 0, 2, 4, ... of the frame; the lower field the odd rows.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build

FRAME, UPPER_LOWER, LOWER_UPPER, UPPER_UPPER, LOWER_LOWER = 0, 1, 2, 3, 4

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        p = ctypes.c_void_p
        _lib.orc_pair_record.argtypes = [p, p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p]
        _lib.orc_pair_record.restype = ctypes.c_int
        _lib.orc_downsample.argtypes = [p, ctypes.c_int, ctypes.c_int, ctypes.c_long, p]
        _lib.orc_sad.argtypes = [p, p] + [ctypes.c_int] * 7
        _lib.orc_sad.restype = ctypes.c_uint32
        _lib.orc_block_search.argtypes = [p, p, p, p] + [ctypes.c_int] * 5 + [p, p]
        _lib.orc_isqrt.argtypes = [ctypes.c_uint64]
        _lib.orc_isqrt.restype = ctypes.c_uint64
        _lib.orc_amm_sum.argtypes = [p, ctypes.c_long]
        _lib.orc_amm_sum.restype = ctypes.c_int64
        _lib.orc_warp_sums.argtypes = [p, p, ctypes.c_int, ctypes.c_int, p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, p]
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass(frozen=True)
class SearchParams:
    """Motion-search parameters (readings fixed for an unspecified estimator)."""
    levels: int = 3        # pyramid depth L
    block: int = 16        # level-0 block side B0
    radius: int = 16       # coarse exhaustive radius R (coarsest level)
    refine: int = 2        # refinement radius r at every finer level
    mv_cost: int = 4       # lambda: cost per pixel of |vx|+|vy| added to the SAD at every level


def field(frame: np.ndarray, which: str) -> np.ndarray:
    """Upper field = even rows, lower field = odd rows (Sec. III.C)."""
    return np.ascontiguousarray(frame[0::2] if which == "upper" else frame[1::2])


def pair_images(kind: int, fa: np.ndarray, fb: np.ndarray):
    if kind == FRAME:
        return np.ascontiguousarray(fa), np.ascontiguousarray(fb)
    if kind == UPPER_LOWER:
        return field(fa, "upper"), field(fb, "lower")
    if kind == LOWER_UPPER:
        return field(fa, "lower"), field(fb, "upper")
    if kind == UPPER_UPPER:
        return field(fa, "upper"), field(fb, "upper")
    if kind == LOWER_LOWER:
        return field(fa, "lower"), field(fb, "lower")
    raise ValueError(kind)


def downsample(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros((h // 2, w // 2), np.uint8)
    lib().orc_downsample(_ptr(img), w, h, w, _ptr(out))
    return out


def pyramid(img: np.ndarray, levels: int) -> list[np.ndarray]:
    pyr = [np.ascontiguousarray(img, dtype=np.uint8)]
    for _ in range(1, levels):
        pyr.append(downsample(pyr[-1]))
    return pyr


def sad(I: np.ndarray, J: np.ndarray, x0: int, y0: int, s: int, vx: int, vy: int) -> int:
    h, w = I.shape
    return int(lib().orc_sad(_ptr(I), _ptr(J), w, h, x0, y0, s, vx, vy))


def block_search(I: np.ndarray, J: np.ndarray, sp: SearchParams = SearchParams()):
    """Level-0 motion field (nby, nbx, 2) int16 [vx, vy] and level-0 SADs (nby, nbx)."""
    pI, pJ = pyramid(I, sp.levels), pyramid(J, sp.levels)
    ws = np.array([p.shape[1] for p in pI], np.int32)
    hs = np.array([p.shape[0] for p in pI], np.int32)
    nbx, nby = I.shape[1] // sp.block, I.shape[0] // sp.block
    vec = np.zeros((nby, nbx, 2), np.int16)
    sad0 = np.zeros((nby, nbx), np.uint32)
    arrI = (ctypes.c_void_p * sp.levels)(*[p.ctypes.data for p in pI])
    arrJ = (ctypes.c_void_p * sp.levels)(*[p.ctypes.data for p in pJ])
    lib().orc_block_search(ctypes.cast(arrI, ctypes.c_void_p), ctypes.cast(arrJ, ctypes.c_void_p), _ptr(ws),
                           _ptr(hs), sp.levels, sp.block, sp.radius, sp.refine, sp.mv_cost, _ptr(vec),
                           _ptr(sad0))
    return vec, sad0


def isqrt(n: int) -> int:
    return int(lib().orc_isqrt(n))


def amm_sum(vec: np.ndarray) -> int:
    v = np.ascontiguousarray(vec, dtype=np.int16)
    return int(lib().orc_amm_sum(_ptr(v), v.size // 2))


def warp_sums(I: np.ndarray, J: np.ndarray, vec: np.ndarray, block: int) -> list[int]:
    I = np.ascontiguousarray(I, dtype=np.uint8)
    J = np.ascontiguousarray(J, dtype=np.uint8)
    v = np.ascontiguousarray(vec, dtype=np.int16)
    h, w = I.shape
    out = np.zeros(6, np.int64)
    lib().orc_warp_sums(_ptr(I), _ptr(J), w, h, _ptr(v), v.shape[1], v.shape[0], block, _ptr(out))
    return [int(x) for x in out]


# record layout: the integer part of one pair measure
REC_FIELDS = ("si", "sj", "sii", "sjj", "sij", "sabs", "samm", "n", "nb")


def pair_record(I: np.ndarray, J: np.ndarray, sp: SearchParams = SearchParams(), want_vec: bool = False):
    """Integer record of one pair: the 6 motion-compensated sums, S_amm, n, nb."""
    I = np.ascontiguousarray(I, dtype=np.uint8)
    J = np.ascontiguousarray(J, dtype=np.uint8)
    h, w = I.shape
    rec = np.zeros(9, np.int64)
    vec = np.zeros((h // sp.block, w // sp.block, 2), np.int16) if want_vec else None
    rc = lib().orc_pair_record(_ptr(I), _ptr(J), w, h, sp.levels, sp.block, sp.radius, sp.refine, sp.mv_cost,
                               _ptr(rec),
                               _ptr(vec) if want_vec else None)
    if rc != 0:
        raise ValueError("oracle: unusable pair size or parameters")
    r = {k: int(x) for k, x in zip(REC_FIELDS, rec)}
    return (r, vec) if want_vec else r


def finalise(r: dict) -> dict:
    """FP64 measures of one pair (Sec. III.A), from its exact integer record.

    C = n*Sij - Si*Sj, Vi = n*Sii - Si^2, Vj = n*Sjj - Sj^2 are exact integers;
    NCC = C / sqrt(Vi*Vj) as three correctly rounded operations (both variances
    zero: 1; one of them zero: 0); SWR = max(0, 1 - NCC);
    AMM = S_amm / (nb * 65536) in px; ACT = sqrt(AMM * SWR), the geometric mean.
    """
    n, si, sj = r["n"], r["si"], r["sj"]
    c = n * r["sij"] - si * sj
    vi = n * r["sii"] - si * si
    vj = n * r["sjj"] - sj * sj
    if vi == 0 and vj == 0:
        ncc = 1.0
    elif vi == 0 or vj == 0:
        ncc = 0.0
    else:
        ncc = float(c) / math.sqrt(float(vi) * float(vj))
    one_minus = 1.0 - ncc
    swr = one_minus if one_minus > 0.0 else 0.0
    amm = float(r["samm"]) / (float(r["nb"]) * 65536.0)
    act = math.sqrt(amm * swr)
    out = dict(r)
    out.update(ncc=ncc, swr=swr, amm=amm, act=act)
    return out


def measure(kind: int, fa: np.ndarray, fb: np.ndarray, sp: SearchParams = SearchParams()) -> dict:
    I, J = pair_images(kind, fa, fb)
    return finalise(pair_record(I, J, sp))


def frame_histogram(frame: np.ndarray) -> dict:
    """Unary measure of a frame (Sec. III.A names histogram measures among the
    unary ones): the 256-bin histogram of its luma and statistics from exact
    integer sums S1 = sum v, S2 = sum v^2 over the n pixels:
    mean = S1/n, std = sqrt((n*S2 - S1^2) / (n*n)) (FP64, this order),
    median = lower median (sorted index (n-1)//2), mad = lower median of
    |v - median|."""
    f = np.asarray(frame, dtype=np.uint8)
    bins = np.bincount(f.ravel(), minlength=256).astype(np.int64)
    n = int(f.size)
    v = np.arange(256, dtype=np.int64)
    s1 = int((v * bins).sum())
    s2 = int((v * v * bins).sum())
    mean = float(s1) / float(n)
    std = math.sqrt(float(n * s2 - s1 * s1) / (float(n) * float(n)))
    k = (n - 1) // 2
    med = int(np.searchsorted(np.cumsum(bins), k + 1))
    dev = np.zeros(256, dtype=np.int64)
    for d in range(256):
        if d == 0:
            dev[d] = bins[med]
        else:
            dev[d] = (bins[med + d] if med + d < 256 else 0) + (bins[med - d] if med - d >= 0 else 0)
    mad = int(np.searchsorted(np.cumsum(dev), k + 1))
    return {"bins": bins, "mean": mean, "std": std, "median": med, "mad": mad}
