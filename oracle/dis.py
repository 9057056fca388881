"""Oracle of the dense sub-pixel flow estimator (test infrastructure only: see
oracle/__init__.py).

The paper computes its motion field with dense inverse search (Sec. III.A,
reference [8]).  This module states that method's steps for one pair of 8-bit
frames, in FP64, in the order the method takes them:

  1. pyramid: the box pyramid of the block-matching path (levels L-1 .. 0);
  2. per level, coarsest first, a grid of P x P patches of the first frame
     (stride S; the last patch of a row or column flush with the border);
  3. per patch, inverse search: the template's gradients (central differences,
     clamp-to-edge) give the 2 x 2 Gauss-Newton matrix H once; then `iters`
     steps of r(x) = J(x + u) - T(x) (J sampled bilinearly, clamp-to-edge),
     b = sum grad T(x) r(x), u <- u - (H + d I)^-1 b, with the damping
     d = damp_rel * trace(H) + damp_abs;
  4. the patch flows start from the next coarser level's dense flow, sampled
     bilinearly at the patch centre and doubled (zero at the coarsest level);
  5. densification: the flow at a pixel is the mean of the flows of the patches
     that cover it, each weighted by 1 / max(1, |J(x + u_i) - I(x)|).

Readings where the method leaves a choice (fixed here for both sides): no
patch-mean normalisation, no early stop or patch rejection, a fixed number of
steps, the damping above, no variational refinement, pixel centres aligned
between levels (coarse coordinate = (fine - 0.5) / 2).  Every step is a
continuous function of the inputs, so a GPU computing the same steps in FP32
differs from this oracle by rounding only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import measures as M


@dataclass(frozen=True)
class DisParams:
    levels: int = 3          # pyramid levels; the flow is returned at level 0
    patch: int = 8           # P
    stride: int = 4          # S
    iters: int = 8
    damp_rel: float = 0.01
    damp_abs: float = 1.0


def patch_origins(n: int, P: int, S: int) -> list[int]:
    """Patch starts along one axis of length n >= P: 0, S, 2S, ... and n - P."""
    if n < P:
        raise ValueError("image smaller than a patch")
    k = list(range(0, n - P + 1, S))
    if k[-1] != n - P:
        k.append(n - P)
    return k


def gradients(img: np.ndarray):
    """Central differences (I(x+1) - I(x-1)) / 2 with clamp-to-edge neighbours."""
    p = np.pad(img.astype(np.float64), 1, mode="edge")
    gx = (p[1:-1, 2:] - p[1:-1, :-2]) / 2.0
    gy = (p[2:, 1:-1] - p[:-2, 1:-1]) / 2.0
    return gx, gy


def bilinear(img: np.ndarray, x, y):
    """img sampled at (x, y), positions clamped to the image, then bilinear
    between the four surrounding pixels."""
    h, w = img.shape
    x = np.clip(np.asarray(x, np.float64), 0.0, w - 1.0)
    y = np.clip(np.asarray(y, np.float64), 0.0, h - 1.0)
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    x1 = np.minimum(x0 + 1, w - 1)
    y1 = np.minimum(y0 + 1, h - 1)
    fx = x - x0
    fy = y - y0
    im = img.astype(np.float64)
    top = im[y0, x0] * (1.0 - fx) + im[y0, x1] * fx
    bot = im[y1, x0] * (1.0 - fx) + im[y1, x1] * fx
    return top * (1.0 - fy) + bot * fy


def patch_grid(h: int, w: int, P: int, S: int):
    """Patch origins (ys, xs) in row-major patch order."""
    ys, xs = patch_origins(h, P, S), patch_origins(w, P, S)
    oy, ox = np.meshgrid(np.array(ys), np.array(xs), indexing="ij")
    return oy.ravel(), ox.ravel(), len(ys), len(xs)


def inverse_search(I: np.ndarray, J: np.ndarray, init: np.ndarray, dp: DisParams = DisParams()):
    """Flows (npatch, 2) of the patch grid of I after `iters` Gauss-Newton steps
    from `init` (npatch, 2), step 3 above."""
    P = dp.patch
    oy, ox, _, _ = patch_grid(*I.shape, P, dp.stride)
    gx, gy = gradients(I)
    T = I.astype(np.float64)
    ry, rx = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    Y = oy[:, None, None] + ry[None]          # (N, P, P) pixel rows
    X = ox[:, None, None] + rx[None]
    t, ggx, ggy = T[Y, X], gx[Y, X], gy[Y, X]
    h00 = (ggx * ggx).sum(axis=(1, 2))
    h01 = (ggx * ggy).sum(axis=(1, 2))
    h11 = (ggy * ggy).sum(axis=(1, 2))
    d = dp.damp_rel * (h00 + h11) + dp.damp_abs
    a, c = h00 + d, h11 + d
    det = a * c - h01 * h01
    u = np.array(init, np.float64).copy()
    for _ in range(dp.iters):
        r = bilinear(J, X + u[:, 0, None, None], Y + u[:, 1, None, None]) - t
        bx = (ggx * r).sum(axis=(1, 2))
        by = (ggy * r).sum(axis=(1, 2))
        u[:, 0] -= (c * bx - h01 * by) / det
        u[:, 1] -= (a * by - h01 * bx) / det
    return u


def densify(I: np.ndarray, J: np.ndarray, flows: np.ndarray, dp: DisParams = DisParams()) -> np.ndarray:
    """Dense flow (h, w, 2): per pixel the photometric-error weighted mean of the
    covering patches' flows (step 5), accumulated patch by patch in row-major
    patch order."""
    h, w = I.shape
    P = dp.patch
    oy, ox, _, _ = patch_grid(h, w, P, dp.stride)
    ry, rx = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    Y = (oy[:, None, None] + ry[None]).reshape(len(oy), -1)      # (N, P*P)
    X = (ox[:, None, None] + rx[None]).reshape(len(oy), -1)
    fx, fy = flows[:, 0, None], flows[:, 1, None]
    e = bilinear(J, X + fx, Y + fy) - I.astype(np.float64)[Y, X]
    wgt = 1.0 / np.maximum(1.0, np.abs(e))
    num = np.zeros((h, w, 2))
    den = np.zeros((h, w))
    # np.add.at applies the patches' contributions in index order (patch-major)
    np.add.at(num[..., 0], (Y.ravel(), X.ravel()), (wgt * fx).ravel())
    np.add.at(num[..., 1], (Y.ravel(), X.ravel()), (wgt * fy).ravel())
    np.add.at(den, (Y.ravel(), X.ravel()), wgt.ravel())
    return num / den[..., None]


def init_from_coarse(h: int, w: int, coarse: np.ndarray | None, dp: DisParams = DisParams()) -> np.ndarray:
    """Patch initial flows at a level of size (h, w) from the coarser dense flow
    (step 4): sampled at the patch centre's coarse position and doubled."""
    oy, ox, _, _ = patch_grid(h, w, dp.patch, dp.stride)
    if coarse is None:
        return np.zeros((len(oy), 2))
    cx = (ox + (dp.patch - 1) / 2.0 - 0.5) / 2.0
    cy = (oy + (dp.patch - 1) / 2.0 - 0.5) / 2.0
    return np.stack([2.0 * bilinear(coarse[..., 0], cx, cy), 2.0 * bilinear(coarse[..., 1], cx, cy)], axis=1)


def dis_flow(fa: np.ndarray, fb: np.ndarray, dp: DisParams = DisParams()) -> np.ndarray:
    """Dense flow (H, W, 2) from frame a to frame b (steps 1-5): frame b at
    x + U(x) matches frame a at x."""
    pa, pb = M.pyramid(fa, dp.levels), M.pyramid(fb, dp.levels)
    U = None
    for l in range(dp.levels - 1, -1, -1):
        I, J = pa[l], pb[l]
        init = init_from_coarse(*I.shape, U, dp)
        flows = inverse_search(I, J, init, dp)
        U = densify(I, J, flows, dp)
    return U


def flow_measure(fa: np.ndarray, fb: np.ndarray, dp: DisParams = DisParams()) -> dict:
    """The pair measures of Sec. III.A with the dense flow U as the motion
    field: AMM = mean |U(x)| over the n pixels; frame b warped by U,
    Jw(x) = J(x + U(x)) (bilinear, clamp-to-edge); NCC of frame a and Jw from
    the sums S_i, S_j, S_ii, S_jj, S_ij as C / sqrt(Vi * Vj) with C = n S_ij -
    S_i S_j, Vi = n S_ii - S_i^2, Vj = n S_jj - S_j^2 (both variances zero or
    below: 1, one of them: 0); SWR = max(0, 1 - NCC); ACT = sqrt(AMM * SWR)."""
    U = dis_flow(fa, fb, dp)
    h, w = fa.shape
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    I = fa.astype(np.float64)
    Jw = bilinear(fb, xx + U[..., 0], yy + U[..., 1])
    n = float(h * w)
    si, sj = I.sum(), Jw.sum()
    sii, sjj, sij = (I * I).sum(), (Jw * Jw).sum(), (I * Jw).sum()
    smag = np.sqrt(U[..., 0] ** 2 + U[..., 1] ** 2).sum()
    c = n * sij - si * sj
    vi = n * sii - si * si
    vj = n * sjj - sj * sj
    if vi <= 0.0 and vj <= 0.0:
        ncc = 1.0
    elif vi <= 0.0 or vj <= 0.0:
        ncc = 0.0
    else:
        ncc = c / np.sqrt(vi * vj)
    swr = max(0.0, 1.0 - ncc)
    amm = smag / n
    return {"amm": float(amm), "ncc": float(ncc), "swr": float(swr), "act": float(np.sqrt(amm * swr)),
            "sums": [float(v) for v in (smag, si, sj, sii, sjj, sij)], "n": int(h * w)}
