"""Pins for the oracle: each test checks it against something other than itself.

Closed forms, invariants, special cases that reduce to a textbook or library
routine, and brute force on tiny inputs written in a different formulation
(padding instead of clamping, numpy instead of loops).
"""
import math
import os

import numpy as np
import pytest

from oracle import measures as M
from oracle.measures import SearchParams
from paper_2502_09202_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- pyramid (box filter, round half up) -------------------------------------

def test_pyramid_golden_blocks():
    for line in open(os.path.join(GOLDEN, "pyramid_2x2.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        a, b, c, d = map(int, lhs.split())
        img = np.array([[a, b], [c, d]], np.uint8)
        assert M.downsample(img)[0, 0] == int(rhs), line


def test_pyramid_constant_and_replicated():
    rng = np.random.default_rng(1)
    const = np.full((37, 53), 77, np.uint8)
    for lvl in M.pyramid(const, 4)[1:]:
        assert (lvl == 77).all()
    small = rng.integers(0, 256, (9, 13), dtype=np.uint8)
    up = np.repeat(np.repeat(small, 2, axis=0), 2, axis=1)
    assert np.array_equal(M.downsample(up), small)
    # odd sizes floor: the last row/column are dropped
    odd = np.pad(up, ((0, 1), (0, 1)), constant_values=255)
    assert np.array_equal(M.downsample(odd), small)


def test_pyramid_matches_float_mean_rounding():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    q = img.reshape(10, 2, 15, 2).astype(np.float64).sum(axis=(1, 3)) / 4.0
    expect = np.floor(q + 0.5).astype(np.uint8)           # round half up
    assert np.array_equal(M.downsample(img), expect)


# ---- block search ----------------------------------------------------------------

def test_identical_pair_gives_zero_field():
    I = synth.random_frame(3, 96, 64)
    vec, sad0 = M.block_search(I, I)
    assert (vec == 0).all() and (sad0 == 0).all()


def test_flat_images_tie_break_to_zero():
    I = np.full((64, 64), 90, np.uint8)
    J = np.full((64, 64), 91, np.uint8)
    vec, sad0 = M.block_search(I, J, SearchParams(mv_cost=0))
    assert (vec == 0).all()
    assert (sad0 == 256).all()


@pytest.mark.parametrize("sx,sy", [(0, 0), (4, -8), (-16, 12), (32, 28), (-40, 12), (64, -4)])
def test_known_global_shift_recovered(sx, sy):
    """A shift that is a multiple of 2^(L-1) is an exact shift at every pyramid
    level, so the zero-SAD match is found at the coarsest level and kept."""
    I, J = synth.shifted_pair(11, 192, 160, sx, sy)
    sp = SearchParams()
    vec, sad0 = M.block_search(I, J, sp)
    nby, nbx = vec.shape[:2]
    checked = 0
    for by in range(nby):
        for bx in range(nbx):
            x0, y0 = bx * sp.block, by * sp.block
            inside = (0 <= x0 + sx and x0 + sx + sp.block <= 192 and 0 <= y0 + sy and y0 + sy + sp.block <= 160)
            # the coarse level must also see the whole matched block inside J
            s2 = sp.block >> (sp.levels - 1)
            inside2 = all(0 <= (x0 >> 2) + d and (x0 >> 2) + d + s2 <= 48 for d in (sx // 4, -(-sx // 4))) and \
                all(0 <= (y0 >> 2) + d and (y0 >> 2) + d + s2 <= 40 for d in (sy // 4, -(-sy // 4)))
            if inside and inside2:
                assert tuple(vec[by, bx]) == (sx, sy), (bx, by, vec[by, bx])
                assert sad0[by, bx] == 0
                checked += 1
    assert checked >= 4


def _brute_single_level(I, J, s, R, lam):
    """Exhaustive search on one level, clamping expressed as edge padding."""
    h, w = I.shape
    P = np.pad(J.astype(np.int64), R, mode="edge")
    nbx, nby = w // s, h // s
    out = np.zeros((nby, nbx, 2), np.int64)
    for by in range(nby):
        for bx in range(nbx):
            blk = I[by * s:(by + 1) * s, bx * s:(bx + 1) * s].astype(np.int64)
            keys = []
            for vy in range(-R, R + 1):
                for vx in range(-R, R + 1):
                    y0, x0 = by * s + vy + R, bx * s + vx + R
                    sad = int(np.abs(blk - P[y0:y0 + s, x0:x0 + s]).sum())
                    n1 = abs(vx) + abs(vy)
                    keys.append((sad + lam * n1, n1, vy, vx))
            k = min(keys)
            out[by, bx] = (k[3], k[2])
    return out


@pytest.mark.parametrize("lam", [0, 4])
def test_single_level_equals_exhaustive_brute_force(lam):
    # small texture and flat patches create many near-ties; clamping is exercised by R beyond the border
    rng = np.random.default_rng(5)
    I = rng.integers(0, 6, (24, 40), dtype=np.uint8)
    J = rng.integers(0, 6, (24, 40), dtype=np.uint8)
    J[:, :8] = 3
    sp = SearchParams(levels=1, block=8, radius=5, refine=0, mv_cost=lam)
    vec, _ = M.block_search(I, J, sp)
    assert np.array_equal(vec.astype(np.int64), _brute_single_level(I, J, 8, 5, lam))


def test_tie_break_order_vy_then_vx():
    # J is periodic with period 6 in x; I equals J shifted by 3: vx = +3 and -3 tie exactly
    row = np.array([0, 50, 100, 150, 200, 250], np.uint8)
    J = np.tile(row, (16, 4))[:, :24]
    I = np.roll(J, 3, axis=1)
    sp = SearchParams(levels=1, block=8, radius=4, refine=0, mv_cost=0)
    vec, sad0 = M.block_search(I, J, sp)
    # interior block bx = 1: SAD 0 at vx = -3 and +3 (|v| equal, vy equal) -> smaller vx wins
    assert tuple(vec[0, 1]) == (-3, 0) and sad0[0, 1] == 0


def test_coarse_stage_equals_exhaustive_search_on_coarsest_level():
    """With no refinement (r = 0) the level-0 vector is 2^(L-1) times the
    exhaustive argmin on the coarsest pyramid level."""
    rng = np.random.default_rng(21)
    I = rng.integers(0, 256, (64, 96), dtype=np.uint8)
    J = np.roll(I, (3, -5), axis=(0, 1))
    J[::7] = 0
    for lam in (0, 4):
        vec, _ = M.block_search(I, J, SearchParams(levels=3, block=16, radius=6, refine=0, mv_cost=lam))
        coarse = _brute_single_level(M.pyramid(I, 3)[2], M.pyramid(J, 3)[2], 4, 6, lam)
        assert np.array_equal(vec.astype(np.int64), 4 * coarse)


def _brute_refine(I, J, parent, s, r, lam):
    h, w = I.shape
    pad = int(np.abs(parent).max()) * 2 + r + 1
    P = np.pad(J.astype(np.int64), pad, mode="edge")
    out = np.zeros_like(parent)
    for by in range(parent.shape[0]):
        for bx in range(parent.shape[1]):
            blk = I[by * s:(by + 1) * s, bx * s:(bx + 1) * s].astype(np.int64)
            keys = []
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    vx, vy = 2 * parent[by, bx, 0] + dx, 2 * parent[by, bx, 1] + dy
                    y0, x0 = by * s + vy + pad, bx * s + vx + pad
                    sad = int(np.abs(blk - P[y0:y0 + s, x0:x0 + s]).sum())
                    n1 = abs(vx) + abs(vy)
                    keys.append((sad + lam * n1, n1, vy, vx))
            k = min(keys)
            out[by, bx] = (k[3], k[2])
    return out


def test_refine_stage_equals_brute_force_around_twice_the_parent():
    rng = np.random.default_rng(22)
    I = rng.integers(0, 256, (48, 80), dtype=np.uint8)
    J = np.roll(I, (-2, 3), axis=(0, 1)) // 2 + rng.integers(0, 60, (48, 80), dtype=np.uint8)
    for lam in (0, 4):
        vec, _ = M.block_search(I, J, SearchParams(levels=2, block=16, radius=3, refine=2, mv_cost=lam))
        parent = _brute_single_level(M.pyramid(I, 2)[1], M.pyramid(J, 2)[1], 8, 3, lam)
        assert np.array_equal(vec.astype(np.int64), _brute_refine(I, J, parent, 16, 2, lam))


# ---- AMM -------------------------------------------------------------------------

def test_isqrt_matches_math_isqrt():
    rng = np.random.default_rng(7)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2 ** 32, 2 ** 40 - 1, 11552 << 32, 2 ** 61 + 12345]
    vals += [int(x) for x in rng.integers(0, 2 ** 62, 300, dtype=np.int64)]
    for v in vals:
        assert M.isqrt(v) == math.isqrt(v)


@pytest.mark.parametrize("sx,sy", [(0, 0), (3, 4), (-5, 12), (70, -70), (1, 1)])
def test_amm_of_uniform_field(sx, sy):
    vec = np.zeros((7, 9, 2), np.int16)
    vec[..., 0], vec[..., 1] = sx, sy
    q = math.isqrt((sx * sx + sy * sy) << 32)          # floor(sqrt(k) * 2^16)
    assert M.amm_sum(vec) == 63 * q
    if (sx, sy) == (3, 4):
        assert q == 5 * 65536
    r = {"si": 0, "sj": 0, "sii": 0, "sjj": 0, "sij": 0, "samm": 63 * q, "n": 10, "nb": 63, "sabs": 0}
    assert abs(M.finalise(r)["amm"] - math.hypot(sx, sy)) < 2.0 ** -16


# ---- warp + NCC + residual --------------------------------------------------------

def _np_warp(J, vec, block):
    h, w = J.shape
    nby, nbx = vec.shape[:2]
    ys, xs = np.mgrid[0:h, 0:w]
    bx = np.minimum(xs // block, nbx - 1)
    by = np.minimum(ys // block, nby - 1)
    vx, vy = vec[by, bx, 0].astype(np.int64), vec[by, bx, 1].astype(np.int64)
    return J[np.clip(ys + vy, 0, h - 1), np.clip(xs + vx, 0, w - 1)]


def test_warp_sums_match_numpy_with_ragged_border():
    rng = np.random.default_rng(9)
    h, w, block = 45, 70, 16                        # 2 x 4 blocks plus ragged strips
    I = rng.integers(0, 256, (h, w), dtype=np.uint8)
    J = rng.integers(0, 256, (h, w), dtype=np.uint8)
    vec = rng.integers(-20, 21, (h // block, w // block, 2)).astype(np.int16)
    s = M.warp_sums(I, J, vec, block)
    Wj = _np_warp(J, vec, block).astype(np.int64)
    Ii = I.astype(np.int64)
    assert s == [int(Ii.sum()), int(Wj.sum()), int((Ii * Ii).sum()), int((Wj * Wj).sum()),
                 int((Ii * Wj).sum()), int(np.abs(Ii - Wj).sum())]
    rec = {"si": s[0], "sj": s[1], "sii": s[2], "sjj": s[3], "sij": s[4], "sabs": s[5], "samm": 0,
           "n": h * w, "nb": 8}
    ncc = M.finalise(rec)["ncc"]
    assert abs(ncc - np.corrcoef(Ii.ravel(), Wj.ravel())[0, 1]) < 1e-12


def test_ncc_closed_forms():
    rng = np.random.default_rng(10)
    I = rng.integers(0, 100, (64, 80), dtype=np.uint8)
    zero = np.zeros((4, 5, 2), np.int16)

    def ncc(J):
        s = M.warp_sums(I, J, zero, 16)
        rec = dict(zip(("si", "sj", "sii", "sjj", "sij", "sabs"), s), samm=0, n=I.size, nb=20)
        return M.finalise(rec)

    assert ncc(I)["ncc"] == 1.0 and ncc(I)["swr"] == 0.0
    assert abs(ncc((2 * I.astype(np.int32) + 10).astype(np.uint8))["ncc"] - 1.0) < 1e-12
    neg = ncc((255 - I.astype(np.int32)).astype(np.uint8))
    assert abs(neg["ncc"] + 1.0) < 1e-12 and abs(neg["swr"] - 2.0) < 1e-12


def test_degenerate_variances():
    flat = np.full((32, 48), 9, np.uint8)
    other = np.full((32, 48), 200, np.uint8)
    tex = synth.random_frame(4, 48, 32)
    both = M.measure(M.FRAME, flat, other)
    assert both["ncc"] == 1.0 and both["act"] == 0.0      # two flat frames: NCC 1
    one = M.measure(M.FRAME, flat, tex)
    assert one["ncc"] == 0.0 and one["swr"] == 1.0


def test_identical_frames_measures():
    f = synth.Clip(synth.config_small()).frame(3)
    r = M.measure(M.FRAME, f, f)
    assert r["ncc"] == 1.0 and r["samm"] == 0 and r["act"] == 0.0 and r["sabs"] == 0
    assert r["si"] == int(f.astype(np.int64).sum())


def test_flash_offset_is_invisible_to_ncc_under_the_true_field():
    """NCC ignores a global offset (Sec. III.A, flashes): with the true (zero)
    field, a static pair differing only by +30 (no clipping) has NCC 1, SWR 0."""
    rng = np.random.default_rng(12)
    f = rng.integers(20, 200, (64, 96), dtype=np.uint8)
    g = (f.astype(np.int32) + 30).astype(np.uint8)
    s = M.warp_sums(f, g, np.zeros((4, 6, 2), np.int16), 16)
    r = M.finalise(dict(zip(("si", "sj", "sii", "sjj", "sij", "sabs"), s), samm=0, n=f.size, nb=24))
    assert r["ncc"] == pytest.approx(1.0, abs=1e-12) and r["act"] == 0.0 and s[5] == 30 * f.size


def test_field_kinds_pick_the_right_rows():
    rng = np.random.default_rng(13)
    a = rng.integers(0, 256, (64, 64), dtype=np.uint8)
    b = rng.integers(0, 256, (64, 64), dtype=np.uint8)
    I, J = M.pair_images(M.UPPER_LOWER, a, b)
    assert np.array_equal(I, a[0::2]) and np.array_equal(J, b[1::2])
    I, J = M.pair_images(M.LOWER_UPPER, a, b)
    assert np.array_equal(I, a[1::2]) and np.array_equal(J, b[0::2])
    I, J = M.pair_images(M.UPPER_UPPER, a, b)
    assert np.array_equal(I, a[0::2]) and np.array_equal(J, b[0::2])
    I, J = M.pair_images(M.LOWER_LOWER, a, b)
    assert np.array_equal(I, a[1::2]) and np.array_equal(J, b[1::2])


def test_same_parity_field_pair_of_a_repeated_field_is_static():
    # a frame whose lower field repeats the previous frame's lower field: the
    # lower-lower pair sees identical images (zero motion field, NCC 1, ACT 0)
    # and the upper-upper pair does not; a repeated field is the cue the
    # same-parity measure adds for 3:2 pulldown
    rng = np.random.default_rng(5)
    prev = rng.integers(0, 256, (96, 128), dtype=np.uint8)
    cur = rng.integers(0, 256, (96, 128), dtype=np.uint8)
    cur[1::2] = prev[1::2]
    m = M.measure(M.LOWER_LOWER, prev, cur)
    assert m["samm"] == 0 and m["ncc"] == 1.0 and m["act"] == 0.0
    assert M.measure(M.UPPER_UPPER, prev, cur)["act"] > 0.0


# ---- unary histogram measure --------------------------------------------------

@pytest.mark.parametrize("shape,seed", [((37, 53), 1), ((64, 64), 2), ((9, 10), 3)])
def test_frame_histogram_against_sorting_and_numpy(shape, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 256, shape, dtype=np.uint8)
    f[: shape[0] // 3] //= 7          # skewed content, a crowded low end
    h = M.frame_histogram(f)
    vals = np.sort(f.ravel().astype(np.int64))
    k = (vals.size - 1) // 2
    assert np.array_equal(h["bins"], np.histogram(f, bins=256, range=(0, 256))[0])
    assert h["median"] == vals[k]
    assert h["mad"] == np.sort(np.abs(vals - vals[k]))[k]
    assert h["mean"] == pytest.approx(f.mean(), abs=1e-12)
    assert h["std"] == pytest.approx(f.std(), abs=1e-12)


def test_frame_histogram_constant_frame():
    h = M.frame_histogram(np.full((16, 24), 77, np.uint8))
    assert h["bins"][77] == 16 * 24 and h["bins"].sum() == 16 * 24
    assert (h["mean"], h["std"], h["median"], h["mad"]) == (77.0, 0.0, 77, 0)
