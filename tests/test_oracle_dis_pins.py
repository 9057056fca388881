"""Pins of the dense sub-pixel flow oracle (oracle/dis.py) against what the
method and the mathematics fix, not against the oracle itself:
- on a linear intensity ramp (rank-one H) a Gauss-Newton step moves the flow
  along the gradient by the closed-form factor lambda / (lambda + d) and not at
  all across it; on a bilinear image (full-rank H, and central differences and
  bilinear sampling exact) the steps converge to the true sub-pixel shift;
- identical frames give zero flow everywhere;
- densification of hand-set patch flows equals the hand-computed weighted means;
- patch origins cover every pixel, the last patch flush with the border;
- a smooth image moved by a sub-pixel shift is recovered coarse to fine within
  the error a bilinear model of 8-bit data allows."""
import numpy as np
import pytest

from oracle import dis as D


def _ramp(h, w, a, b, c, sx=0.0, sy=0.0):
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    return a * (xx - sx) + b * (yy - sy) + c


def test_patch_origins_cover_every_pixel():
    assert D.patch_origins(20, 8, 4) == [0, 4, 8, 12]
    assert D.patch_origins(21, 8, 4) == [0, 4, 8, 12, 13]
    assert D.patch_origins(8, 8, 4) == [0]
    with pytest.raises(ValueError):
        D.patch_origins(7, 8, 4)
    for n in range(8, 40):
        cov = np.zeros(n, int)
        for o in D.patch_origins(n, 8, 4):
            cov[o:o + 8] += 1
        assert cov.min() >= 1


def test_central_differences_and_bilinear_are_exact_on_a_ramp():
    I = _ramp(20, 30, 1.5, -0.75, 100.0)
    gx, gy = D.gradients(I)
    assert np.allclose(gx[:, 1:-1], 1.5) and np.allclose(gy[1:-1, :], -0.75)
    assert np.allclose(gx[:, 0], 0.75) and np.allclose(gx[:, -1], 0.75)   # clamped neighbour: half the slope
    x, y = np.array([3.25, 10.5, 17.875]), np.array([4.5, 9.125, 2.0])
    assert np.allclose(D.bilinear(I, x, y), 1.5 * x - 0.75 * y + 100.0)
    assert D.bilinear(I, -3.0, -2.0) == I[0, 0]                          # clamp-to-edge


def test_gauss_newton_on_a_linear_ramp_recovers_the_gradient_component():
    # J(x) = I(x - s) with I linear: the residual is g.(u - s) with g constant,
    # H = 64 g g^T has rank one (the aperture problem), and a step from u
    # moves u by (H + dI)^-1 H (s - u): along g by the factor lam / (lam + d),
    # lam = 64 |g|^2, and not at all across g
    h, w, s = 40, 48, np.array([0.3, -1.7])
    g = np.array([2.0, 1.0])
    I = _ramp(h, w, *g, 60.0)
    J = _ramp(h, w, *g, 60.0, *s)
    oy, ox, _, _ = D.patch_grid(h, w, 8, 4)
    inner = (ox >= 8) & (ox <= w - 16) & (oy >= 8) & (oy <= h - 16)
    lam = 64.0 * g @ g
    proj = (s @ g) / (g @ g)                   # the component of s along g, in units of g
    for damp_rel, damp_abs, iters in ((0.0, 1.0, 1), (0.01, 1.0, 1), (0.01, 1.0, 8)):
        dp = D.DisParams(levels=1, iters=iters, damp_rel=damp_rel, damp_abs=damp_abs)
        u = D.inverse_search(I, J, np.zeros((len(oy), 2)), dp)[inner]
        d = damp_rel * lam + damp_abs
        along = proj * (1.0 - (d / (lam + d)) ** iters)
        assert np.allclose(u, along * g, atol=1e-9), (damp_rel, iters)


def test_gauss_newton_converges_to_the_shift_of_a_bilinear_image():
    # f = a + b x + c y + e x y: bilinear sampling and central differences are
    # exact, H has full rank (the gradient (b + e y, c + e x) varies over a
    # patch), and u = s is the fixed point (zero residual).  Without damping the
    # steps converge quadratically (from a start 1.4 px away: 0.08, 3e-4, then rounding)
    h, w, s = 64, 64, np.array([0.6, -0.4])
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)

    def f(sx, sy):
        X, Y = xx - sx, yy - sy
        return 50.0 + 0.5 * X + 0.3 * Y + 0.2 * X * Y

    oy, ox, _, _ = D.patch_grid(h, w, 8, 4)
    inner = (ox >= 8) & (ox <= w - 16) & (oy >= 8) & (oy <= h - 16)
    for start in ((0.0, 0.0), (-1.0, 1.0)):
        init = np.tile(start, (len(oy), 1))
        err = [np.abs(D.inverse_search(f(0, 0), f(*s), init, D.DisParams(levels=1, iters=k, damp_rel=0.0,
                                                                         damp_abs=1e-6))[inner] - s).max()
               for k in (1, 2, 4)]
        assert err[0] < 0.1 and err[1] < 1e-3 and err[1] < 0.1 * err[0] and err[2] < 1e-9, err
    # with the default damping the fixed point is the same: started on it, it stays
    u = D.inverse_search(f(0, 0), f(*s), np.tile(s, (len(oy), 1)), D.DisParams(levels=1))
    assert np.allclose(u[inner], s, atol=1e-12)


def test_identical_frames_give_zero_flow():
    rng = np.random.default_rng(3)
    f = rng.integers(0, 256, (45, 70), dtype=np.uint8)
    assert np.array_equal(D.dis_flow(f, f), np.zeros((45, 70, 2)))


def test_densification_by_hand():
    # two 8x8 patches overlapping in columns 4..7 of a 8x12 image (stride 4)
    h, w = 8, 12
    I = np.full((h, w), 50.0)
    dp = D.DisParams(levels=1)
    flows = np.array([[1.0, 0.0], [3.0, 2.0]])
    # J == I: every weight is 1 -> plain means where the patches overlap
    U = D.densify(I, I.copy(), flows, dp)
    assert np.allclose(U[:, :4], [1.0, 0.0]) and np.allclose(U[:, 8:], [3.0, 2.0])
    assert np.allclose(U[:, 4:8], [2.0, 1.0])
    # J = I + 6 at the second patch's sampled positions, I + 2 elsewhere: weights 1/6 and 1/2
    J = np.full((h, w), 52.0)
    J[:, 7:] = 56.0          # sampled by the second patch at columns >= 4 + 3 = 7
    U = D.densify(I, J, flows, dp)
    # a pixel x in 4..7: patch 0 samples J at x + 1, patch 1 at x + 3 (both clamped to 11)
    for x in range(4, 8):
        e0 = J[0, min(x + 1, 11)] - 50.0
        e1 = J[0, min(x + 3, 11)] - 50.0
        w0, w1 = 1.0 / max(1.0, abs(e0)), 1.0 / max(1.0, abs(e1))
        assert np.allclose(U[0, x], (w0 * flows[0] + w1 * flows[1]) / (w0 + w1))


def test_smooth_image_subpixel_shift_is_recovered():
    h, w = 96, 160
    yy, xx = np.mgrid[0:h, 0:w].astype(float)

    def img(sx, sy):
        X, Y = xx - sx, yy - sy
        v = 128 + 50 * np.sin(X / 7.0) + 40 * np.cos(Y / 9.0) + 20 * np.sin((X + Y) / 5.0)
        return np.clip(np.rint(v), 0, 255).astype(np.uint8)

    for s in ((2.5, -1.25), (-5.75, 3.0), (0.0, 0.0)):
        U = D.dis_flow(img(0, 0), img(*s))
        c = U[16:-16, 16:-16]
        assert abs(c[..., 0].mean() - s[0]) < 0.02 and abs(c[..., 1].mean() - s[1]) < 0.02
        assert np.abs(c[..., 0] - s[0]).max() < 0.3 and np.abs(c[..., 1] - s[1]).max() < 0.3


def test_flow_measure_reduces_to_plain_correlation_without_flow():
    # no step: the flow is exactly zero, Jw = J, AMM = 0 and NCC is the plain
    # correlation of the two frames (numpy's corrcoef)
    rng = np.random.default_rng(11)
    a = rng.integers(0, 256, (48, 64)).astype(np.uint8)
    b = np.clip(a.astype(int) // 2 + rng.integers(0, 40, a.shape), 0, 255).astype(np.uint8)
    m = D.flow_measure(a, b, D.DisParams(iters=0))
    assert m["amm"] == 0.0 and m["act"] == 0.0
    assert abs(m["ncc"] - np.corrcoef(a.ravel().astype(float), b.ravel().astype(float))[0, 1]) < 1e-12
    assert abs(m["swr"] - (1.0 - m["ncc"])) < 1e-15
    inv = (255 - a.astype(int)).astype(np.uint8)
    m = D.flow_measure(a, inv, D.DisParams(iters=0))
    assert abs(m["ncc"] + 1.0) < 1e-12 and abs(m["swr"] - 2.0) < 1e-12
    flat = np.full_like(a, 7)
    assert D.flow_measure(flat, flat, D.DisParams(iters=0))["ncc"] == 1.0
    assert D.flow_measure(a, flat, D.DisParams(iters=0))["ncc"] == 0.0


def test_flow_measure_of_identical_frames_and_of_a_shift():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 256, (40, 56)).astype(np.uint8)
    m = D.flow_measure(a, a)
    assert m["amm"] == 0.0 and m["ncc"] == 1.0 and m["act"] == 0.0
    h, w = 96, 160
    yy, xx = np.mgrid[0:h, 0:w].astype(float)

    def img(sx, sy):
        X, Y = xx - sx, yy - sy
        v = 128 + 50 * np.sin(X / 7.0) + 40 * np.cos(Y / 9.0) + 20 * np.sin((X + Y) / 5.0)
        return np.clip(np.rint(v), 0, 255).astype(np.uint8)

    m = D.flow_measure(img(0, 0), img(2.5, -1.25))
    assert abs(m["amm"] - np.hypot(2.5, 1.25)) < 0.05      # mean |U| near the true |s| (borders included)
    assert m["ncc"] > 0.99                                  # the warped frame matches
