"""Pins of the oracle's per-level maps of Algorithm 1 (Section 5.3).

Occlusion maps: the triangulated warp grid rendered into the four views with a
z-buffer of closeness (reading C25) against closed forms on a fronto-parallel
plane and on a square occluder in front of a plane; their prolongation against
a bilinear interpolation written out. Illumination correction maps (reading
C26): the Gaussian low-pass against scipy.ndimage, the stereo residual and the
correction against a quadruple whose right images carry a known offset."""

import numpy as np
import pytest

import oracle as O
from paper_1610_07159_gb300 import scenes


def _const_fields(G, s, m, d):
    return np.repeat(np.array([s[0], s[1], m[0], m[1], d[0], d[1]], dtype=np.float64)[:, None], G, axis=1)


def _in_image(x, y, offs, w, h):
    ok = np.ones_like(x, dtype=bool)
    for ox, oy in offs:
        qx, qy = np.floor(x + ox + 0.5), np.floor(y + oy + 0.5)
        ok &= (qx >= 0) & (qx <= w - 1) & (qy >= 0) & (qy <= h - 1)
    return ok


def test_occlusion_of_a_fronto_parallel_plane_is_only_the_image_border():
    """Constant fields: nothing occludes anything; a pixel is invisible only
    when one of its four sample positions (Eqs. 1-6) leaves the image."""
    w, h, st = 64, 48, 4
    nx, ny = O.grid_dims(w, h, st)
    s, m, d = (-3.25, 0.0), (1.25, -0.5), (0.25, 0.75)
    T = _const_fields(nx * ny, s, m, d)
    V = O.occlusion_map(w, h, st, T.reshape(-1))
    S, M, D = np.array(s), np.array(m), np.array(d)
    offs = [-S - M + D, S - M - D, -S + M - D, S + M + D]
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    expect = _in_image(xs, ys, offs, w, h)
    assert 0.5 < expect.mean() < 1.0
    assert np.array_equal(V.astype(bool), expect)


def test_occlusion_of_a_square_occluder_is_the_exact_strips_beside_it():
    """A foreground square (nodes 8..15 x 4..11, disparity 23) in front of a
    background plane (disparity 4), no motion: in the left images the square
    hides the background strip right of it that its extra disparity covers
    (Delta/2 = 9.5 px), in the right images the strip left of it. On the rows
    where the square is foreground from top to bottom, every pixel outside the
    two transition cells has a closed-form visibility."""
    w, h, st = 96, 64, 4
    nx, ny = O.grid_dims(w, h, st)
    db, dfg = 4.0, 23.0
    disp = np.full((ny, nx), db)
    disp[4:12, 8:16] = dfg
    T = np.zeros((6, ny, nx))
    T[0] = -disp / 2.0  # s_x = -disparity / 2 (reading C4)
    V = O.occlusion_map(w, h, st, T.reshape(-1))
    half = (dfg - db) / 2.0
    fg_lo, fg_hi = 8 * st, 15 * st  # foreground pixels 32..60
    for y in range(18, 43):
        for x in range(w):
            if fg_lo - st < x < fg_lo or fg_hi < x < fg_hi + st:
                continue  # transition cells: the surface ramps between the two depths
            if fg_lo <= x <= fg_hi:
                expect = True  # the square is nearest everywhere it projects
            else:
                in_img = 2 <= x <= w - 1 - 2  # background samples at x -+ 2
                hidden_left = fg_hi + st <= x < fg_hi + half   # left images: behind the square
                hidden_right = fg_lo - half < x <= fg_lo - st  # right images
                expect = in_img and not hidden_left and not hidden_right
            assert bool(V[y, x]) == expect, (x, y)
    assert V[30, 64:70].sum() == 0 and V[30, 23:29].sum() == 0 and V[30, 70] == 1 and V[30, 22] == 1


def test_occlusion_closeness_tolerance():
    """A point is hidden only when the nearer surface's closeness exceeds its
    own by more than tau: the square of the previous test is 19 px of
    disparity nearer than the background it hides."""
    w, h, st = 96, 64, 4
    nx, ny = O.grid_dims(w, h, st)
    disp = np.full((ny, nx), 4.0)
    disp[4:12, 8:16] = 23.0
    T = np.zeros((6, ny, nx))
    T[0] = -disp / 2.0
    for tau, hidden in ((0.5, True), (18.9, True), (19.1, False)):
        V = O.occlusion_map(w, h, st, T.reshape(-1), tau=tau)
        assert (V[30, 66] == 0) == hidden and (V[30, 25] == 0) == hidden, tau


def test_visibility_prolongation_is_a_thresholded_bilinear_interpolation():
    rng = np.random.default_rng(3)
    Oc = (rng.random((9, 13)) < 0.7).astype(np.uint8)
    w, h = 25, 17
    V = O.vis_upsample(Oc, w, h)
    from scipy.ndimage import map_coordinates
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    interp = map_coordinates(Oc.astype(np.float64), [ys / 2.0, xs / 2.0], order=1, mode="nearest")
    assert np.array_equal(V.astype(bool), interp >= 0.5)
    one = np.ones((8, 10), np.uint8)
    one[3, 4] = 0
    V1 = O.vis_upsample(one, 20, 16)
    assert V1.sum() == 20 * 16 - 1 and V1[6, 8] == 0  # only the fine pixel on the coarse one


@pytest.mark.parametrize("sigma", [3.2, 1.5])
def test_gaussian_low_pass_matches_scipy(sigma):
    """Normalised Gaussian truncated at ceil(3 sigma), edges clamped: scipy's
    gaussian_filter with mode 'nearest' and the same radius."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(4)
    img = rng.random((29, 37))
    R = int(np.ceil(3 * sigma))
    ref = gaussian_filter(img, sigma, mode="nearest", truncate=(R + 0.25) / sigma)
    assert int((R + 0.25) / sigma * sigma + 0.5) == R
    np.testing.assert_allclose(O.gauss_blur(img, sigma), ref, atol=1e-13)
    np.testing.assert_allclose(O.gauss_blur(np.full((20, 30), 0.37), sigma), 0.37, atol=1e-15)


def test_illumination_prolongation_is_a_box_filter():
    Rc = np.arange(2 * 5 * 7, dtype=np.float64).reshape(2, 5, 7)
    L = O.illum_upsample(Rc, 13, 10)
    for t in range(2):
        for y in range(10):
            for x in range(13):
                assert L[t, y, x] == Rc[t, min(y // 2, 4), min(x // 2, 6)]


def _plane_truth(q_shape, st):
    # plane_quadruple: disparity 8, motion (2, -1) -> s = (-4, 0), m = (1, -0.5), d = 0 (reading C4)
    h, w = q_shape[-2:]
    nx, ny = O.grid_dims(w, h, st)
    return _const_fields(nx * ny, (-4.0, 0.0), (1.0, -0.5), (0.0, 0.0)).reshape(-1)


def test_stereo_residual_is_the_right_camera_offset_and_the_correction_removes_it():
    """Exact integer-shift rendering: at the true fields the data residual is
    zero; adding a constant c to both right images makes the stereo residual
    c at every interior pixel (Section 5.3), and with the correction map L = c
    the energy equals the unmodified quadruple's."""
    q = scenes.plane_quadruple(sigma=0.0)
    st = 4
    T = _plane_truth(q.shape, st)
    c = 0.05
    q2 = q.astype(np.float64).copy()
    q2[1] += c
    q2[3] += c
    lv = O.Level(O.level_planes(q.astype(np.float64)), st)
    lv2 = O.Level(O.level_planes(q2), st)
    r = O.illum_residual(lv2, T)
    inner = (slice(8, lv.h - 8), slice(12, lv.w - 12))
    np.testing.assert_allclose(r[0][inner], c, atol=1e-12)
    np.testing.assert_allclose(r[1][inner], c, atol=1e-12)
    wf = np.ones(lv.G)
    p = O.Params(eps_p=0.0)
    zero = np.zeros_like(T)
    E0, t0, _ = O.energy(lv, T, zero, wf, p)
    Lmap = np.full((2, lv.h, lv.w), c)
    E1, t1, _ = O.energy_maps(lv2, T, zero, wf, p, Lmap=Lmap)
    E2, _, _ = O.energy(lv2, T, zero, wf, p)
    assert abs(E1 - E0) < 1e-9 * E0 and E2 > E0 * 1.5


def test_occlusion_map_removes_pixels_from_the_data_terms():
    lv = O.Level(O.level_planes(scenes.random_quadruple(40, 32, 2).astype(np.float64)), 4)
    rng = np.random.default_rng(5)
    T = 0.3 * rng.standard_normal(6 * lv.G)
    wf = np.ones(lv.G)
    p = O.Params(eps_p=0.0)
    V = (rng.random((lv.h, lv.w)) < 0.6).astype(np.uint8)
    _, terms_v, _ = O.energy_maps(lv, T, np.zeros_like(T), wf, p, V=V)
    # the same sums over the visible pixels alone
    Tm = T.reshape(6, lv.G)
    Ep = Eg = 0.0
    for y in range(lv.h):
        for x in range(lv.w):
            if not V[y, x]:
                continue
            nodes, wts = O.grid_weights(x, y, lv.s, lv.nx, lv.ny)
            out = O.pixel_terms(lv.planes, x, y, (Tm[:, nodes] * wts).sum(axis=1))
            Ep += np.sqrt(out["e"] ** 2 + p.eps ** 2).sum()
            Eg += np.sqrt((out["g"] ** 2).sum(axis=1) + p.eps ** 2).sum()
    assert abs(terms_v[0] - Ep) < 1e-9 and abs(terms_v[1] - Eg) < 1e-9
    # the system with the maps is the Gauss-Newton system of that energy: b = -grad(E)/2
    A, b, E, W = O.assemble_maps(lv, T, np.zeros_like(T), wf, p, V=V)
    hstep = 1e-6
    b = b.reshape(lv.G, 6)
    for n in (3, lv.G // 2, lv.G - 5):
        for u in range(6):
            dp, dm = np.zeros_like(T), np.zeros_like(T)
            dp[u * lv.G + n] += hstep
            dm[u * lv.G + n] -= hstep
            g = (O.energy_maps(lv, T, dp, wf, p, V=V, W=W)[0] - O.energy_maps(lv, T, dm, wf, p, V=V, W=W)[0]) / (
                2 * hstep)
            assert abs(b[n, u] + 0.5 * g) < 1e-5 * (1 + abs(b[n, u]))


def test_frames_with_maps_keep_the_energy_monotone_and_the_correction_helps():
    """With both maps on, the energy never rises within a step; with the right
    images brighter by a smooth field the correction brings the fields nearer
    the true ones than the uncorrected solve."""
    q = scenes.plane_quadruple(sigma=0.005)
    h, w = q.shape[-2:]
    ys, xs = np.mgrid[0:h, 0:w]
    shade = 0.08 + 0.04 * np.sin(2 * np.pi * xs / w)
    q2 = q.astype(np.float64).copy()
    q2[1] += shade
    q2[3] += shade
    # light priors, so that the data terms decide the fields
    base = dict(gn_iters=(6,) * 8, pcg_iters=(30,) * 8, eps_p=0.0, w_reg=0.1)
    r_on = O.solve_frame(q2, 4, 3, O.Params(occlusion=1, illumination=1, **base))
    r_off = O.solve_frame(q2, 4, 3, O.Params(**base))
    for l in range(3):
        for g in range(6):
            st_ = r_on.step(l, g)
            assert st_[1] <= st_[0]
    truth = np.array([-4.0, 0.0, 1.0, -0.5, 0.0, 0.0])[:, None, None]
    err_on = np.abs(r_on.fields(0) - truth)[:, 3:-3, 3:-3].mean()
    err_off = np.abs(r_off.fields(0) - truth)[:, 3:-3, 3:-3].mean()
    assert err_on < 0.7 * err_off, (err_on, err_off)
    assert r_on.energy < 0.5 * r_off.energy
