"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests re-derives an expected value from the oracle itself: each
one checks the oracle against a closed form, a library routine (numpy, scipy),
finite differences of the oracle's own energy, a dense direct solve, or an
invariant that the method must keep. The paper prints no worked numeric
example; its printed numbers (Table 1, the 720K unknown count of Section 5)
live under tests/golden/.
"""

import os

import numpy as np
import pytest

import oracle as O
from paper_1610_07159_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- #
# printed numbers
# --------------------------------------------------------------------------- #

def test_table1_matches_golden():
    cols = {"fig2": 0, "fig568": 1, "fig79": 2}
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_parameters.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        rows[name] = [float(v) for v in vals]
    assert len(rows) == 10
    for preset, c in cols.items():
        for name, vals in rows.items():
            assert O.TABLE1[preset][name] == vals[c], (preset, name)
    p = O.Params()
    assert p.w_smooth == 1.0 and p.w_mag == 1.0
    assert p.eps == 1e-3 and p.eps_p == 0.2  # Eq. 12 and Section 4.1


def test_unknown_count_matches_section5():
    for line in open(os.path.join(GOLDEN, "counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w, h, s, n = (int(v) for v in line.split())
        nx, ny = O.grid_dims(w, h, s)
        assert 6 * nx * ny == n


# --------------------------------------------------------------------------- #
# pyramid, gradients, sampling, grid
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("h,w", [(8, 12), (7, 9), (1 + 2 * 5, 2 * 6)])
def test_downsample_is_edge_clamped_block_mean(h, w):
    rng = np.random.default_rng(0)
    img = rng.random((h, w))
    padded = np.pad(img, ((0, h % 2), (0, w % 2)), mode="edge")
    ref = padded.reshape(padded.shape[0] // 2, 2, padded.shape[1] // 2, 2).mean(axis=(1, 3))
    np.testing.assert_allclose(O.downsample(img), ref, rtol=0, atol=1e-15)


def test_gradients_central_differences():
    rng = np.random.default_rng(1)
    img = rng.random((9, 11))
    gx, gy = O.gradients(img)
    ref_gy, ref_gx = np.gradient(img)
    np.testing.assert_allclose(gx[:, 1:-1], ref_gx[:, 1:-1], atol=1e-15)
    np.testing.assert_allclose(gy[1:-1, :], ref_gy[1:-1, :], atol=1e-15)
    # clamp to edge: one-sided difference halved
    np.testing.assert_allclose(gx[:, 0], 0.5 * (img[:, 1] - img[:, 0]), atol=1e-15)
    np.testing.assert_allclose(gx[:, -1], 0.5 * (img[:, -1] - img[:, -2]), atol=1e-15)
    np.testing.assert_allclose(gy[0, :], 0.5 * (img[1, :] - img[0, :]), atol=1e-15)


def test_sample_matches_scipy_map_coordinates():
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(2)
    P = rng.random((13, 17))
    pts = np.column_stack([rng.uniform(-3, 20, 400), rng.uniform(-3, 16, 400)])
    for px, py in pts:
        v, _, _ = O.sample(P, px, py)
        ref = map_coordinates(P, [[np.clip(py, 0, 12)], [np.clip(px, 0, 16)]], order=1, mode="nearest")[0]
        assert abs(v - ref) < 1e-12


def test_sample_derivative_is_bilinear_derivative():
    rng = np.random.default_rng(3)
    P = rng.random((10, 10))
    h = 1e-7
    for px, py in rng.uniform(0.1, 8.9, size=(200, 2)):
        if min(abs(px - round(px)), abs(py - round(py))) < 1e-4:
            continue
        _, dx, dy = O.sample(P, px, py)
        fx = (O.sample(P, px + h, py)[0] - O.sample(P, px - h, py)[0]) / (2 * h)
        fy = (O.sample(P, px, py + h)[0] - O.sample(P, px, py - h)[0]) / (2 * h)
        assert abs(dx - fx) < 1e-7 and abs(dy - fy) < 1e-7
    # clamped axis: zero derivative
    assert O.sample(P, -2.0, 4.5)[1] == 0.0
    assert O.sample(P, 4.5, 12.0)[2] == 0.0


@pytest.mark.parametrize("w,h,s", [(20, 12, 4), (23, 13, 4), (17, 9, 8)])
def test_grid_weights_partition_of_unity_and_linear_reproduction(w, h, s):
    nx, ny = O.grid_dims(w, h, s)
    assert (nx - 1) * s <= w - 1 < nx * s
    for y in range(h):
        for x in range(w):
            nodes, wts = O.grid_weights(x, y, s, nx, ny)
            assert abs(wts.sum() - 1.0) < 1e-15 and (wts >= 0).all()
            ni, nj = nodes % nx, nodes // nx
            # node positions interpolate the pixel position (clamped past the last node)
            assert abs((wts * ni * s).sum() - min(x, (nx - 1) * s)) < 1e-12
            assert abs((wts * nj * s).sum() - min(y, (ny - 1) * s)) < 1e-12
            assert ni.max() - ni.min() == 1 and nj.max() - nj.min() == 1


# --------------------------------------------------------------------------- #
# consistency checks (Eqs. 1-6)
# --------------------------------------------------------------------------- #

def _ramp_planes(coefs, h=40, w=48):
    """Four linear ramp images a x + b y + c; bilinear sampling is exact on them."""
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    imgs = np.stack([a * xs + b * ys + c for a, b, c in coefs])
    return O.level_planes(imgs)


def test_pixel_terms_closed_form_on_ramps():
    rng = np.random.default_rng(4)
    coefs = [(0.011, -0.007, 0.3), (-0.004, 0.013, 0.5), (0.009, 0.002, 0.1), (0.003, -0.012, 0.7)]
    planes = _ramp_planes(coefs)
    I = [lambda X, Y, c=c: c[0] * X + c[1] * Y + c[2] for c in coefs]
    for _ in range(20):
        x, y = rng.uniform(15, 30), rng.uniform(15, 25)
        f = rng.uniform(-3, 3, 6)
        s, m, d = f[0:2], f[2:4], f[4:6]
        X = np.array([x, y])
        # Eqs. 1-6 as printed: I_1^0(x+s-m-d) - I_0^0(x-s-m+d), ...
        p00, p10 = X - s - m + d, X + s - m - d
        p01, p11 = X - s + m - d, X + s + m + d
        I00, I10, I01, I11 = I[0](*p00), I[1](*p10), I[2](*p01), I[3](*p11)
        expect = [I10 - I00, I11 - I01, I01 - I00, I11 - I10, I11 - I00, I01 - I10]
        out = O.pixel_terms(planes, x, y, f)
        np.testing.assert_allclose(out["e"], expect, atol=1e-12)
        # gradient constancy: the ramp gradients are constant inside the image
        grads = [np.array(c[:2]) for c in coefs]
        pairs = [(1, 0), (3, 2), (2, 0), (3, 1), (3, 0), (2, 1)]
        for k, (a, b) in enumerate(pairs):
            np.testing.assert_allclose(out["g"][k], grads[a] - grads[b], atol=1e-12)
        # d e_0 / d s_x = a_1 * (+1) - a_0 * (-1), d e_0 / d d_x = a_1 * (-1) - a_0 * (+1)
        assert abs(out["Je"][0, 0] - (coefs[1][0] + coefs[0][0])) < 1e-12
        assert abs(out["Je"][0, 4] - (-coefs[1][0] - coefs[0][0])) < 1e-12
        assert abs(out["Je"][2, 3] - (coefs[2][1] + coefs[0][1])) < 1e-12  # d e_2 / d m_y


def _noise_planes(w=36, h=28, seed=5):
    q = scenes.random_quadruple(w, h, seed)
    return O.level_planes(q.astype(np.float64))


def test_pixel_terms_jacobian_by_finite_differences():
    rng = np.random.default_rng(6)
    planes = _noise_planes()
    hstep = 1e-6
    checked = 0
    for _ in range(60):
        x, y = rng.integers(6, 30), rng.integers(6, 22)
        f = rng.uniform(-2.5, 2.5, 6)
        out = O.pixel_terms(planes, x, y, f)
        for u in range(6):
            fp, fm = f.copy(), f.copy()
            fp[u] += hstep
            fm[u] -= hstep
            op, om = O.pixel_terms(planes, x, y, fp), O.pixel_terms(planes, x, y, fm)
            fd_e = (op["e"] - om["e"]) / (2 * hstep)
            fd_g = (op["g"] - om["g"]).reshape(-1) / (2 * hstep)
            if np.max(np.abs(fd_e - out["Je"][:, u])) > 1e-6 or np.max(np.abs(fd_g - out["Jg"][:, u])) > 1e-6:
                # a bilinear kink within the step: allowed only if a position sits on a cell edge
                pos = _positions(x, y, f)
                assert np.min(np.abs(pos - np.round(pos))) < 1e-5
            else:
                checked += 1
    assert checked > 300


def _positions(x, y, f):
    s, m, d = f[0:2], f[2:4], f[4:6]
    X = np.array([x, y], dtype=np.float64)
    return np.stack([X - s - m + d, X + s - m - d, X - s + m - d, X + s + m + d])


# --------------------------------------------------------------------------- #
# energy and normal equations
# --------------------------------------------------------------------------- #

def _tiny_level(level=0, w=24, h=16, s=4, seed=7):
    planes = _noise_planes(w, h, seed)
    return O.Level(planes, s, level)


def _smooth_state(lv, rng, scale=1.5):
    G = lv.G
    base = rng.uniform(-scale, scale, (6, 1)) + 0.3 * rng.standard_normal((6, G))
    delta = 0.3 * rng.standard_normal((6, G))
    return base.reshape(-1), delta.reshape(-1)


def test_energy_terms_closed_forms():
    lv = _tiny_level()
    G = lv.G
    p = O.Params(w_epi=0.7)
    wf = np.full(G, 2.0)
    # constant totals: smoothness zero; magnitude = sum m_f |delta|^2
    base = np.repeat(np.array([-1.0, 0.25, 0.5, -0.5, 0.1, 0.2])[:, None], G, axis=1).reshape(-1)
    delta = np.zeros(6 * G)
    delta[:G] = 0.1  # a constant delta on s_x; totals = base + delta still constant
    _, terms, _ = O.energy(lv, base - delta, delta, wf, p)
    assert abs(terms[2]) < 1e-24
    assert abs(terms[4] - p.m_s * 0.01 * G) < 1e-12
    # rectified F: residuals (r_y - l_y) = 2 (s_y -+ d_y) at every node
    sy, dy = 0.25, 0.2
    assert abs(terms[3] - G * (4 * (sy - dy) ** 2 + 4 * (sy + dy) ** 2)) < 1e-10
    # a field linear in the node index: each horizontal edge differs by c
    c = 0.3
    ii = np.tile(np.arange(lv.nx), lv.ny).astype(np.float64)
    T = np.zeros((6, G))
    T[2] = c * ii  # m_x
    _, terms, _ = O.energy(lv, T.reshape(-1), np.zeros(6 * G), wf, p)
    n_h_edges = (lv.nx - 1) * lv.ny
    assert abs(terms[2] - n_h_edges * (2.0 + 2.0) * p.w_m * c * c) < 1e-10


def test_energy_data_terms_and_outlier_weight():
    lv = _tiny_level()
    rng = np.random.default_rng(8)
    base, delta = _smooth_state(lv, rng)
    p = O.Params(eps_p=0.25)
    wf = np.ones(lv.G)
    E, terms, W = O.energy(lv, base, delta, wf, p)
    T = (base + delta).reshape(6, lv.G)
    Ep = Eg = 0.0
    nW = 0
    for y in range(lv.h):
        for x in range(lv.w):
            nodes, wts = O.grid_weights(x, y, lv.s, lv.nx, lv.ny)
            f = (T[:, nodes] * wts).sum(axis=1)
            out = O.pixel_terms(lv.planes, x, y, f)
            ok = np.max(np.abs(out["e"])) < p.eps_p
            assert W[y, x] == ok
            nW += ok
            if ok:
                Ep += np.sqrt(out["e"] ** 2 + p.eps ** 2).sum()
                Eg += np.sqrt((out["g"] ** 2).sum(axis=1) + p.eps ** 2).sum()
    assert 0 < nW < lv.w * lv.h  # the threshold really excludes some pixels here
    assert abs(terms[0] - Ep) < 1e-9 and abs(terms[1] - Eg) < 1e-9


@pytest.mark.parametrize("level,robust,gradmode", [(0, O.IRLS, O.GRAD_BROX), (1, O.IRLS, O.GRAD_LITERAL),
                                                   (0, O.SQRT_PAPER, O.GRAD_BROX)])
def test_rhs_is_half_negative_gradient(level, robust, gradmode):
    """b = -grad(E)/2 with W and w_i frozen (Section 5.1: GN on the same energy)."""
    lv = _tiny_level(level=level)
    rng = np.random.default_rng(9 + level)
    base, delta = _smooth_state(lv, rng)
    F = (1e-6, -2e-5, 3e-4, 1e-5, 2e-6, -1.0, -2e-4, 1.0, 5e-3)  # general, nearly rectified
    p = O.Params(w_epi=0.5, F=F, eps_p=0.3, robust_mode=robust, grad_mode=gradmode)
    wf = 1.0 + rng.random(lv.G)
    A, b, E, W = O.assemble(lv, base, delta, wf, p)
    assert abs(E - O.energy(lv, base, delta, wf, p, W)[0]) < 1e-9
    hstep = 1e-6
    b = b.reshape(lv.G, 6)
    errs = []
    for n in range(lv.G):
        for u in range(6):
            dp, dm = delta.copy(), delta.copy()
            dp[u * lv.G + n] += hstep
            dm[u * lv.G + n] -= hstep
            g = (O.energy(lv, base, dp, wf, p, W)[0] - O.energy(lv, base, dm, wf, p, W)[0]) / (2 * hstep)
            errs.append(abs(b[n, u] + 0.5 * g) / (1.0 + abs(b[n, u])))
    errs = np.array(errs)
    # a handful of unknowns may straddle a bilinear kink; all others match to FD accuracy
    assert np.quantile(errs, 0.97) < 1e-5
    assert np.mean(errs < 1e-5) > 0.95


def test_system_matrix_is_the_weighted_gauss_newton_matrix():
    """v^T A v = sum_w omega (D_v r)^2 with D_v r from finite differences of the residuals."""
    lv = _tiny_level()
    rng = np.random.default_rng(10)
    base, delta = _smooth_state(lv, rng)
    # weak priors, so that the data term dominates the quadratic form
    p = O.Params(eps_p=0.3, w_epi=0.0, w_s=0.05, w_m=0.05, w_d=0.05, m_s=0.01, m_m=0.01, m_d=0.01)
    wf = 1.0 + rng.random(lv.G)
    A, b, E, W = O.assemble(lv, base, delta, wf, p)
    Ad = _dense(A, lv.nx, lv.ny)
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-12)
    G = lv.G
    hstep = 1e-6
    for trial in range(4):
        v = rng.standard_normal(6 * G)  # component-major like delta
        vi = v.reshape(6, G).T.reshape(-1)  # interleaved like A
        T0 = (base + delta).reshape(6, G)
        Tp = T0 + hstep * v.reshape(6, G)
        Tm = T0 - hstep * v.reshape(6, G)
        quad = 0.0
        for y in range(lv.h):
            for x in range(lv.w):
                if not W[y, x]:
                    continue
                nodes, wts = O.grid_weights(x, y, lv.s, lv.nx, lv.ny)
                f0 = (T0[:, nodes] * wts).sum(axis=1)
                o0 = O.pixel_terms(lv.planes, x, y, f0)
                op = O.pixel_terms(lv.planes, x, y, (Tp[:, nodes] * wts).sum(axis=1))
                om = O.pixel_terms(lv.planes, x, y, (Tm[:, nodes] * wts).sum(axis=1))
                De = (op["e"] - om["e"]) / (2 * hstep)
                Dg = (op["g"] - om["g"]) / (2 * hstep)
                # IRLS weights of the pseudo-Huber terms (Eq. 12)
                om_p = p.w_photo / (2 * np.sqrt(o0["e"] ** 2 + p.eps ** 2))
                om_g = p.w_grad / (2 * np.sqrt((o0["g"] ** 2).sum(axis=1) + p.eps ** 2))
                quad += (om_p * De ** 2).sum() + (om_g * (Dg ** 2).sum(axis=1)).sum()
        # smoothness (Eq. 14) and magnitude (Eq. 18) are quadratic: their GN rows are exact
        V = v.reshape(6, G)
        wfl = [p.w_s, p.w_s, p.w_m, p.w_m, p.w_d, p.w_d]
        mfl = [p.m_s, p.m_s, p.m_m, p.m_m, p.m_d, p.m_d]
        for j in range(lv.ny):
            for i in range(lv.nx):
                n = j * lv.nx + i
                for (i2, j2) in ((i + 1, j), (i, j + 1)):
                    if i2 < lv.nx and j2 < lv.ny:
                        m = j2 * lv.nx + i2
                        for u in range(6):
                            quad += p.w_reg * p.w_smooth * (wf[n] + wf[m]) * wfl[u] * (V[u, n] - V[u, m]) ** 2
                for u in range(6):
                    quad += p.w_reg * p.w_mag * mfl[u] * V[u, n] ** 2
        assert abs(vi @ Ad @ vi - quad) < 1e-5 * abs(quad)


def _dense(A, nx, ny):
    G = nx * ny
    D = np.zeros((6 * G, 6 * G))
    for j in range(ny):
        for i in range(nx):
            n = j * nx + i
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    i2, j2 = i + di, j + dj
                    if 0 <= i2 < nx and 0 <= j2 < ny:
                        m = j2 * nx + i2
                        D[6 * n:6 * n + 6, 6 * m:6 * m + 6] = A[n, 3 * (dj + 1) + (di + 1)]
    return D


def test_epipolar_rows_match_residual_derivatives_and_level_scaling():
    # level scaling of F: Frobenius norm kept, proportional to S F S
    F = np.array([0.1, -0.3, 0.2, 0.4, 0.05, -1.0, -0.2, 1.0, 0.3])
    for level in range(4):
        Fl = O.level_F(F, level)
        S = np.diag([2.0 ** level, 2.0 ** level, 1.0])
        SFS = S @ F.reshape(3, 3) @ S
        assert abs(np.linalg.norm(Fl) - np.linalg.norm(F)) < 1e-12
        np.testing.assert_allclose(Fl, SFS * np.linalg.norm(F) / np.linalg.norm(SFS), atol=1e-14)
    np.testing.assert_allclose(O.level_F(O.RECTIFIED_F, 3), np.array(O.RECTIFIED_F).reshape(3, 3), atol=1e-15)
    # only the epipolar prior: A = J^T J, b = -J^T r over the node residuals (Eqs. 15-17)
    lv = _tiny_level(level=1)
    rng = np.random.default_rng(11)
    base, delta = _smooth_state(lv, rng)
    p = O.Params(w_photo=0.0, w_grad=0.0, w_smooth=0.0, w_mag=0.0, w_epi=1.0, F=tuple(F), eps_p=0.0)
    wf = np.ones(lv.G)
    A, b, E, W = O.assemble(lv, base, delta, wf, p)
    Fl = O.level_F(F, 1)
    G = lv.G
    T = (base + delta).reshape(6, G)

    def resid(Tn, X, Y):
        s, m, d = Tn[0:2], Tn[2:4], Tn[4:6]
        P = np.array([X, Y])
        l0, r0 = np.append(P - s - m + d, 1), np.append(P + s - m - d, 1)
        l1, r1 = np.append(P - s + m - d, 1), np.append(P + s + m + d, 1)
        return np.array([l0 @ Fl @ r0, l1 @ Fl @ r1])

    Esum = 0.0
    for j in range(lv.ny):
        for i in range(lv.nx):
            n = j * lv.nx + i
            X, Y = i * lv.s, j * lv.s
            r = resid(T[:, n], X, Y)
            Esum += (r ** 2).sum()
            J = np.zeros((2, 6))
            for u in range(6):
                e = np.zeros(6)
                e[u] = 1e-6
                J[:, u] = (resid(T[:, n] + e, X, Y) - resid(T[:, n] - e, X, Y)) / 2e-6
            np.testing.assert_allclose(A[n, 4], J.T @ J, rtol=1e-6, atol=1e-6)
            np.testing.assert_allclose(b[n], -J.T @ r, rtol=1e-6, atol=1e-6)
    assert abs(E - Esum) < 1e-9 * max(1.0, Esum)


def test_pcg_matches_dense_cholesky_and_decreases_model():
    lv = _tiny_level()
    rng = np.random.default_rng(12)
    base, delta = _smooth_state(lv, rng)
    p = O.Params(eps_p=0.3)
    wf = 1.0 + rng.random(lv.G)
    A, b, _, _ = O.assemble(lv, base, delta, wf, p)
    Ad = _dense(A, lv.nx, lv.ny)
    L = np.linalg.cholesky(Ad)  # SPD: raises otherwise
    xd = np.linalg.solve(L.T, np.linalg.solve(L, b.reshape(-1)))
    # matrix-vector product of the block form
    v = rng.standard_normal(6 * lv.G)
    np.testing.assert_allclose(O.apply(lv.nx, lv.ny, A, v.reshape(lv.G, 6)).reshape(-1), Ad @ v, rtol=1e-12,
                               atol=1e-10)
    x, model, its = O.pcg(lv.nx, lv.ny, A, b, 3000)
    assert np.max(np.abs(x.reshape(-1) - xd)) < 1e-8 * max(1.0, np.max(np.abs(xd)))
    # Fig. 4: within one GN step the quadratic model only decreases
    x10, model10, its10 = O.pcg(lv.nx, lv.ny, A, b, 10)
    assert its10 == 10
    assert np.all(np.diff(model10) <= 1e-12 * np.abs(model10[:-1]))
    m_star = -0.5 * b.reshape(-1) @ xd
    assert model10[-1] >= m_star - 1e-9 * abs(m_star)


def test_pcg_iterate_is_the_preconditioned_krylov_minimiser():
    """Section 5.1 solves each step by Jacobi-preconditioned CG from x = 0. In
    exact arithmetic its k-th iterate is the point of the Krylov space
    span{M b, (M A) M b, ..., (M A)^(k-1) M b}, M = diag(A)^-1, closest to the
    solution in the A-norm. That optimality property fixes every iterate
    without any of CG's own recurrences: here it is formed with a dense
    orthonormal basis of the space and the projected system, and the oracle's
    iterates must match it for k = 1 .. 8 (a wrong preconditioner, step length
    or direction update gives other points of other spaces)."""
    lv = _tiny_level()
    rng = np.random.default_rng(21)
    base, delta = _smooth_state(lv, rng)
    A, b, _, _ = O.assemble(lv, base, delta, 1.0 + rng.random(lv.G), O.Params(eps_p=0.3))
    Ad = _dense(A, lv.nx, lv.ny)
    bv = b.reshape(-1)
    d = np.diag(Ad).copy()
    Minv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 1.0)
    K = [Minv * bv]
    for k in range(1, 9):
        V, _ = np.linalg.qr(np.stack(K, axis=1))
        y = np.linalg.solve(V.T @ Ad @ V, V.T @ bv)
        x_star = V @ y
        x, _, its = O.pcg(lv.nx, lv.ny, A, b, k)
        assert its == k
        np.testing.assert_allclose(x.reshape(-1), x_star, rtol=0, atol=1e-9 * np.max(np.abs(x_star)))
        K.append(Minv * (Ad @ K[-1]))


# --------------------------------------------------------------------------- #
# hierarchy and temporal transfer
# --------------------------------------------------------------------------- #

def _tiny_system(seed=13, w=40, h=28, s=4):
    lv = _tiny_level(w=w, h=h, s=s, seed=seed)
    rng = np.random.default_rng(seed)
    base, delta = _smooth_state(lv, rng)
    A, b, _, _ = O.assemble(lv, base, delta, 1.0 + rng.random(lv.G), O.Params(eps_p=0.3))
    return lv, A, b


def test_schwarz_with_one_subdomain_is_plain_pcg():
    """A single subdomain holding the whole grid, one sweep: the local solve
    is the global Jacobi-PCG from zero (Section 5.2 reduces to Section 5.1)."""
    lv, A, b = _tiny_system()
    for it in (1, 4, 12):
        x_pcg, _, _ = O.pcg(lv.nx, lv.ny, A, b, it)
        x_sw = O.schwarz(lv.nx, lv.ny, A, b, 1, it, tile=max(lv.nx, lv.ny), overlap=0)
        np.testing.assert_allclose(x_sw, x_pcg, rtol=0, atol=1e-13 * np.abs(x_pcg).max())


@pytest.mark.parametrize("tile,overlap", [(2, 0), (3, 1), (4, 2)])
def test_schwarz_with_exact_local_solves_is_restricted_additive_schwarz(tile, overlap):
    """With enough patch iterations the local PCG solves exactly, and each
    sweep is x <- x + sum_k R~_k^T A_k^-1 R_k (b - A x) with A_k the dense
    subdomain block (numpy.linalg.solve) and R~_k keeping the tile's own
    nodes: restricted additive Schwarz, written out here on the dense matrix."""
    lv, A, b = _tiny_system()
    nx, ny = lv.nx, lv.ny
    D = _dense(A, nx, ny)
    bb = b.reshape(-1)
    x = np.zeros_like(bb)
    sweeps = 3
    for _ in range(sweeps):
        r = bb - D @ x
        xn = x.copy()
        for tj in range(0, ny, tile):
            for ti in range(0, nx, tile):
                ext = [(i, j) for j in range(max(tj - overlap, 0), min(tj + tile + overlap, ny))
                       for i in range(max(ti - overlap, 0), min(ti + tile + overlap, nx))]
                idx = np.array([6 * (j * nx + i) + u for (i, j) in ext for u in range(6)])
                e = np.linalg.solve(D[np.ix_(idx, idx)], r[idx])
                for k, (i, j) in enumerate(ext):
                    if ti <= i < ti + tile and tj <= j < tj + tile:
                        n = j * nx + i
                        xn[6 * n:6 * n + 6] = x[6 * n:6 * n + 6] + e[6 * k:6 * k + 6]
        x = xn
    x_sw = O.schwarz(nx, ny, A, b, sweeps, 400, tile=tile, overlap=overlap).reshape(-1)
    np.testing.assert_allclose(x_sw, x, rtol=0, atol=1e-9 * np.abs(x).max())


def test_schwarz_sweeps_converge_to_the_dense_solution():
    lv, A, b = _tiny_system()
    D = _dense(A, lv.nx, lv.ny)
    x_star = np.linalg.solve(D, b.reshape(-1))
    errs = [np.abs(O.schwarz(lv.nx, lv.ny, A, b, k, 10, tile=3, overlap=1).reshape(-1) - x_star).max()
            for k in (1, 4, 16, 64)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-8 * np.abs(x_star).max()


def test_upsample_constant_and_linear_fields():
    nxc, nyc, nx, ny = 6, 5, 12, 9
    Tc = np.repeat(np.arange(1.0, 7.0)[:, None], nxc * nyc, axis=1)
    base = O.upsample(Tc.reshape(-1), nxc, nyc, nx, ny).reshape(6, ny, nx)
    for c in range(6):
        assert np.all(base[c] == 2.0 * (c + 1))
    ic = np.tile(np.arange(nxc), nyc).astype(np.float64)
    jc = np.repeat(np.arange(nyc), nxc).astype(np.float64)
    lin = np.stack([0.5 * ic - 0.25 * jc + 1.0] * 6)
    up = O.upsample(lin.reshape(-1), nxc, nyc, nx, ny).reshape(6, ny, nx)
    jj, ii = np.mgrid[0:ny, 0:nx]
    expect = 2.0 * (0.5 * ii / 2 - 0.25 * jj / 2 + 1.0)
    inner = (ii / 2 <= nxc - 1) & (jj / 2 <= nyc - 1)
    np.testing.assert_allclose(up[0][inner], expect[inner], atol=1e-13)


def test_temporal_transfer_closed_forms():
    s, nx, ny = 8, 10, 7
    G = nx * ny
    rng = np.random.default_rng(13)
    dprev = rng.standard_normal(6 * G)
    Tzero = np.zeros(6 * G)
    np.testing.assert_array_equal(O.temporal(s, nx, ny, dprev, Tzero, O.TEMPORAL_PROPAGATE), dprev)
    np.testing.assert_array_equal(O.temporal(s, nx, ny, dprev, Tzero + 5, O.TEMPORAL_COPY), dprev)
    assert not O.temporal(s, nx, ny, dprev, Tzero, O.TEMPORAL_ZERO).any()
    # linear delta in the node index, constant motion m: the node at X takes X - 2m
    ii = np.tile(np.arange(nx), ny).astype(np.float64)
    lin = np.stack([0.1 * ii + 0.5] * 6).reshape(-1)
    T = np.zeros((6, G))
    T[2] = -4.0  # m_x = -4 px: source at X + 8 px = one node to the right
    out = O.temporal(s, nx, ny, lin, T.reshape(-1)).reshape(6, ny, nx)
    np.testing.assert_allclose(out[0][:, :-1], (0.1 * (np.arange(nx - 1) + 1) + 0.5)[None, :].repeat(ny, 0),
                               atol=1e-14)


# --------------------------------------------------------------------------- #
# whole-frame closed forms and invariants
# --------------------------------------------------------------------------- #

def _weak_prior_params(**kw):
    d = dict(m_s=1e-6, m_m=1e-6, m_d=1e-6, gn_iters=(20,) * 8, pcg_iters=(50,) * 8)
    d.update(kw)
    return O.Params(**d)


def test_static_plane_gives_analytic_disparity():
    q = scenes.plane_quadruple(disparity=6, motion=(0, 0), sigma=0.0, seed=21)
    r = O.solve_frame(q, 4, 3, _weak_prior_params())
    F = r.fields(0)[:, 3:-3, 3:-3]
    assert np.max(np.abs(F[0] + 3.0)) < 1e-2  # s = (-disparity / 2, 0)
    for c in range(1, 6):
        assert np.max(np.abs(F[c])) < 1e-2


def test_rigid_translation_is_recovered():
    q = scenes.plane_quadruple(disparity=8, motion=(2, -1), sigma=0.0, seed=1)
    r = O.solve_frame(q, 4, 3, _weak_prior_params())
    F = r.fields(0)[:, 3:-3, 3:-3]
    expect = [-4.0, 0.0, 1.0, -0.5, 0.0, 0.0]  # s = (-8/2, 0), m = v/2, d = 0
    for c in range(6):
        assert np.max(np.abs(F[c] - expect[c])) < 1e-2, c


def test_stereo_only_keeps_motion_and_difference_zero():
    q = scenes.plane_quadruple(disparity=8, motion=(0, 0), sigma=0.01, seed=3)
    q[2], q[3] = q[0], q[1]  # the same pair at both time steps (Section 6.4)
    r = O.solve_frame(q, 4, 3, O.Params(gn_iters=(4,) * 8, pcg_iters=(10,) * 8))
    F = r.fields(0)
    assert np.max(np.abs(F[2:])) < 1e-9
    assert np.max(np.abs(F[0])) > 1.0


def test_identical_images_give_zero_fields():
    q = scenes.plane_quadruple(disparity=0, motion=(0, 0), sigma=0.0, seed=4)
    q[1:] = q[0]
    r = O.solve_frame(q, 4, 2, O.Params(gn_iters=(3,) * 8, pcg_iters=(10,) * 8))
    assert np.max(np.abs(r.total)) == 0.0


def test_energy_never_rises_within_a_step_and_across_steps_without_W():
    q = scenes.plane_quadruple()
    r = O.solve_frame(q, 4, 3, O.Params(gn_iters=(5,) * 8, pcg_iters=(10,) * 8))
    for l in range(3):
        for g in range(5):
            st = r.step(l, g)
            assert st[1] <= st[0]
    r2 = O.solve_frame(q, 4, 3, O.Params(eps_p=0.0, gn_iters=(5,) * 8, pcg_iters=(10,) * 8))
    for l in range(3):
        seq = [r2.step(l, g)[0] for g in range(5)] + [r2.step(l, 4)[1]]
        assert all(b <= a for a, b in zip(seq, seq[1:]))


def test_feature_weight_eigenvalue_step():
    """w_i from the smaller eigenvalue of the 3x3 structure tensor of the halfway image."""
    lv = _tiny_level(w=40, h=32, s=4)
    p = O.Params(wfeat_gain=9.0, wfeat_tau=1e-3)
    T = np.zeros(6 * lv.G)
    wf = O.feature_weights(lv, T, p).reshape(lv.ny, lv.nx)
    H = lv.planes[:, 0].mean(axis=0)  # zero fields: halfway image = mean of the four
    Hy, Hx = np.gradient(H)
    for j in range(1, lv.ny - 1):
        for i in range(1, lv.nx - 1):
            X, Y = i * lv.s, j * lv.s
            gx = Hx[Y - 1:Y + 2, X - 1:X + 2].reshape(-1)
            gy = Hy[Y - 1:Y + 2, X - 1:X + 2].reshape(-1)
            M = np.array([[gx @ gx, gx @ gy], [gx @ gy, gy @ gy]])
            lmin = max(np.linalg.eigvalsh(M)[0], 0.0)
            assert abs(wf[j, i] - (1.0 + 9.0 * np.exp(-lmin / 1e-3))) < 1e-9
    assert O.feature_weights(lv, T, O.Params(wfeat_mode=O.WFEAT_OFF)).max() == 1.0


def _pixel_fields_closed_form(T, s, nx, ny, w, h):
    """[6, h, w]: the bilinear interpolation of Eq. 7 written out (node (i, j)
    at pixel (i s, j s); pixels past the last node clamp to it)."""
    T = T.reshape(6, ny, nx)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    u, v = np.minimum(xs / s, nx - 1), np.minimum(ys / s, ny - 1)
    i0, j0 = np.minimum(np.floor(u).astype(int), nx - 2), np.minimum(np.floor(v).astype(int), ny - 2)
    a, b = u - i0, v - j0
    return ((1 - a) * (1 - b) * T[:, j0, i0] + a * (1 - b) * T[:, j0, i0 + 1]
            + (1 - a) * b * T[:, j0 + 1, i0] + a * b * T[:, j0 + 1, i0 + 1])


def test_halfway_image_closed_form_on_ramps_at_nonzero_fields():
    """H(x) = mean of the four images at the positions of Eqs. 1-6; on linear
    ramps a x + b y + c bilinear sampling is exact, so H has a closed form."""
    rng = np.random.default_rng(21)
    w, h, s = 48, 40, 4
    coefs = [(0.011, -0.007, 0.3), (-0.004, 0.013, 0.5), (0.009, 0.002, 0.1), (0.003, -0.012, 0.7)]
    lv = O.Level(_ramp_planes(coefs, h=h, w=w), s)
    T = rng.uniform(-2.5, 2.5, (6, lv.G))
    H = O.halfway_image(lv, T.reshape(-1))
    f = _pixel_fields_closed_form(T, s, lv.nx, lv.ny, w, h)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    S, M, D = f[0:2], f[2:4], f[4:6]
    X = np.stack([xs, ys])
    pos = [X - S - M + D, X + S - M - D, X - S + M - D, X + S + M + D]  # I_0^0, I_1^0, I_0^1, I_1^1
    expect = sum(a * p[0] + b * p[1] + c for (a, b, c), p in zip(coefs, pos)) / 4.0
    inside = np.all([(p[0] >= 0) & (p[0] <= w - 1) & (p[1] >= 0) & (p[1] <= h - 1) for p in pos], axis=0)
    assert inside.mean() > 0.6
    np.testing.assert_allclose(H[inside], expect[inside], atol=1e-12)


def test_halfway_image_and_feature_weight_at_integer_fields():
    """Integer s, m, d move every sample onto a pixel, so H is a mean of four
    shifted images (exact on any image) and w_i follows from its structure
    tensor in closed form (Section 4.3)."""
    lv = _tiny_level(w=56, h=44, s=4, seed=31)
    s, m, d = np.array([1.0, 0.0]), np.array([1.0, -1.0]), np.array([0.0, 1.0])
    T = np.repeat(np.concatenate([s, m, d])[:, None], lv.G, axis=1)
    H = O.halfway_image(lv, T.reshape(-1))
    offs = [-s - m + d, s - m - d, -s + m - d, s + m + d]  # Eqs. 1-6 for I_0^0, I_1^0, I_0^1, I_1^1
    r = int(max(np.abs(o).max() for o in offs))
    ref = np.zeros((lv.h - 2 * r, lv.w - 2 * r))
    for c, o in enumerate(offs):
        ox, oy = int(o[0]), int(o[1])
        ref += lv.planes[c, 0, r + oy:lv.h - r + oy, r + ox:lv.w - r + ox]
    ref /= 4.0
    np.testing.assert_allclose(H[r:lv.h - r, r:lv.w - r], ref, atol=1e-12)
    # structure tensor of the exact H over the 3x3 pixels at interior nodes
    Hy, Hx = np.gradient(H)
    lmins, nodes = [], []
    for j in range(lv.ny):
        for i in range(lv.nx):
            X, Y = i * lv.s, j * lv.s
            if X - 2 < r or Y - 2 < r or X + 2 > lv.w - 1 - r or Y + 2 > lv.h - 1 - r:
                continue
            gx = Hx[Y - 1:Y + 2, X - 1:X + 2].reshape(-1)
            gy = Hy[Y - 1:Y + 2, X - 1:X + 2].reshape(-1)
            Mst = np.array([[gx @ gx, gx @ gy], [gx @ gy, gy @ gy]])
            lmins.append(max(np.linalg.eigvalsh(Mst)[0], 0.0))
            nodes.append(j * lv.nx + i)
    assert len(nodes) >= 40
    tau = float(np.median(lmins))  # so that exp(-lambda/tau) spreads over (0, 1)
    wf = O.feature_weights(lv, T.reshape(-1), O.Params(wfeat_gain=9.0, wfeat_tau=tau))
    expect = 1.0 + 9.0 * np.exp(-np.array(lmins) / tau)
    assert np.ptp(expect) > 1.0
    np.testing.assert_allclose(wf[nodes], expect, atol=1e-9)


def test_sqrt_paper_system_matrix_is_the_gauss_newton_matrix_of_the_square_roots():
    """Paper-literal linearisation (Section 5: one residual per pixel and term,
    M = 2N + 14G): each pixel contributes the residuals sqrt(rho_photo) and
    sqrt(rho_grad), rho the weighted sums of the six penalties, so
    v^T A v = sum_px (D_v sqrt(rho_photo))^2 + (D_v sqrt(rho_grad))^2 + priors,
    with D_v the directional derivative, here by central differences."""
    lv = _tiny_level()
    rng = np.random.default_rng(12)
    base, delta = _smooth_state(lv, rng)
    p = O.Params(eps_p=0.3, w_epi=0.0, w_s=0.05, w_m=0.05, w_d=0.05, m_s=0.01, m_m=0.01, m_d=0.01,
                 robust_mode=O.SQRT_PAPER)
    wf = 1.0 + rng.random(lv.G)
    A, b, E, W = O.assemble(lv, base, delta, wf, p)
    Ad = _dense(A, lv.nx, lv.ny)
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-12)
    G = lv.G
    hstep = 1e-6

    def roots(out):
        rp = p.w_photo * np.sqrt(out["e"] ** 2 + p.eps ** 2).sum()
        rg = p.w_grad * np.sqrt((out["g"] ** 2).sum(axis=1) + p.eps ** 2).sum()
        return np.sqrt(rp), np.sqrt(rg)

    for trial in range(3):
        v = rng.standard_normal(6 * G)
        vi = v.reshape(6, G).T.reshape(-1)
        T0 = (base + delta).reshape(6, G)
        Tp, Tm = T0 + hstep * v.reshape(6, G), T0 - hstep * v.reshape(6, G)
        quad = 0.0
        for y in range(lv.h):
            for x in range(lv.w):
                if not W[y, x]:
                    continue
                nodes, wts = O.grid_weights(x, y, lv.s, lv.nx, lv.ny)
                rp_p, rg_p = roots(O.pixel_terms(lv.planes, x, y, (Tp[:, nodes] * wts).sum(axis=1)))
                rp_m, rg_m = roots(O.pixel_terms(lv.planes, x, y, (Tm[:, nodes] * wts).sum(axis=1)))
                quad += ((rp_p - rp_m) / (2 * hstep)) ** 2 + ((rg_p - rg_m) / (2 * hstep)) ** 2
        V = v.reshape(6, G)
        wfl = [p.w_s, p.w_s, p.w_m, p.w_m, p.w_d, p.w_d]
        mfl = [p.m_s, p.m_s, p.m_m, p.m_m, p.m_d, p.m_d]
        for j in range(lv.ny):
            for i in range(lv.nx):
                n = j * lv.nx + i
                for (i2, j2) in ((i + 1, j), (i, j + 1)):
                    if i2 < lv.nx and j2 < lv.ny:
                        mm = j2 * lv.nx + i2
                        for u in range(6):
                            quad += p.w_reg * p.w_smooth * (wf[n] + wf[mm]) * wfl[u] * (V[u, n] - V[u, mm]) ** 2
                for u in range(6):
                    quad += p.w_reg * p.w_mag * mfl[u] * V[u, n] ** 2
        assert abs(vi @ Ad @ vi - quad) < 1e-5 * abs(quad)


def test_backtracking_safeguard_is_exercised_and_keeps_energy_monotone():
    """The paper-literal square-root linearisation overshoots here; the safeguard halves t."""
    q = scenes.random_quadruple(48, 40, 1, sigma=0.01)
    p = O.Params(gn_iters=(6,) * 8, pcg_iters=(30,) * 8, m_s=1e-4, m_m=1e-4, m_d=1e-4, w_s=0.1, w_m=0.1,
                 w_d=0.1, robust_mode=O.SQRT_PAPER)
    r = O.solve_frame(q, 4, 1, p)
    steps = [r.step(0, g) for g in range(6)]
    assert any(0.0 < st[2] < 1.0 for st in steps)
    for st in steps:
        assert st[1] <= st[0]
        assert st[2] in (0.0, 1.0, 0.5, 0.25, 0.125, 0.0625)


def test_backtracking_takes_the_first_halving_that_does_not_raise_the_energy():
    """C18: a step takes the first t of 1, 1/2, 1/4, 1/8, 1/16 with E(delta + t x; W) <= E(delta; W), with
    W taken at the step's linearisation point. On the overshooting scene above, each step is rebuilt from the state
    the solve reached before it (a solve with fewer steps), its energies at those t are evaluated, and the t (and
    accepted energy) the solve recorded must be the first that passes."""
    q = scenes.random_quadruple(48, 40, 1, sigma=0.01)
    kw = dict(pcg_iters=(30,) * 8, m_s=1e-4, m_m=1e-4, m_d=1e-4, w_s=0.1, w_m=0.1, w_d=0.1,
              robust_mode=O.SQRT_PAPER)
    lv = O.Level(O.level_planes(O.pyramid(q, 1)[0]), 4, 0)
    p = O.Params(gn_iters=(6,) * 8, **kw)
    base = np.zeros(6 * lv.G)
    wf = O.feature_weights(lv, base, p)
    full = O.solve_frame(q, 4, 1, p)
    checked = 0
    for g in range(6):
        st = full.step(0, g)
        if not 0.0 < st[2] < 1.0:
            continue
        delta = (O.solve_frame(q, 4, 1, O.Params(gn_iters=(g,) * 8, **kw)).deltas(0).reshape(-1) if g else
                 np.zeros(6 * lv.G))
        A, b, E0, W = O.assemble(lv, base, delta, wf, p)
        assert abs(E0 - st[0]) <= 1e-12 * abs(E0)
        x, _, _ = O.pcg(lv.nx, lv.ny, A, b, 30)
        x = x.T.reshape(-1)  # [G, 6] -> component-major like delta
        t_first, e_first = 0.0, E0
        for t in (1.0, 0.5, 0.25, 0.125, 0.0625):
            Et, _, _ = O.energy(lv, base, delta + t * x, wf, p, W)
            if Et <= E0:
                t_first, e_first = t, Et
                break
        assert st[2] == t_first and abs(st[1] - e_first) <= 1e-12 * abs(e_first), (g, st[:3], t_first)
        checked += 1
    assert checked > 0
