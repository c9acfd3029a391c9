"""Mixed precision against the FP64 oracle.

In the mixed modes the image pyramid (intensity and gradient planes, Section
5.3) is stored in FP16 or BF16, so every bilinear sample that feeds the
residuals and the analytic Jacobian (Section 5.1) reads 16-bit texels; the
residuals, robust weights, Jacobian products and all accumulation stay FP32.
The error of every output field against the FP64 oracle is reported (run with
-s to see the table) and bounded here."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1610_07159_gb300 import scenes, sf
from tests.gpu_common import make_params

pytestmark = pytest.mark.gpu

FIELDS = ("s_x", "s_y", "m_x", "m_y", "d_x", "d_y")
# unit roundoff of the texel formats (significand bits p: u = 2^-p)
UNIT_ROUNDOFF = {sf.FP32: 2.0 ** -24, sf.MIXED_FP16: 2.0 ** -11, sf.MIXED_BF16: 2.0 ** -8}
NAMES = {sf.FP32: "fp32", sf.MIXED_FP16: "fp16", sf.MIXED_BF16: "bf16"}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("prec", [sf.MIXED_FP16, sf.MIXED_BF16])
@pytest.mark.parametrize("w,h,L", [(160, 120, 3), (157, 93, 4)])
def test_pyramid_16bit_within_rounding(prec, w, h, L):
    """Level l is the 2x2 box of level l-1's rounded intensities, rounded
    again; so the intensity carries at most (l+1) roundings of relative size
    u, and a gradient (half the difference of two box values, rounded) at
    most l roundings of its inputs plus its own: both within (l+1) u M, M the
    largest intensity magnitude."""
    q = scenes.random_quadruple(w, h, 3, sigma=0.01)
    sp, _ = make_params([1], [1], precision=prec)
    s = sf.Solver(w, h, 2, L, sp)
    ref = O.pyramid(q.astype(np.float64), L)
    u = UNIT_ROUNDOFF[prec]
    M = float(np.max(np.abs(q)))
    for l in range(L):
        planes = s.probe_pyramid(_dev(q), l).cpu().numpy().astype(np.float64)
        err = np.abs(planes - O.level_planes(ref[l]))
        bound = (l + 1) * u * M
        assert err.max() <= bound, (l, err.max(), bound)
        # 16-bit storage really is in effect: the error is far above FP32 rounding
        assert err.max() > 16 * UNIT_ROUNDOFF[sf.FP32], (l, err.max())


CELL_MARGIN = 1e-3  # px: a replayed cell decision may part from the FP64 one only this close to a cell edge


def _frame_errors(q, s_, L, gn, pcg, prec, preset, replay_cells=False):
    sp, op = make_params(gn, pcg, preset=preset, precision=prec, record_cells=int(replay_cells))
    h, w = q.shape[-2:]
    solver = sf.Solver(w, h, s_, L, sp)
    F = solver.solve(_dev(q)).cpu().numpy()
    st = solver.stats()
    assert st.status == sf.OK
    # the oracle replays the kernel's outlier decisions W (an integer decision
    # taken in the kernel's precision), and with replay_cells its bilinear cell
    # decisions at cell edges, so the comparison measures the continuous error
    # of the fields
    cells = solver.cell_records() if replay_cells else None
    ref = O.solve_frame(q.astype(np.float64), s_, L, op, W_given=solver.wmasks(), cells_given=cells)
    if replay_cells:
        for l in range(L):
            for g in range(op.gn_iters[l]):
                ndis, margin = ref.step(l, g)[7], ref.step(l, g)[8]
                assert margin <= CELL_MARGIN, (l, g, ndis, margin)
    err = np.abs(F - ref.fields(0))
    e_rel = abs(st.energy - ref.energy) / abs(ref.energy)
    return err, e_rel


def _report(tag, prec, err, e_rel):
    mx = err.max(axis=(1, 2))
    frac = float(np.mean(err.max(axis=0) > 1e-3))
    print("\n%s %s max-abs px: %s | energy rel %.2e | nodes > 1e-3 px: %.2e" % (
        tag, NAMES[prec], " ".join("%s %.2e" % (n, v) for n, v in zip(FIELDS, mx)), e_rel, frac))
    return mx, frac


# error budget of the 16-bit modes, stated for both workloads: a texel
# rounding of u M moves a sample by about u M / |grad I| px, which the solve
# averages over the pixels of a cell
MIXED_FIELD_TOL = {sf.MIXED_FP16: 0.25, sf.MIXED_BF16: 0.5}   # px, max-abs per field
MIXED_ENERGY_TOL = {sf.MIXED_FP16: 1e-3, sf.MIXED_BF16: 1e-3}  # relative


@pytest.mark.parametrize("prec", [sf.FP32, sf.MIXED_FP16, sf.MIXED_BF16])
def test_webcam_frame_per_field_error(prec):
    """640x480 frame of the webcam-like video (stride 8, 4 levels, 3 GN x 20 PCG)."""
    q = scenes.SceneVideo(640, 480, 1, seed=100).frames(1)[0]
    err, e_rel = _frame_errors(q, 8, 4, [3], [20], prec, "fig2")
    mx, _ = _report("640x480", prec, err, e_rel)
    if prec == sf.FP32:
        assert np.all(mx <= 1e-3) and e_rel <= 1e-4, (mx, e_rel)
    else:
        assert np.all(mx <= MIXED_FIELD_TOL[prec]) and e_rel <= MIXED_ENERGY_TOL[prec], (mx, e_rel)


@pytest.mark.parametrize("prec", [sf.FP32, sf.MIXED_FP16, sf.MIXED_BF16])
def test_high_resolution_frame_per_field_error(prec):
    """1920x1080 frame of the high-resolution video (disparities up to 96 px,
    motion up to 40 px; stride 16, 6 levels, 3 GN x 20 PCG, Figure 5/6/8
    weights). The bilinear cell of a sample is a second integer decision taken
    in floating point (reading C7), and the analytic Jacobian of the bilinear
    interpolant (Section 5.1) jumps between cells; with offsets of ~70 px a
    sample can lie within FP32 rounding of a cell edge. In FP32 the oracle
    therefore replays the kernel's cell decisions for samples within 1e-3 px
    of a cell edge (like W), and every replayed decision that differs from the
    oracle's own must sit within that distance of the edge. Then every node
    is within 1e-3 px."""
    q = scenes.SceneVideo(1920, 1080, 1, seed=300, disparity=(15.0, 96.0), max_motion=40.0).frames(1)[0]
    err, e_rel = _frame_errors(q, 16, 6, [3], [20], prec, "fig568", replay_cells=prec == sf.FP32)
    mx, frac = _report("1920x1080", prec, err, e_rel)
    if prec == sf.FP32:
        assert np.all(mx <= 1e-3) and e_rel <= 1e-4, (mx, e_rel)
    else:
        assert np.all(mx <= MIXED_FIELD_TOL[prec]) and e_rel <= MIXED_ENERGY_TOL[prec], (mx, e_rel)


def test_recording_cells_changes_nothing():
    """The recording variant of the assembly (a test aid) computes the same
    frame as the solve path, bit for bit."""
    q = scenes.SceneVideo(640, 480, 1, seed=100).frames(1)[0]
    out = []
    for rec in (0, 1):
        sp, _ = make_params([3], [20], record_cells=rec)
        s = sf.Solver(640, 480, 8, 4, sp)
        out.append((s.solve(_dev(q)).cpu().numpy(), s.stats().energy))
        if rec:
            cells = s.cell_records()
            assert sum(len(c) for per in cells for c in per) > 0
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
