"""The stereo-only workload of the paper's 12 MP experiments (Section 6: a
still stereo pair, used at both times) at 4288x2848 on the GPU.

A crop of the 12 MP pair is compared with the oracle field by field (W and the
bilinear cell decisions replayed: disparities reach ~100 px); the full-size
pair, which no CPU solve finishes in test time, is checked by the property
the method fixes at any size: with identical times the energy is even in the
motion and difference flows, so m = d = 0 up to FP32 rounding, while the
stereo flow follows the scene's disparities."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1610_07159_gb300 import scenes, scenes_device, sf
from tests.gpu_common import make_params

pytestmark = pytest.mark.gpu

W12, H12 = 4288, 2848
SCHED = dict(solver=O.SOLVER_SCHWARZ, patch_iters=[6], schwarz_tile=7, schwarz_overlap=1)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


def _pair_12mp():
    video = scenes.SceneVideo(W12, H12, 1, seed=700, disparity=(30.0, 200.0), max_motion=0.0)
    return scenes_device.stereo_pair_quadruple(video, "cuda")


def test_stereo_only_crop_parity():
    q = _pair_12mp()[:, 1024:1024 + 712, 1600:1600 + 1072].contiguous()
    sp, op = make_params([3], [6], preset="fig79", record_cells=1, **SCHED)
    s = sf.Solver(1072, 712, 8, 5, sp)
    fields = s.solve(q).cpu().numpy()
    st = s.stats()
    assert st.status == sf.OK
    ref = O.solve_frame(q.cpu().numpy().astype(np.float64), 8, 5, op, W_given=s.wmasks(),
                        cells_given=s.cell_records())
    err = np.max(np.abs(fields - ref.fields(0)), axis=(1, 2))
    e_rel = abs(st.energy - ref.energy) / abs(ref.energy)
    print(f"\n12 MP crop 1072x712: max-abs px {np.array2string(err, precision=2)}, energy rel {e_rel:.2e}")
    assert np.all(err <= 1e-3) and e_rel <= 1e-4, (err, e_rel)
    assert np.max(np.abs(fields[2:])) <= 1e-3  # m = d = 0 on the crop too


def test_stereo_only_12mp_full_size():
    q = _pair_12mp()
    sp, _ = make_params([3], [6], preset="fig79", **SCHED)
    s = sf.Solver(W12, H12, 8, 7, sp)
    fields = s.solve(q)
    torch.cuda.synchronize()
    st = s.stats()
    assert st.status == sf.OK and np.isfinite(st.energy)
    f = fields.cpu().numpy()
    assert np.all(np.isfinite(f))
    md = float(np.max(np.abs(f[2:])))
    sx = -2.0 * f[0]  # disparity of each node (s_x = -disparity / 2)
    print(f"\n12 MP pair: |m|, |d| <= {md:.2e} px; disparity range {np.percentile(sx, 1):.1f} .. "
          f"{np.percentile(sx, 99):.1f} px (scene 30 .. 200); energy {st.energy:.6g}")
    assert md <= 1e-3
    assert 20.0 <= np.percentile(sx, 50) <= 210.0
