"""The Schwarz domain decomposition (Section 5.2) on the GPU against the oracle.

Step level: the same assembled system solved by the CUDA kernel (one CTA per
subdomain, local PCG in shared memory, sweeps at a grid barrier) and by the
oracle's sfo_schwarz, element by element. Frame level: whole frames solved with
SF_SOLVER_SCHWARZ against the oracle with the same solver, W replayed, at the
bars of the plain path (1e-3 px, 1e-4 relative energy)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1610_07159_gb300 import scenes, sf
from tests.gpu_common import lib_blocks_to_oracle, make_params, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _system(w, h, s_, L, level, seed=5, **kw):
    q = scenes.random_quadruple(w, h, seed, sigma=0.01)
    sp, op = make_params([1], [1], solver=O.SOLVER_SCHWARZ, **kw)
    solver = sf.Solver(w, h, s_, L, sp)
    planes = solver.probe_pyramid(_dev(q), level).cpu().numpy().astype(np.float64)
    lv = O.Level(planes, s_, level)
    rng = np.random.default_rng(3)
    G = lv.G
    base = (rng.uniform(-1, 1, (6, 1)) + 0.2 * rng.standard_normal((6, G))).astype(np.float32)
    delta = (0.2 * rng.standard_normal((6, G))).astype(np.float32)
    blocks, rhs, _, _ = solver.probe_assemble(level, _dev(base), _dev(delta), _dev(np.ones(G, np.float32)))
    A = lib_blocks_to_oracle(blocks.cpu().numpy().astype(np.float64), lv.nx, lv.ny)
    return solver, lv, A, rhs.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("w,h,s_,tile,overlap,sweeps,patch", [
    (160, 120, 4, 8, 1, 5, 5),     # 40x30 nodes, 5x4 subdomains of up to 10x10
    (150, 110, 4, 8, 1, 3, 7),     # 38x28 nodes: ragged last tiles
    (160, 120, 4, 4, 2, 4, 5),     # 8x8 extended subdomains, 10x8 tiles
    (640, 480, 8, 8, 1, 5, 5),     # level 0 of the webcam frame, 80 subdomains
    (96, 64, 8, 16, 0, 2, 30),     # one subdomain: plain PCG on the whole level
])
def test_schwarz_parity_on_the_same_system(w, h, s_, tile, overlap, sweeps, patch):
    solver, lv, A, b = _system(w, h, s_, 3, 0, schwarz_tile=tile, schwarz_overlap=overlap)
    x_gpu = solver.probe_schwarz(0, sweeps, patch).cpu().numpy().astype(np.float64)
    x_ref = O.schwarz(lv.nx, lv.ny, A, b, sweeps, patch, tile=tile, overlap=overlap)
    err = rel_max(x_gpu, x_ref)
    print(f"\nschwarz {w}x{h} s{s_} tile {tile}+{overlap}: {sweeps} sweeps x {patch}: rel max err {err:.2e}")
    # FP32 local iterations against FP64: the same bound per iteration as the global PCG's parity test
    assert err < 2e-4 * sweeps * patch


def test_schwarz_with_more_subdomains_than_resident_ctas():
    """Tiles of one node with one node of overlap at 1280x720, stride 4
    (57 600 subdomains of up to 3x3 nodes; a level the global PCG plan cannot
    hold in one launch): the CTAs of the cooperative launch loop over several
    subdomains each and restage their blocks every time."""
    solver, lv, A, b = _system(1280, 720, 4, 2, 0, schwarz_tile=1, schwarz_overlap=1)
    x_gpu = solver.probe_schwarz(0, 3, 4).cpu().numpy().astype(np.float64)
    x_ref = O.schwarz(lv.nx, lv.ny, A, b, 3, 4, tile=1, overlap=1)
    assert rel_max(x_gpu, x_ref) < 2e-4 * 12


def _frame(q, s_, L, gn, sweeps, patch, tile=8, overlap=1, preset="fig2"):
    sp, op = make_params(gn, sweeps, preset=preset, solver=O.SOLVER_SCHWARZ, patch_iters=patch,
                         schwarz_tile=tile, schwarz_overlap=overlap)
    h, w = q.shape[-2:]
    solver = sf.Solver(w, h, s_, L, sp)
    fields = solver.solve(_dev(q)).cpu().numpy()
    st = solver.stats()
    assert st.status == sf.OK
    ref = O.solve_frame(q.astype(np.float64), s_, L, op, W_given=solver.wmasks())
    return fields, st, ref, op


@pytest.mark.parametrize("q_fn,s_,L,tile,overlap", [
    (lambda: scenes.plane_quadruple(), 4, 3, 8, 1),
    (lambda: scenes.SceneVideo(150, 110, 1, seed=11, disparity=(2, 12), max_motion=4).frames(1)[0], 4, 3, 4, 2),
    (lambda: scenes.SceneVideo(640, 480, 1, seed=100).frames(1)[0], 8, 4, 8, 1),
])
def test_schwarz_frame_parity(q_fn, s_, L, tile, overlap):
    """Whole frames with the paper's schedule shape (5 sweeps x 5 patch
    iterations per Gauss-Newton step) against the oracle with the same solver."""
    q = q_fn()
    fields, st, ref, op = _frame(q, s_, L, [3], [5], [5], tile, overlap)
    err = np.max(np.abs(fields - ref.fields(0)), axis=(1, 2))
    e_rel = abs(st.energy - ref.energy) / abs(ref.energy)
    print(f"\nschwarz frame {q.shape[-1]}x{q.shape[-2]}: max-abs px {np.array2string(err, precision=2)}, "
          f"energy rel {e_rel:.2e}")
    assert np.all(err <= 1e-3) and e_rel <= 1e-4, (err, e_rel)
    for l in range(L):
        for g in range(op.gn_iters[l]):
            st_l = ref.step(l, g)
            assert st.step_t[l][g] == st_l[2], (l, g)
