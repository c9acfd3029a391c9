"""Batched solve (sf_batch_*): many sequences of uneven sizes, one launch per
frame step, one thread-block cluster per sequence, against the FP64 oracle.

Each sequence of a batch must match the oracle run on that sequence alone
(fields within 1e-3 px max-abs, energy within 1e-4 relative, with the
kernel's outlier masks W replayed as in the single-sequence tests), whatever
the schedule (CTAs per sequence, cells per assembly pass)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1610_07159_gb300 import scenes, sf
from tests.gpu_common import make_params

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-3
ENERGY_TOL = 1e-4
W_MARGIN = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


def _videos(sizes, frames, seed0=500, **kw):
    return [scenes.SceneVideo(w, h, frames, seed=seed0 + i, **kw).frames(frames) for i, (w, h) in enumerate(sizes)]


def _check_sequence(view, F, q, s_, L, op, prev):
    st = view.stats()
    assert st.status == sf.OK
    ref = O.solve_frame(q.astype(np.float64), s_, L, op, prev=prev, W_given=view.wmasks())
    for l in range(L):
        npx = np.prod(O.level_dims(q.shape[-1], q.shape[-2], l))
        for g in range(op.gn_iters[l]):
            ndis, margin = ref.step(l, g)[5], ref.step(l, g)[6]
            assert ndis <= max(2, 1e-3 * npx) and margin <= W_MARGIN, (l, g, ndis, margin)
    err = np.max(np.abs(F - ref.fields(0)), axis=(1, 2))
    assert np.all(err <= FIELD_TOL), err
    assert abs(st.energy - ref.energy) <= ENERGY_TOL * abs(ref.energy), (st.energy, ref.energy)
    return ref


SMALL = [(160, 120), (150, 110), (96, 80), (200, 90)]
SMALL_L = [3, 3, 2, 3]


@pytest.mark.parametrize("schedule", [(8, 1), (2, 1), (4, 2), (16, 1)])
def test_batch_matches_oracle_per_sequence_over_frames(schedule):
    """Four uneven sequences, two frames (temporal transfer), stride 4."""
    sp, op = make_params([3], [10], preset="fig568")
    b = sf.Batch(SMALL, SMALL_L, 4, sp)
    b.set_schedule(*schedule)
    assert b.schedule() == schedule
    vids = _videos(SMALL, 2, disparity=(2, 12), max_motion=4)
    prev = [None] * len(SMALL)
    out = torch.empty(b.out_total, device="cuda", dtype=torch.float32)
    for f in range(2):
        packed = b.pack([torch.from_numpy(v[f]) for v in vids])
        b.solve(packed, out)
        torch.cuda.synchronize()
        fields = [t.cpu().numpy() for t in b.unpack(out)]
        for i in range(len(SMALL)):
            prev[i] = _check_sequence(b.sequence(i), fields[i], vids[i][f], 4, SMALL_L[i], op, prev[i])
            assert b.sequence(i).stats().frames == f + 1


def test_batch_equals_single_sequence_solver():
    """The batched and the per-level kernels solve the same problem; their
    fields agree to FP32 reduction-order differences."""
    sp, _ = make_params([3], [10])
    b = sf.Batch(SMALL[:2], SMALL_L[:2], 4, sp)
    vids = _videos(SMALL[:2], 1)
    out = b.solve(b.pack([torch.from_numpy(v[0]) for v in vids]))
    got = [t.cpu().numpy() for t in b.unpack(out)]
    for i, (w, h) in enumerate(SMALL[:2]):
        s = sf.Solver(w, h, 4, SMALL_L[i], make_params([3], [10])[0])
        ref = s.solve(torch.from_numpy(vids[i][0]).cuda()).cpu().numpy()
        assert np.max(np.abs(got[i] - ref)) <= 5e-4


def test_batch_tune_picks_and_caches_a_schedule():
    sp, _ = make_params([2], [8])
    sizes, levels = [(128, 96), (96, 64), (160, 120)], [3, 2, 3]
    b = sf.Batch(sizes, levels, 4, sp)
    packed = b.pack([torch.from_numpy(v[0]) for v in _videos(sizes, 1)])
    out = torch.empty(b.out_total, device="cuda", dtype=torch.float32)
    ms = b.tune(packed, out, steps=2)
    assert ms > 0
    sched = b.schedule()
    assert sched[0] in (2, 4, 8, 16) and sched[1] in (1, 2)
    # every sequence is back at frame 0, and solving works after tuning
    b.solve(packed, out)
    assert all(b.sequence(i).stats().frames == 1 for i in range(3))
    # a second batch of the same shape takes the cached schedule
    b2 = sf.Batch(sizes, levels, 4, sp)
    assert b2.tune(packed, out, steps=2) == pytest.approx(ms)
    assert b2.schedule() == sched
    with pytest.raises(sf.SFError):
        b.tune(packed, out)  # not at frame 0 any more


def test_batch_rejects_bad_arguments():
    sp, _ = make_params([3], [10])
    with pytest.raises(sf.SFError):
        sf.Batch([(160, 120)], [3], 4, make_params([3], [10], precision=sf.MIXED_FP16)[0])
    with pytest.raises(sf.SFError):
        sf.Batch([(3, 3)], [3], 4, sp)
    b = sf.Batch([(160, 120)], [3], 4, sp)
    with pytest.raises(sf.SFError):
        b.set_schedule(3, 1)
    with pytest.raises(sf.SFError):
        b.set_schedule(8, 5)


def test_batched_uneven_mix_at_scale_sampled_against_the_oracle():
    """64 sequences drawn uniformly from {320x240, 640x480, 960x540, 1280x720},
    stride 8, 4-5 levels, 3 GN x 20 PCG, one frame step. The oracle checks the
    smallest and one 640x480 sequence in full; every sequence must report a
    finite energy that no accepted step raised."""
    rng = np.random.default_rng(4000)
    choices = [(320, 240, 4), (640, 480, 4), (960, 540, 5), (1280, 720, 5)]
    pick = rng.integers(0, 4, 64)
    sizes = [choices[k][:2] for k in pick]
    levels = [choices[k][2] for k in pick]
    sp, op = make_params([3], [20])
    b = sf.Batch(sizes, levels, 8, sp)
    vids = [scenes.SceneVideo(w, h, 1, seed=700 + i).frames(1)[0] for i, (w, h) in enumerate(sizes)]
    out = b.solve(b.pack([torch.from_numpy(v) for v in vids]))
    torch.cuda.synchronize()
    fields = [t.cpu().numpy() for t in b.unpack(out)]
    for i in range(64):
        st = b.sequence(i).stats()
        assert st.status == sf.OK and np.isfinite(st.energy)
        for l in range(levels[i]):
            for g in range(3):
                assert st.step_accepted[l][g] <= st.step_energy[l][g]
    small = int(np.argmin([w * h for w, h in sizes]))
    mid = next(i for i in range(64) if sizes[i] == (640, 480))
    for i in (small, mid):
        _check_sequence(b.sequence(i), fields[i], vids[i], 8, levels[i], op, None)
