"""The oracle's replay of integer decisions taken elsewhere (test infrastructure).

The parity tests let the oracle take the CUDA path's outlier masks W and its
bilinear cell decisions at cell edges (both integer decisions taken in
floating point). These tests pin the replay itself: replaying the oracle's
own decisions changes nothing, and a replayed decision that differs is used,
counted and measured."""

import numpy as np

import oracle as O
from paper_1610_07159_gb300 import scenes


def _records(w, h, cell_of_x):
    """Decisions for every sample of every pixel at integer positions (zero
    fields): x axis cell cell_of_x(x), y axis cell min(y, h-2), none clamped."""
    ys, xs = np.mgrid[0:h, 0:w]
    pix = (ys * w + xs).reshape(-1).astype(np.uint32)
    recs = []
    for img in range(4):
        cx = cell_of_x(xs).reshape(-1).astype(np.uint32)
        cy = np.minimum(ys, h - 2).reshape(-1).astype(np.uint32)
        recs.append(np.stack([pix, (cx << 4) | (img << 1) | 0], axis=1))
        recs.append(np.stack([pix, (cy << 4) | (img << 1) | 1], axis=1))
    return np.concatenate(recs).astype(np.uint32)


def test_replaying_the_oracles_own_cell_decisions_changes_nothing():
    q = scenes.random_quadruple(32, 24, 3, sigma=0.01)
    p = O.Params(gn_iters=(2,) * 8, pcg_iters=(8,) * 8)
    w, h = 32, 24
    own = _records(w, h, lambda x: np.minimum(x, w - 2))
    r0 = O.solve_frame(q, 4, 1, p)
    r1 = O.solve_frame(q, 4, 1, p, cells_given=[[own, np.zeros((0, 2), np.uint32)]])
    assert np.array_equal(r0.total, r1.total) and r0.energy == r1.energy
    assert r1.step(0, 0)[7] == 0 and r1.step(0, 0)[8] == 0.0


def test_a_differing_cell_decision_is_used_counted_and_measured():
    """At zero fields every sample sits on a pixel; taking the left cell
    (fraction 1) instead of the right one (fraction 0) keeps the values and
    changes the x derivatives, so the first step's system and result change,
    and every replayed x decision counts as differing at distance 0."""
    q = scenes.random_quadruple(32, 24, 3, sigma=0.01)
    p = O.Params(gn_iters=(1,) * 8, pcg_iters=(8,) * 8)
    w, h = 32, 24
    left = _records(w, h, lambda x: np.maximum(np.minimum(x, w - 2) - (x < w - 1), 0))
    r0 = O.solve_frame(q, 4, 1, p)
    r1 = O.solve_frame(q, 4, 1, p, cells_given=[[left]])
    n_differ = 4 * h * (w - 2)  # x = 1 .. w-2 move to the left cell; x = 0 and x = w-1 keep theirs
    assert r1.step(0, 0)[7] == n_differ and r1.step(0, 0)[8] == 0.0
    # same values at the linearisation point, a different step
    assert r1.step(0, 0)[0] == r0.step(0, 0)[0]
    assert not np.array_equal(r0.total, r1.total)
