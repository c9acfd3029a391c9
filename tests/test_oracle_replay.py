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


def _w_setup(eps_p=0.05):
    q = scenes.random_quadruple(32, 24, 3, sigma=0.01)
    lv = O.Level(O.level_planes(O.pyramid(q, 1)[0]), 4, 0)
    kw = dict(pcg_iters=(8,) * 8, eps_p=eps_p)
    base = np.zeros(6 * lv.G)
    wf = O.feature_weights(lv, base, O.Params(gn_iters=(1,) * 8, **kw))
    return q, lv, kw, base, wf


def test_replaying_the_oracles_own_W_changes_nothing():
    """W of each step, taken by the oracle at that step's linearisation point
    (C11) and given back, gives the same solve, with no pixel counted as
    differing."""
    q, lv, kw, base, wf = _w_setup()
    p2 = O.Params(gn_iters=(2,) * 8, **kw)
    W = []
    for g in range(2):
        delta = (O.solve_frame(q, 4, 1, O.Params(gn_iters=(g,) * 8, **kw)).deltas(0).reshape(-1) if g
                 else np.zeros(6 * lv.G))
        W.append(O.assemble(lv, base, delta, wf, p2)[3])
    assert 0 < int(W[0].sum()) < W[0].size  # both decisions occur
    r0 = O.solve_frame(q, 4, 1, p2)
    r1 = O.solve_frame(q, 4, 1, p2, W_given=[W])
    assert np.array_equal(r0.total, r1.total) and r0.energy == r1.energy
    for g in range(2):
        assert r1.step(0, g)[5] == 0 and r1.step(0, g)[6] == 0.0


def test_a_differing_W_is_used_counted_and_measured():
    """The complement of the oracle's own W: every pixel counts as differing,
    the margin is the largest distance of max_k |e_k| from eps_p, and the step
    runs on the given mask (its energy at the linearisation point is the
    energy under that mask)."""
    q, lv, kw, base, wf = _w_setup()
    p1 = O.Params(gn_iters=(1,) * 8, **kw)
    zero = np.zeros(6 * lv.G)
    W_own = O.assemble(lv, base, zero, wf, p1)[3]
    W_flip = (1 - W_own).astype(np.uint8)
    r0 = O.solve_frame(q, 4, 1, p1)
    r1 = O.solve_frame(q, 4, 1, p1, W_given=[[W_flip]])
    st = r1.step(0, 0)
    assert st[5] == W_own.size
    E_flip = O.energy(lv, base, zero, wf, p1, W_flip)[0]
    assert st[0] == E_flip and E_flip != r0.step(0, 0)[0]
    assert not np.array_equal(r0.total, r1.total)
    # the margin: max over pixels of | max_k |e_k| - eps_p | at zero fields
    margins = []
    for y in range(lv.h):
        for x in range(lv.w):
            e = O.pixel_terms(lv.planes, float(x), float(y), np.zeros(6))["e"]
            margins.append(abs(np.max(np.abs(e)) - kw["eps_p"]))
    assert abs(st[6] - max(margins)) <= 1e-12
