"""A model of the tagged partial-sum protocol of the grid PCG reduction
(allreduce2_tagged in sf_pcg.cu), run under random interleavings on the CPU.

In the kernel, every block publishes each reduction's partial as words that
carry the reduction's tag (1, 2, ...), in slot [tag & 1][block]. One warp per
block then polls all blocks' words until every one carries the tag, and folds
them. Slots are cleared to tag 0 before the launch's first grid barrier. The
claim is that two slots by tag parity suffice: a block writes tag k + 2 only
after every block has published k + 1, and each block publishes k + 1 only
after it has read k. Here each block is a generator that yields after every
single memory operation, and a seeded scheduler interleaves them at random.
The test checks that every block gets every reduction's exact total and that
nothing deadlocks. It also checks that two planted mistakes are caught: one
slot instead of two, and stale tags from an earlier launch left uncleared.
"""

import random

import pytest


def _block(b, nb, K, slots, nslots, values, results):
    """Block b: for k = 1..K publish (k, value), then poll every block's slot
    until all carry tag k in one pass, then fold them in block order."""
    for k in range(1, K + 1):
        s = k % nslots
        slots[s][b] = (k, values[k][b])
        yield "write"
        while True:
            seen = []
            ready = True
            for c in range(nb):
                tag, v = slots[s][c]
                yield "read"
                if tag != k:
                    ready = False
                seen.append(v)
            if ready:
                break
        results[b].append(sum(seen))


def _run(nb, K, seed, nslots=2, clear=True, max_steps=200000):
    rng = random.Random(seed)
    values = {k: [rng.randint(-1000, 1000) for _ in range(nb)] for k in range(1, K + 1)}
    # words left by an earlier launch: tags of its own reductions
    slots = [[(rng.randint(1, K), rng.randint(-1000, 1000)) for _ in range(nb)] for _ in range(nslots)]
    if clear:
        # each block clears its own slots, then the launch's first grid barrier
        for s in range(nslots):
            for b in range(nb):
                slots[s][b] = (0, 0)
    results = [[] for _ in range(nb)]
    gens = [_block(b, nb, K, slots, nslots, values, results) for b in range(nb)]
    live = list(range(nb))
    steps = 0
    while live:
        i = rng.choice(live)
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        if steps > max_steps:
            return None, values
    return results, values


@pytest.mark.parametrize("nb,K", [(2, 6), (3, 21), (5, 21), (8, 10)])
def test_two_slots_give_every_block_every_exact_total(nb, K):
    for seed in range(40):
        results, values = _run(nb, K, seed)
        assert results is not None, f"no progress (seed {seed})"
        want = [sum(values[k]) for k in range(1, K + 1)]
        for b in range(nb):
            assert results[b] == want, (seed, b)


def test_one_slot_is_caught():
    """With one slot a fast block overwrites tag k with k + 1 while a slow
    block still polls for k: the slow block never sees k again."""
    failures = 0
    for seed in range(40):
        results, values = _run(3, 8, seed, nslots=1, max_steps=20000)
        want = [sum(values[k]) for k in range(1, 9)]
        if results is None or any(r != want for r in results):
            failures += 1
    assert failures > 0


def test_uncleared_stale_tags_are_caught():
    """Without the clear, a stale word whose tag equals a current reduction's
    tag passes the poll with the earlier launch's value."""
    failures = 0
    for seed in range(200):
        results, values = _run(3, 4, seed, clear=False, max_steps=20000)
        want = [sum(values[k]) for k in range(1, 5)]
        if results is None or any(r != want for r in results):
            failures += 1
    assert failures > 0
