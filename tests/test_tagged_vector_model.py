"""A model of the self-tagged vector exchange of the staged grid PCG
(k_pcg1h and k_pcg1p in sf_pcg.cu), run under random interleavings on the
CPU.

In the kernel every published vector value is one word (tag << 32 | value),
and a reader checks the tag of every word it loads and loads it again while
it is stale; nothing orders the vectors before the partial sums. Iteration i
reads buffer i & 1 expecting tag i + 1 and publishes into buffer (i + 1) & 1
with tag i + 2; before the launch's one full barrier each block writes its
initial words (tag 1, buffer 0) and clears buffer 1 (tag 0). The claims: a
word that a reader still needs is never overwritten (the owner reaches the
iteration that overwrites it only after every block's partial sums of the
iteration in between, which each block publishes after its reads), and no
word left by an earlier launch passes a check.

Here each block owns one node of a ring and is a generator that yields after
every single memory operation; a seeded scheduler interleaves them, and lets
each block's stores land in any order (relaxed stores to different addresses,
no fences), except that the barrier lands all of a block's stores first. Per
iteration a block reads its two neighbours' words, forms its next value from
them, its own value and the previous iteration's total, publishes it, and
takes part in the tagged partial-sum reduction of the new values. Launches
of different lengths run back to back on the same buffers. As k_pcg1h's warps
1.. do while warp 0 polls, a block may fetch the next iteration's neighbour
words between publishing its partial sum and reading the total (chosen at
random per iteration). The test checks every
block's values against a sequential evaluation and that nothing deadlocks,
and that three planted mistakes are caught: one vector buffer instead of
two, buffer 1 not cleared, and no barrier between the clear and the
iterations.
"""

import random

import pytest


def _next_value(left, own, right, total):
    return (left + 2 * own + right + total) % 1000003


def _reference(v0, K):
    nb = len(v0)
    v, total, out = list(v0), sum(v0) % 1000003, []
    for _ in range(K):
        v = [_next_value(v[(b - 1) % nb], v[b], v[(b + 1) % nb], total) for b in range(nb)]
        total = sum(v) % 1000003
        out.append(list(v))
    return out


def _block(b, nb, K, v0, words, nbuf, slots, results, barrier, clear, early=None):
    """One block over one launch: initial words, clear, barrier, K iterations.
    A store is yielded as ("st", array, index, word) and lands when the
    scheduler commits it; loads read what has landed. early: a random.Random
    that decides per iteration whether the block fetches the next iteration's
    neighbour words (tag i + 2) before its poll of the partial sums, as
    k_pcg1h's warps 1.. do while warp 0 polls, or after it (None: after)."""
    yield ("st", words[0], b, (1, v0[b]))
    if clear:
        for s in range(1, nbuf):
            yield ("st", words[s], b, (0, 0))
    for s in range(2):
        yield ("st", slots[s], b, (0, 0))
    if barrier is not None:
        yield ("arrive",)  # the block's stores land before its arrival counts
        while barrier["arrived"] < barrier["target"]:
            yield ("wait",)
    own, total = v0[b], sum(v0) % 1000003
    fetched = None

    def fetch(vals, buf, want):
        for c in ((b - 1) % nb, (b + 1) % nb):
            while True:  # a stale word is read again
                tag, val = words[buf][c]
                yield ("ld",)
                if tag == want:
                    vals[c] = val
                    break

    for i in range(K):
        buf = i % nbuf
        if fetched is None:
            vals = {}
            yield from fetch(vals, buf, i + 1)
        else:
            vals, fetched = fetched, None
        own = _next_value(vals[(b - 1) % nb], own, vals[(b + 1) % nb], total)
        yield ("st", words[(i + 1) % nbuf], b, (i + 2, own))
        # the tagged partial sums (two slots by tag parity, as allreduce2_tagged)
        k = i + 1
        yield ("st", slots[k % 2], b, (k, own))
        if early is not None and i + 1 < K and early.random() < 0.5:
            fetched = {}
            yield from fetch(fetched, (i + 1) % nbuf, i + 2)
        while True:
            seen, ready = [], True
            for c in range(nb):
                tag, val = slots[k % 2][c]
                yield ("ld",)
                ready = ready and tag == k
                seen.append(val)
            if ready:
                break
        total = sum(seen) % 1000003
        results[b].append(own)


def _run(nb, Ks, seed, nbuf=2, clear=True, barrier=True, max_steps=400000, land=0.35, early=False):
    """Launches of Ks[0], Ks[1], ... iterations back to back on the same buffers
    (a solve that stops early leaves low tags for the next one to meet).
    Stores of one block land in any order, as relaxed stores to different
    addresses may: the scheduler commits a random pending one at random."""
    rng = random.Random(seed)
    words = [[(0, 0)] * nb for _ in range(nbuf)]
    slots = [[(0, 0)] * nb for _ in range(2)]
    outs, wants = [], []
    for K in Ks:
        v0 = [rng.randint(0, 1000) for _ in range(nb)]
        results = [[] for _ in range(nb)]
        bar = {"arrived": 0, "target": nb} if barrier else None
        gens = [_block(b, nb, K, v0, words, nbuf, slots, results, bar, clear,
                       random.Random(rng.random()) if early else None) for b in range(nb)]
        pending = [[] for _ in range(nb)]
        live, steps = list(range(nb)), 0
        while live or any(pending):
            owners = [b for b in range(nb) if pending[b]]
            if owners and (not live or rng.random() < land):
                b = rng.choice(owners)
                arr, idx, word = pending[b].pop(rng.randrange(len(pending[b])))
                arr[idx] = word
            else:
                b = rng.choice(live)
                try:
                    op = next(gens[b])
                except StopIteration:
                    live.remove(b)
                    continue
                if op[0] == "st":
                    pending[b].append(op[1:])
                elif op[0] == "arrive":
                    for arr, idx, word in pending[b]:
                        arr[idx] = word
                    pending[b] = []
                    bar["arrived"] += 1
            steps += 1
            if steps > max_steps:
                return None, None
        outs.append(results)
        want = _reference(v0, K)
        wants.append([[want[i][b] for i in range(K)] for b in range(nb)])
    return outs, wants


@pytest.mark.parametrize("early", [False, True])
@pytest.mark.parametrize("land", [0.05, 0.35])
@pytest.mark.parametrize("nb,Ks", [(2, (5, 5)), (3, (9, 2)), (5, (2, 8)), (7, (1, 6, 3))])
def test_self_tagged_exchange_gives_every_block_the_sequential_values(nb, Ks, land, early):
    for seed in range(30):
        outs, wants = _run(nb, Ks, seed, land=land, early=early)
        assert outs is not None, f"no progress (seed {seed})"
        assert outs == wants, seed


def test_one_vector_buffer_is_caught():
    """With one buffer an owner overwrites a word (tag i + 2 over i + 1) that
    a slower neighbour has not read yet: the neighbour waits for a tag that
    never comes back."""
    failures = 0
    for seed in range(30):
        outs, wants = _run(4, (6, 6), seed, nbuf=1, max_steps=40000, early=seed % 2 == 1)
        if outs is None or outs != wants:
            failures += 1
    assert failures > 0


def test_uncleared_buffer_is_caught():
    """Without the clear, buffer 1 still holds the words of tag 2 of an
    earlier launch that stopped after two iterations, which pass the next
    launch's check at iteration 1."""
    failures = 0
    for seed in range(200):
        outs, wants = _run(4, (2, 6), seed, clear=False, max_steps=40000, land=0.05, early=seed % 2 == 1)
        if outs is None or outs != wants:
            failures += 1
    assert failures > 0


def test_missing_barrier_after_the_clear_is_caught():
    """Without the launch's barrier, a fast block can read a neighbour's
    buffer-1 word of the earlier launch before the neighbour cleared it."""
    failures = 0
    for seed in range(60):
        outs, wants = _run(4, (2, 6), seed, barrier=False, max_steps=40000, early=seed % 2 == 1)
        if outs is None or outs != wants:
            failures += 1
    assert failures > 0
