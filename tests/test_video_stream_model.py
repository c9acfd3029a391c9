"""A model of the stream and event ordering of the level pipeline
(enqueue_video in sf_capi.cu: sf_solve_video and sf_solve_video_host),
checked on the CPU.

The model enqueues the same operations in the same order as enqueue_video:
the fork from the caller's stream, the temporal-state copies of a call that
continues a video, per pipeline step the join of the level streams (each
records an event, each waits for the others') and level l of frame
s - (L - 1 - l) on level l's stream (coarsest first; its frame's images
copied in and its pyramid before it), and, from host memory, each frame's
fields copied out on the copy stream after its level 0 (an event from level
0's stream), the copy stream recording the slot's "copied" event, and level 0
waiting for that event before it writes the slot again; at the end the
caller's stream waits for every level stream and the copy stream, the state
is handed back, and the host call synchronises.

CUDA's rules are taken as stated in its documentation: a stream runs its
operations in order; a wait on an event orders the stream after the latest
record of that event enqueued before the wait (none: no effect); a host
synchronisation orders everything enqueued later after the stream's work.
From these the model forms the happens-before relation, and checks every pair
of operations that touch one buffer, at least one writing it, against the
order of the plain sequential solve (frame by frame, coarsest level first):
the earlier one must happen before the later. It checks videos of one to nine
frames at two to four levels, in one call and in two calls (the second
continuing the first), from device and from host memory; and that five
planted mistakes are caught: level 0 not waiting for the slot's copy, the
copy not waiting for level 0, the caller's stream not waiting for the copy
stream, no join between the steps, and a ring one slot short.
"""

import itertools

import pytest


class StreamModel:
    def __init__(self):
        self.anc = []        # ancestors of each operation (bit set)
        self.last = {}       # stream -> its last operation
        self.ev = {}         # event -> its latest record
        self.fence = None    # last host synchronisation
        self.acc = []        # (operation, sequential position, reads, writes)

    def _add(self, stream, deps):
        i = len(self.anc)
        a = 0
        for d in [self.last.get(stream), self.fence] + deps:
            if d is not None:
                a |= self.anc[d] | (1 << d)
        self.anc.append(a)
        self.last[stream] = i
        return i

    def record(self, ev, stream):
        self.ev[ev] = self._add(stream, [])

    def wait(self, stream, ev):
        self._add(stream, [self.ev[ev]] if ev in self.ev else [])

    def work(self, stream, pos, reads=(), writes=()):
        i = self._add(stream, [])
        self.acc.append((i, pos, tuple(reads), tuple(writes)))

    def host_sync(self, stream):
        self.fence = self.last.get(stream, self.fence)

    def violations(self):
        by_buf = {}
        for i, pos, reads, writes in self.acc:
            for b in reads:
                by_buf.setdefault(b, []).append((pos, i, False))
            for b in writes:
                by_buf.setdefault(b, []).append((pos, i, True))
        bad = []
        for b, lst in by_buf.items():
            lst.sort()
            for (pa, ia, wa), (pb, ib, wb) in itertools.combinations(lst, 2):
                if ia != ib and (wa or wb) and not (self.anc[ib] >> ia) & 1:
                    bad.append((b, pa, pb))
        return bad


def enqueue_video(m, L, R, n, f0, call, host, mistakes=()):
    """The operations of one sf_solve_video(_host) call, in enqueue order."""
    st = "caller"
    m.record("fork", st)
    for l in range(L):
        m.wait(f"level{l}", "fork")
    if host:
        m.wait("copy", "fork")
    if f0 > 0:  # the previous call's state into the pipeline's buffers
        for l in range(L):
            m.work(f"level{l}", (call, 0, l), reads=[f"prev{l}"],
                   writes=[f"delta{l}.{(f0 - 1) & 1}", f"total{l}.{(f0 - 1) & 1}"])
    for s in range(n + L - 1):
        if s > 0 and "no_join" not in mistakes:
            for l in range(L):
                m.record(f"step{l}", f"level{l}")
            for l in range(L):
                for k in range(L):
                    if k != l:
                        m.wait(f"level{l}", f"step{k}")
        for l in range(L - 1, -1, -1):
            fl = s - (L - 1 - l)
            if fl < 0 or fl >= n:
                continue
            fg, bs = f0 + fl, f"level{l}"
            slot = fg % R
            if l == L - 1:
                src = f"dev_in{call}.{fl}"
                if host:
                    m.work(bs, (call, 1, fl, 0), reads=[f"host_in{call}.{fl}"], writes=[f"in{slot}"])
                    src = f"in{slot}"
                m.work(bs, (call, 1, fl, 1), reads=[src], writes=[f"tex{slot}.{k}" for k in range(L)])
            out = f"out{slot}" if host else f"dev_out{call}.{fl}"
            if l == 0 and host and "no_slot_wait" not in mistakes:
                m.wait(bs, f"copied{slot}")
            reads = [f"tex{slot}.{l}", f"vis{l}.{fg & 1}", f"delta{l}.{(fg + 1) & 1}", f"total{l}.{(fg + 1) & 1}",
                     f"scratch{l}"]
            writes = [f"delta{l}.{fg & 1}", f"total{l}.{fg & 1}", f"scratch{l}"]
            if l < L - 1:
                reads.append(f"total{l + 1}.{fg & 1}")
            if l > 0:
                writes.append(f"vis{l - 1}.{fg & 1}")
            if l == 0:
                writes.append(out)
            m.work(bs, (call, 1, fl, 2 + (L - 1 - l)), reads, writes)
            if l == 0 and host:
                if "copy_no_wait" not in mistakes:
                    m.record("level0_done", bs)
                    m.wait("copy", "level0_done")
                m.work("copy", (call, 1, fl, 2 + L), reads=[out], writes=[f"host_out{call}.{fl}"])
                m.record(f"copied{slot}", "copy")
    for l in range(L):
        m.record(f"step{l}", f"level{l}")
        m.wait(st, f"step{l}")
    if host and "no_final_copy_wait" not in mistakes:
        m.record("level0_done", "copy")
        m.wait(st, "level0_done")
    fz = f0 + n - 1
    for l in range(L):  # the last frame's state back to the single-frame path
        m.work(st, (call, 2, l), reads=[f"delta{l}.{fz & 1}", f"total{l}.{fz & 1}"], writes=[f"prev{l}"])
    if host:
        m.host_sync(st)
        for fl in range(n):
            m.work("host", (call, 3, fl), reads=[f"host_out{call}.{fl}"])


def run(L, calls, host, mistakes=(), ring=None):
    m = StreamModel()
    f0 = 0
    for call, n in enumerate(calls):
        enqueue_video(m, L, L if ring is None else ring, n, f0, call, host, mistakes)
        f0 += n
    return m.violations()


@pytest.mark.parametrize("host", [False, True])
@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("calls", [(1,), (2,), (5,), (9,), (4, 2), (1, 7), (3, 3, 1)])
def test_pipeline_orders_every_conflicting_access(L, calls, host):
    assert run(L, calls, host) == []


@pytest.mark.parametrize("mistake,host", [("no_slot_wait", True), ("copy_no_wait", True),
                                          ("no_final_copy_wait", True), ("no_join", False), ("no_join", True)])
def test_planted_ordering_mistakes_are_caught(mistake, host):
    assert any(run(L, calls, host, mistakes=(mistake,)) for L in (2, 3, 4) for calls in ((6,), (4, 3)))


@pytest.mark.parametrize("host", [False, True])
def test_a_ring_one_slot_short_is_caught(host):
    assert any(run(L, (6,), host, ring=L - 1) for L in (2, 3, 4))
