"""The key-ring protocol of the staged blind rotation
(csrc/mk_bootstrap_staged.cuh), as a model run under random interleavings.

G groups walk the same steps s = 0 .. S-1.  Two buffers (b = 0: D, read in
phase A; b = 1: F, read in phase B) each hold one step's key data.  Per
step and buffer a group: waits until the buffer's mbarrier has completed
phase s (parity s & 1), reads the buffer, then (after its group barrier)
adds one to the buffer's monotonic counter; the add that makes the count a
multiple of G issues the copy of step s + 1 into the buffer (if s + 1 < S).
A skipped step (e = 0) waits for and releases both buffers without reading.
Waits give up after a budget or when the CTA's abort word is set (setting
it when they give up); after the step loop thread 0 waits, without the
abort word, for the last copy issued into each buffer.

The model asserts: the run ends; no copy lands in a buffer that a group is
still reading (or has yet to read) for an earlier step; every group reads
step s's data when it reads at step s; and no copy is in flight when the
CTA leaves.  A planted mistake (the releases counted before the group has
read) is detected.
"""
import random

import pytest


class Barrier:
    def __init__(self):
        self.phase = 0

    def complete(self):
        self.phase += 1

    def passed(self, parity):
        return (self.phase & 1) != parity


def run_ring(G, S, seed, skip_step=None, budget=20000, release_early=False, skips=()):
    rnd = random.Random(seed)
    full = [Barrier(), Barrier()]
    buf = [None, None]          # the step whose data each buffer holds (None: not yet)
    count = [0, 0]
    issued = [0, 0]
    inflight = {}               # buffer -> step of the copy in flight
    readers = [set(), set()]    # groups reading a buffer right now
    st = {"abort": False, "left": 0}
    exit_state = {}

    def issue(b, s):
        if s == skip_step:
            return
        assert b not in inflight
        assert not readers[b], "a copy was issued into a buffer still being read"
        inflight[b] = s
        issued[b] += 1

    def wait(b, s):
        spins = 0
        while not full[b].passed(s & 1):
            if st["abort"]:
                return False
            spins += 1
            if spins > budget:
                st["abort"] = True
                return False
            yield
        return True

    def release(b, s):
        old = count[b]
        count[b] += 1
        if (old + 1) % G == 0 and s + 1 < S:
            issue(b, s + 1)

    def group(g):
        for s in range(S):
            for b in (0, 1):
                ok = yield from wait(b, s)
                if not ok:
                    st["left"] += 1
                    return
                if (g, s) in skips:
                    release(b, s)
                    yield
                    continue
                if release_early:
                    release(b, s)
                readers[b].add(g)
                assert buf[b] == s, "group %d read step %s's data at step %d" % (g, buf[b], s)
                yield
                assert buf[b] == s, "the buffer changed while group %d read it" % g
                readers[b].discard(g)
                if not release_early:
                    release(b, s)
                yield
        st["left"] += 1

    def copy_engine():
        while st["left"] < G or inflight:
            if inflight and rnd.random() < 0.3:
                b = rnd.choice(sorted(inflight))
                buf[b] = inflight.pop(b)
                full[b].complete()
            yield

    def leader_drain():
        while st["left"] < G:
            yield
        if st["abort"]:
            for b in (0, 1):
                if issued[b]:
                    while not full[b].passed((issued[b] - 1) & 1):
                        yield
        exit_state["inflight"] = dict(inflight)

    if S > 0:
        issue(0, 0)
        issue(1, 0)
    alive = [group(g) for g in range(G)] + [copy_engine(), leader_drain()]
    for _ in range(5_000_000):
        if not alive:
            break
        a = rnd.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert not alive, "deadlock"
    assert exit_state["inflight"] == {}, "a copy was in flight when the CTA left"
    return st["abort"]


@pytest.mark.parametrize("G", [2, 3])
@pytest.mark.parametrize("S", [1, 2, 7])
def test_ring_completes_without_hazards(G, S):
    for seed in range(25):
        skips = {(g, s) for g in range(G) for s in range(S) if random.Random(seed * 31 + g * 7 + s).random() < 0.2}
        assert not run_ring(G, S, seed, skips=skips)


@pytest.mark.parametrize("skip_step", [0, 1, 4])
def test_ring_skipped_copy_times_out_cleanly(skip_step):
    """A step whose copies are never issued: the waits for it give up, every
    group leaves, and nothing is in flight when the CTA leaves."""
    for seed in range(25):
        assert run_ring(3, 6, seed, skip_step=skip_step, budget=2000)


def test_ring_model_detects_an_early_release():
    """The model is not vacuous: releasing a buffer before reading it lets the
    next step's copy land under a reader."""
    with pytest.raises(AssertionError):
        for seed in range(40):
            run_ring(3, 5, seed, release_early=True)
