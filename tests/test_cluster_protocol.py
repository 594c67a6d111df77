"""CPU model of the key staging in the cluster latency kernel
(csrc/mk_bootstrap_cluster.cuh): the control flow of one CTA, with bulk
copies that land after random delays and mbarriers modelled by their phase
count.

Checked for every party count the kernel takes, random rotation words (some
zero: steps the whole cluster skips) and step limits:
  * every wait on a buffer returns only once that buffer holds the keys of
    the step being computed (parity bookkeeping and the choice of the next
    step to copy);
  * a copy into a buffer is issued only after the current step's reads of it;
  * when the CTA exits, no copy it issued is still in flight;
  * with one step's copy never issued (the test hook), a wait runs out, no
    copy is issued after it, every later wait returns at once (the keys read
    after that are stale: the kernel's results are garbage and the status
    reports the timeout), and the exit still finds nothing in flight;
  * the public keys, copied once before the first step, are not taken for a
    skipped step (the hook's "no step" value is negative too).
A planted mistake in the model (the wrong parity, or F copied for steps of
another party) is caught.
"""
import random

import pytest


class Bar:
    """An mbarrier with one arrival per phase, completed by its copy's bytes."""

    def __init__(self):
        self.completed = 0
        self.pending = []  # (land time, step) of copies in flight
        self.content = None
        self.issued = 0

    def land(self, now):
        self.pending.sort()
        while self.pending and self.pending[0][0] <= now:
            _, step = self.pending.pop(0)
            self.content = step
            self.completed += 1

    def try_wait(self, parity):
        # mbarrier.try_wait.parity P succeeds once the phase of parity P has
        # completed, i.e. while the current phase's parity differs from P
        return (self.completed & 1) != parity


def run_cta(k, n, jj, abar, limit, rng, skip=-1, bound=60, mutant=None, stage_a=True):
    """The kernel's sequence for CTA jj; returns (timed_out, log).  stage_a:
    the public keys are staged (the layouts where they fit); otherwise they
    are read through L1 and the A buffer is never used."""
    now = [0]
    bars = {b: Bar() for b in "ADF"}
    abort = [False]
    reading = {b: None for b in "ADF"}  # step whose keys the CTA is reading
    log = []

    def tick(t=1):
        now[0] += t
        for b in bars.values():
            b.land(now[0])

    def next_step(s0, for_f):
        for s in range(s0, limit):
            if abar[s] == 0:
                continue
            if for_f and jj != 0 and jj != s // n + 1 and mutant != "f_any_party":
                continue
            return s
        return limit

    def issue(b, s):
        if abort[0] or (s >= 0 and s == skip):
            return
        assert reading[b] is None, "copy issued into a buffer that is being read"
        bars[b].pending.append((now[0] + rng.randint(0, 8), s))
        bars[b].issued += 1
        log.append(("issue", b, s))

    def wait(b, parity):
        bar = bars[b]
        t0 = now[0]
        while True:
            bar.land(now[0])
            if bar.try_wait(parity):
                return True
            if abort[0]:
                return False
            if now[0] - t0 > bound:
                abort[0] = True
                log.append(("timeout", b))
                return False
            tick()

    if stage_a:
        issue("A", -1)
    s = next_step(0, False)
    if s < limit:
        issue("D", s)
    s = next_step(0, True)
    if s < limit:
        issue("F", s)
    if stage_a and wait("A", 0):
        assert bars["A"].content == -1
    nd = nf = 0
    for s in range(limit):
        if abar[s] == 0:
            continue
        i = s // n + 1
        with_f = jj == 0 or jj == i
        tick(rng.randint(0, 5))  # rotation, digits, forward transform
        par = (nd + 1) & 1 if mutant == "parity" else nd & 1
        if wait("D", par) and not abort[0]:
            assert bars["D"].content == s, ("D holds", bars["D"].content, "at step", s)
        nd += 1
        reading["D"] = s
        tick(rng.randint(0, 2))  # the two products
        reading["D"] = None  # __syncthreads: every read of d is done
        sd = next_step(s + 1, False)
        if sd < limit:
            issue("D", sd)
        tick(rng.randint(0, 5))  # cluster barriers and phase 2
        if with_f:
            if wait("F", nf & 1) and not abort[0]:
                assert bars["F"].content == s, ("F holds", bars["F"].content, "at step", s)
            nf += 1
            reading["F"] = s
            tick(rng.randint(0, 2))
            reading["F"] = None
            sf = next_step(s + 1, True)
            if sf < limit:
                issue("F", sf)
        tick(rng.randint(0, 3))  # inverse transform
    # drain: thread 0 waits (bounded) for the last copy issued into each buffer
    for b in "ADF":
        bar = bars[b]
        if bar.issued:
            t0 = now[0]
            while not bar.try_wait((bar.issued - 1) & 1) and now[0] - t0 <= 10 * bound:
                tick()
        assert not bar.pending, "a copy is still in flight at exit"
    return abort[0], log


def _abar(k, n, rng, zeros=0.15):
    return [0 if rng.random() < zeros else rng.randint(1, 511) for _ in range(k * n)]


@pytest.mark.parametrize("stage_a", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_every_wait_sees_its_step(k, stage_a):
    rng = random.Random(100 + k)
    n = 13
    for trial in range(40):
        abar = _abar(k, n, rng, zeros=rng.choice([0.0, 0.2, 0.6]))
        limit = rng.choice([k * n, k * n, rng.randint(0, k * n)])
        for jj in range(k + 1):
            timed_out, log = run_cta(k, n, jj, abar, limit, rng, stage_a=stage_a)
            assert not timed_out
            d_steps = [s for (ev, b, *rest) in [(e[0], e[1], *e[2:]) for e in log] if ev == "issue" and b == "D"
                       for s in rest]
            assert d_steps == [s for s in range(limit) if abar[s]]


def test_skipped_copy_times_out_and_drains():
    rng = random.Random(7)
    k, n = 2, 11
    for trial in range(60):
        abar = _abar(k, n, rng)
        active = [s for s in range(k * n) if abar[s]]
        skip = rng.choice(active)
        for jj in range(k + 1):
            needs = jj == 0 or jj == skip // n + 1
            timed_out, log = run_cta(k, n, jj, abar, k * n, rng, skip=skip)
            assert timed_out  # the D copy of `skip` is needed by every CTA
            t = next(idx for idx, e in enumerate(log) if e[0] == "timeout")
            assert all(e[0] != "issue" for e in log[t + 1:]), "copy issued after the abort"
            assert needs or log[t][1] == "D"


@pytest.mark.parametrize("mutant", ["parity", "f_any_party"])
def test_planted_mistakes_are_caught(mutant):
    rng = random.Random(3)
    k, n = 3, 9
    caught = False
    for trial in range(30):
        abar = _abar(k, n, rng)
        for jj in range(k + 1):
            try:
                timed_out, _ = run_cta(k, n, jj, abar, k * n, rng, mutant=mutant)
                caught |= timed_out
            except AssertionError:
                caught = True
    assert caught
