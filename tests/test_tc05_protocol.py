"""The mbarrier protocol of the persistent tcgen05 products kernel
(csrc/mk_tensor_tc05.cu), as a model run under random interleavings.

Three roles share one pass sequence gp = 0 .. items * 2 * nchunks - 1 (pass
gp: TMEM half gp % 2, unit arrays of that half):
  producer  -- digit tile j = gp * KSTEPS + kc into stage j % S; waits
               empty[stage] with parity (j / S - 1) & 1 for j >= S, then
               arrives on full[stage] (the TMA's complete_tx);
  MMA warp  -- waits ready[h] with parity (gp / 2) & 1, then full[stage]
               with parity (j / S) & 1 per tile, commits empty[stage] per
               tile and done[h] per pass;
  workers   -- build the units of passes 0 and 1 and arrive on ready[0],
               ready[1]; step gp: wait done[(gp-1) % 2] with parity
               ((gp-1) / 2) & 1, drain, write the item's outputs after its
               last pass, then build the units of pass gp + 1 (if gp + 1 >= 2)
               and arrive on ready[(gp+1) % 2].
A barrier completes a phase when its pending count reaches zero; waiting
with parity P returns once the phase of parity P has completed (PTX
mbarrier.try_wait.parity).  The model asserts that the run ends (no
deadlock) and that no buffer is reused early: a unit array is rebuilt only
after the MMAs that read it completed, a TMEM half is overwritten only after
it was drained, a stage is refilled only after its MMAs committed, and every
item's outputs are written once, in order.
"""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        assert self.pending > 0
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def passed(self, parity):
        return (self.phase & 1) != parity


def run_protocol(nch, nitems, stages, ksteps, seed, workers=1):
    rnd = random.Random(seed)
    PI = 2 * nch
    PT = PI * nitems
    full = [Barrier(1) for _ in range(stages)]
    empty = [Barrier(1) for _ in range(stages)]
    done = [Barrier(1), Barrier(1)]
    ready = [Barrier(workers), Barrier(workers)]
    st = {"units": [None, None], "tmem": [None, None], "stage": [None] * stages}
    drained, mma_done, outputs = set(), set(), []

    def producer():
        for gp in range(PT):
            for kc in range(ksteps):
                j = gp * ksteps + kc
                s = j % stages
                if j >= stages:
                    while not empty[s].passed(((j // stages) - 1) & 1):
                        yield
                prev = st["stage"][s]
                assert prev is None or prev + stages == j
                st["stage"][s] = j
                yield
                full[s].arrive()

    def mma():
        for gp in range(PT):
            h = gp & 1
            while not ready[h].passed((gp >> 1) & 1):
                yield
            assert st["units"][h] == gp
            assert st["tmem"][h] is None or st["tmem"][h] in drained
            st["tmem"][h] = gp
            for kc in range(ksteps):
                j = gp * ksteps + kc
                s = j % stages
                while not full[s].passed((j // stages) & 1):
                    yield
                assert st["stage"][s] == j
                yield
                empty[s].arrive()
            mma_done.add(gp)
            done[h].arrive()

    def worker(w):
        for h in range(2):
            if w == 0:
                st["units"][h] = h
            yield
            ready[h].arrive()
        for gp in range(PT + 1):
            if gp >= 1:
                pp = gp - 1
                while not done[pp & 1].passed((pp >> 1) & 1):
                    yield
                assert pp in mma_done and st["tmem"][pp & 1] == pp
                if w == 0:
                    drained.add(pp)
                    if pp % PI == PI - 1:
                        outputs.append(pp // PI)
                yield
            q = gp + 1
            if 2 <= q < PT:
                assert (q - 2) in mma_done
                if w == 0:
                    st["units"][q & 1] = q
                yield
                ready[q & 1].arrive()

    agents = [producer(), mma()] + [worker(w) for w in range(workers)]
    alive = list(agents)
    for _ in range(2_000_000):
        if not alive:
            break
        a = rnd.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert not alive, "deadlock"
    assert drained == set(range(PT))
    assert outputs == list(range(nitems))


@pytest.mark.parametrize("nch", [1, 2, 3])
@pytest.mark.parametrize("nitems", [1, 2, 5])
def test_tc05_protocol_completes_without_hazards(nch, nitems):
    for seed in range(40):
        run_protocol(nch, nitems, stages=4, ksteps=4, seed=seed)


def test_tc05_protocol_with_several_worker_threads():
    """The ready barriers count every worker thread: with three modelled
    workers a phase completes only after all three arrive."""
    for seed in range(30):
        run_protocol(3, 3, stages=4, ksteps=2, seed=seed, workers=3)


def test_tc05_model_detects_a_wrong_parity():
    """The model is not vacuous: a ready wait with the wrong parity (waiting
    for phase (gp / 2 + 1) & 1) lets the MMAs run on unit arrays that are
    not built yet, which the model reports."""
    orig = Barrier.passed

    def wrong(self, parity):
        return orig(self, parity ^ 1) if self.count > 1 else orig(self, parity)

    Barrier.passed = wrong
    try:
        with pytest.raises(AssertionError):
            for seed in range(20):
                run_protocol(2, 2, stages=4, ksteps=2, seed=seed, workers=2)
    finally:
        Barrier.passed = orig
