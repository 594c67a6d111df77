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


# ----------------------------------------------------------------------------- timeouts
def run_protocol_abort(nch, nitems, stages, ksteps, seed, skip_tile=None, budget=20000, drain=True, copy_rate=0.5):
    """The same three roles with the kernel's exits: every role's waits give
    up after `budget` polls or as soon as the CTA's abort word is set (and set
    it when they give up); the producer then waits for its copies still in
    flight and the MMA warp commits once more and waits for that commit --
    waits that are not cut short by the abort word.  Copies land and MMAs
    complete asynchronously (two more agents: the copy engine completes any
    copy in flight; the tensor pipe executes the MMA warp's operations in
    order, a commit arriving once every earlier MMA is done).  skip_tile: a
    tile whose copy is never issued (the kernel's test hook).  Returns whether
    the CTA aborted; asserts that the run ends and that when the last role
    leaves (the CTA's final barrier, after which TMEM is released and the CTA
    exits) no copy and no MMA is in flight.  drain=False removes the
    producer's wait for its copies (a planted mistake); copy_rate is the
    chance per turn that the copy engine lands a copy."""
    rnd = random.Random(seed)
    PI = 2 * nch
    PT = PI * nitems
    full = [Barrier(1) for _ in range(stages)]
    empty = [Barrier(1) for _ in range(stages)]
    done = [Barrier(1), Barrier(1)]
    ready = [Barrier(1), Barrier(1)]
    fin = Barrier(1)
    st = {"abort": False, "roles_left": 3}
    tma_inflight = set()   # tiles whose copy was issued and has not landed
    tensor_queue = []      # ("mma", j) / ("commit", barrier), executed in order
    mma_inflight = set()
    exit_state = {}

    def wait(bar, parity, abortable):
        spins = 0
        while not bar.passed(parity):
            if abortable and st["abort"]:
                return False
            spins += 1
            if spins > budget:
                assert abortable, "a wait for the CTA's own copies or MMAs did not finish"
                st["abort"] = True
                return False
            yield
        return True

    def leave():
        st["roles_left"] -= 1
        if st["roles_left"] == 0:  # the CTA's final barrier: TMEM is released, the CTA exits
            exit_state["tma"] = set(tma_inflight)
            exit_state["mma"] = set(mma_inflight)

    def producer():
        issued, skipped, ok = 0, None, True
        for gp in range(PT):
            for kc in range(ksteps):
                j = gp * ksteps + kc
                s = j % stages
                if j >= stages:
                    ok = yield from wait(empty[s], ((j // stages) - 1) & 1, True)
                    if not ok:
                        break
                if j == skip_tile:
                    skipped = j
                else:
                    tma_inflight.add(j)
                issued = j + 1
                yield
            if not ok:
                break
        for j in range(max(0, issued - stages), issued):
            if drain and j != skipped:
                yield from wait(full[j % stages], (j // stages) & 1, False)
        leave()

    def mma():
        ok = True
        for gp in range(PT):
            h = gp & 1
            ok = yield from wait(ready[h], (gp >> 1) & 1, True)
            if not ok:
                break
            for kc in range(ksteps):
                j = gp * ksteps + kc
                s = j % stages
                ok = yield from wait(full[s], (j // stages) & 1, True)
                if not ok:
                    break
                mma_inflight.add(j)
                tensor_queue.append(("mma", j))
                tensor_queue.append(("commit", empty[s]))
                yield
            if not ok:
                break
            tensor_queue.append(("commit", done[h]))
        tensor_queue.append(("commit", fin))
        yield from wait(fin, 0, False)
        leave()

    def worker():
        for h in range(2):
            yield
            ready[h].arrive()
        for gp in range(PT + 1):
            if gp >= 1:
                pp = gp - 1
                ok = yield from wait(done[pp & 1], (pp >> 1) & 1, True)
                if not ok:
                    break
                yield
            q = gp + 1
            if 2 <= q < PT:
                yield
                ready[q & 1].arrive()
        leave()

    def copy_engine():
        while st["roles_left"] > 0 or tma_inflight:
            if tma_inflight and rnd.random() < copy_rate:
                j = rnd.choice(sorted(tma_inflight))
                tma_inflight.remove(j)
                full[j % stages].arrive()
            yield

    def tensor_pipe():
        while st["roles_left"] > 0 or tensor_queue:
            if tensor_queue and rnd.random() < 0.5:
                kind, x = tensor_queue.pop(0)
                if kind == "mma":
                    mma_inflight.remove(x)
                else:
                    x.arrive()
            yield

    alive = [producer(), mma(), worker(), copy_engine(), tensor_pipe()]
    for _ in range(5_000_000):
        if not alive:
            break
        a = rnd.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    assert not alive, "deadlock"
    assert exit_state["tma"] == set(), "a copy was in flight when the CTA left"
    assert exit_state["mma"] == set(), "an MMA was in flight when TMEM was released"
    return st["abort"]


@pytest.mark.parametrize("nch,nitems", [(1, 1), (3, 2)])
def test_tc05_protocol_no_timeout_without_a_fault(nch, nitems):
    """With every copy issued, no wait gives up (the budget is never reached)."""
    for seed in range(15):
        assert not run_protocol_abort(nch, nitems, stages=4, ksteps=4, seed=seed)


@pytest.mark.parametrize("skip", [0, 3, 5, 17, 31])
def test_tc05_protocol_skipped_copy_times_out_cleanly(skip):
    """A tile whose copy is never issued: the MMA warp's wait for it gives up,
    every role leaves, and nothing is in flight when the CTA releases TMEM."""
    for seed in range(15):
        assert run_protocol_abort(2, 2, stages=4, ksteps=4, seed=seed, skip_tile=skip, budget=3000)


def test_tc05_model_detects_a_missing_drain():
    """The model is not vacuous: a producer that leaves without waiting for
    its copies in flight is reported when the copies land slowly."""
    with pytest.raises(AssertionError, match="copy was in flight"):
        for seed in range(10):
            run_protocol_abort(2, 1, stages=4, ksteps=4, seed=seed, skip_tile=5, budget=3000, drain=False,
                               copy_rate=0.002)
