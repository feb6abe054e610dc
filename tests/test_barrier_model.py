"""Host model of the step kernel's grid barrier, run on the CPU.

The model restates `grid_barrier` (paper_1310_4218_gb300/csrc/lb_step_kernel.cuh)
and the host's reset of the barrier words before every launch (`launch` in
lb_api.cu).  It is the step boundary of Fig. 2: every processor waits for all
others before the next step (the paper's MPI_Waits), here with a time limit.

Thread 0 of each CTA is a generator.  It yields after every access to a shared
word: the arrival counter, the generation, the status word.  A seeded scheduler
picks which CTA moves next, so each seed is one interleaving.  The kernel's
fences order each CTA's own accesses, so the model is sequentially consistent.
The clock is the number of scheduler moves; the kernel reads globaltimer and
clock64 instead.  The kernel's __nanosleep between polls only changes timing,
so it is left out.

Checked:
- no CTA leaves barrier s before every CTA has arrived at it;
- without a time limit firing, every CTA passes every step, and the counter
  ends at 0 with the generation advanced once per step, across a 32-bit wrap;
- a time limit ends every CTA of the launch and leaves LB_ETIMEOUT in the
  status word; a status already set ends the launch at its first barrier;
- after the host's reset and status clear, the next launch is clean, and a
  counter not reset lets a CTA through early.
Three planted protocol mistakes must each be caught, so the checks can fail.
"""
import random

import pytest

LB_ETIMEOUT = 3
M32 = 0xFFFFFFFF
POLL = 32                 # spin iterations between status and time-limit checks


class Words:
    """Device words of one launch: arrival counter, generation, status."""

    def __init__(self, count=0, gen=0, status=0):
        self.count, self.gen, self.status = count, gen, status
        self.clock = 0


class Log:
    def __init__(self, nblocks, nsteps):
        self.nblocks = nblocks
        self.arrived = [set() for _ in range(nsteps)]
        self.passed = [set() for _ in range(nsteps)]
        self.exited = {}
        self.violations = []

    def arrive(self, s, b):
        self.arrived[s].add(b)

    def leave(self, s, b):
        if len(self.arrived[s]) < self.nblocks:
            self.violations.append((s, b, sorted(self.arrived[s])))
        self.passed[s].add(b)


def grid_barrier(w, nblocks, timeout, mutant=None):
    """One CTA's barrier call; returns whether the CTA may go on."""
    if mutant != "gen_after_arrive":
        gen = w.gen                                   # generation before arriving
        yield
    prev = w.count                                    # atomicAdd on the counter
    w.count = (w.count + 1) & M32
    yield
    if mutant == "gen_after_arrive":
        gen = w.gen
        yield
    ok = True
    last = nblocks - 2 if mutant == "early_last" else nblocks - 1
    if prev == last:
        if mutant == "publish_before_reset":
            w.gen = (w.gen + 1) & M32
            yield
            w.count = 0
            yield
        else:
            w.count = 0                               # reset, fence, then publish
            yield
            w.gen = (w.gen + 1) & M32
            yield
    else:
        t0, it = w.clock, 0
        while True:
            g = w.gen
            yield
            if g != gen:
                break
            it += 1
            if it % POLL == 0:
                st = w.status
                yield
                if st != 0:                           # another CTA recorded a failure
                    ok = False
                    break
                if w.clock - t0 > timeout:            # atomicCAS(status, 0, LB_ETIMEOUT)
                    if w.status == 0:
                        w.status = LB_ETIMEOUT
                    yield
                    ok = False
                    break
    st = w.status
    yield
    return ok and st == 0


def cta(w, b, nsteps, work, nblocks, timeout, log, mutant):
    for s in range(nsteps):
        for _ in range(work[b][s]):
            yield
        log.arrive(s, b)
        ok = yield from grid_barrier(w, nblocks, timeout, mutant)
        if not ok:
            log.exited[b] = s
            return
        log.leave(s, b)
    log.exited[b] = None


def run(nblocks, work, timeout, seed, words=None, mutant=None, max_moves=2_000_000):
    nsteps = len(work[0])
    w = words if words is not None else Words()
    log = Log(nblocks, nsteps)
    rng = random.Random(seed)
    live = [cta(w, b, nsteps, work, nblocks, timeout, log, mutant) for b in range(nblocks)]
    moves = 0
    while live:
        i = rng.randrange(len(live))
        try:
            next(live[i])
        except StopIteration:
            live.pop(i)
        w.clock += 1
        moves += 1
        assert moves <= max_moves, "a CTA did not terminate"
    return w, log


def random_work(nblocks, nsteps, seed, hi=6):
    rng = random.Random(1000 + seed)
    return [[rng.randint(0, hi) for _ in range(nsteps)] for _ in range(nblocks)]


@pytest.mark.parametrize("nblocks", [1, 2, 3, 5, 8])
def test_no_cta_leaves_a_barrier_early_and_every_step_completes(nblocks):
    nsteps = 4
    for seed in range(60):
        w, log = run(nblocks, random_work(nblocks, nsteps, seed), 4000, seed)
        assert not log.violations, (seed, log.violations[:3])
        assert w.status == 0, seed
        assert all(len(p) == nblocks for p in log.passed), seed
        assert all(v is None for v in log.exited.values()), seed
        assert w.count == 0 and w.gen == nsteps, seed


def test_generation_counter_wraps():
    nblocks, nsteps = 4, 5
    for seed in range(20):
        words = Words(gen=M32 - 1)
        w, log = run(nblocks, random_work(nblocks, nsteps, seed), 4000, seed, words=words)
        assert not log.violations and w.status == 0, seed
        assert w.gen == (M32 - 1 + nsteps) & M32, seed


def test_time_limit_ends_every_cta_and_records_the_timeout():
    """One CTA's step-1 work outlasts the limit: the others give up at
    barrier 1, the late CTA finds the status set, and nobody passes it."""
    nblocks, nsteps, timeout = 6, 3, 2000
    for seed in range(10):
        work = random_work(nblocks, nsteps, seed)
        work[2][1] = 5 * timeout
        w, log = run(nblocks, work, timeout, seed)
        assert w.status == LB_ETIMEOUT, seed
        assert len(log.exited) == nblocks, seed
        assert all(s == 1 for s in log.exited.values()), (seed, log.exited)
        assert not log.passed[1] and not log.violations, seed


def test_status_set_before_the_launch_ends_it_at_the_first_barrier():
    nblocks, nsteps = 5, 4
    for seed in range(10):
        w, log = run(nblocks, random_work(nblocks, nsteps, seed), 4000, seed,
                     words=Words(status=LB_ETIMEOUT))
        assert all(s == 0 for s in log.exited.values()) and len(log.exited) == nblocks
        assert not any(log.passed) and w.status == LB_ETIMEOUT


def test_launch_after_a_timeout_is_clean_once_the_words_are_reset():
    """A launch that timed out may leave the counter part-filled.  The host
    zeroes both barrier words before each launch and lb_sync clears the
    status, after which every step completes."""
    nblocks, nsteps, timeout = 5, 3, 1500
    for seed in range(10):
        work = random_work(nblocks, nsteps, seed)
        work[seed % nblocks][seed % nsteps] = 4 * timeout
        w, _ = run(nblocks, work, timeout, seed)
        assert w.status == LB_ETIMEOUT
        w.count, w.gen, w.status = 0, 0, 0
        w2, log = run(nblocks, random_work(nblocks, nsteps, seed + 50), 4000, seed, words=w)
        assert not log.violations and w2.status == 0, seed
        assert all(len(p) == nblocks for p in log.passed), seed


def test_counter_that_is_not_reset_lets_a_cta_through_early():
    """With one stale arrival, the second-to-last CTA releases barrier 0 while
    the slow CTA is still working on step 0."""
    nblocks, nsteps = 4, 3
    caught = 0
    for seed in range(10):
        work = random_work(nblocks, nsteps, seed)
        work[seed % nblocks][0] = 200
        w, log = run(nblocks, work, 2000, seed, words=Words(count=1))
        caught += any(s == 0 for s, _, _ in log.violations)
    assert caught == 10


@pytest.mark.parametrize("mutant", ["gen_after_arrive", "publish_before_reset", "early_last"])
def test_planted_protocol_mistakes_are_caught(mutant):
    """Reading the generation after arriving can miss the release; publishing
    the new generation before the counter reset can lose an arrival; releasing
    one arrival early lets a CTA through.  Each shows up as a CTA passing
    early or as a time limit firing with no slow CTA."""
    nblocks, nsteps, timeout = 4, 4, 2000
    caught = 0
    for seed in range(60):
        w, log = run(nblocks, random_work(nblocks, nsteps, seed, hi=2), timeout, seed,
                     mutant=mutant)
        caught += bool(log.violations) or w.status != 0
    assert caught > 0, mutant
