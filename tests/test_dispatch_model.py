"""Host model of the step kernel's work dispatch, run on the CPU.

The model restates `pop_item` and `pop_with_stealing`
(paper_1310_4218_gb300/csrc/lb_step_kernel.cuh): how the warps of every
processor (CTA) take the step's work items.  This is the paper's mapping of
over-decomposed VPs to processors (Sec. VI), as a processor's item table, an
atomic task queue, or a table with end-of-step stealing.  The model also covers
the counter resets between steps.  During step s, each processor zeroes its own
stealing counter of parity (s+1) mod 2, and processor 0 zeroes the queue head of
that parity, while the other warps pop from parity s mod 2.  The grid barrier
then orders those resets before step s+1.

Each warp is a generator.  It yields after every access to a shared counter:
an atomic add, or one lane's read of a processor's count in the stealing scan.
A seeded scheduler picks which warp moves next.  Modelling each read as its own
access allows more orders than a warp's single load instruction does.

Checked, per step, over many interleavings:
- every item index runs exactly once;
- every warp terminates;
- a stealing warp gives up only when every processor's counter has passed
  its item count, and never by exhausting its attempt bound.
Planted mistakes (resetting the current parity, a pop that is not atomic, a
smaller attempt bound) must each be caught.
"""
import random

import pytest


class Dev:
    def __init__(self, lens):
        self.nbins = len(lens)
        self.start = [0]
        for n in lens:
            self.start.append(self.start[-1] + n)
        self.nitems = self.start[-1]
        self.ctr = [[0] * self.nbins, [0] * self.nbins]   # stealing counters [parity][bin]
        self.qhead = [0, 0]                                 # queue heads [parity]
        self.s_ctr = [0] * self.nbins                       # shared-memory counter per CTA
        self.gave_up_early = []

    def length(self, b):
        return self.start[b + 1] - self.start[b]


def atomic_add(arr, i, mutant):
    """atomicAdd(&arr[i], 1): old value.  The planted mistake splits it into
    a read and a later write."""
    if mutant == "non_atomic_pop":
        old = arr[i]
        yield
        arr[i] = old + 1
        yield
        return old
    old = arr[i]
    arr[i] = old + 1
    yield
    return old


def pop_with_stealing(d, par, b, mutant):
    ctr = d.ctr[par]
    c = yield from atomic_add(ctr, b, mutant)
    if c < d.length(b):
        return d.start[b] + c
    bound = d.nbins // 2 if mutant == "short_attempt_bound" else 4 * d.nbins + 8
    for _ in range(bound):
        best_rem, best_v = 0, -1
        for v in range(d.nbins):                  # lane v reads processor v's count
            rem = d.length(v) - ctr[v]
            yield
            if rem > best_rem:                    # max remaining, ties to the lowest index
                best_rem, best_v = rem, v
        if best_rem <= 0:
            return -1
        got = yield from atomic_add(ctr, best_v, mutant)
        if got < d.length(best_v):
            return d.start[best_v] + got
    if any(ctr[v] < d.length(v) for v in range(d.nbins)):
        d.gave_up_early.append(b)
    return -1


def pop_item(d, mode, s, b, mutant):
    if mode == "steal":
        return (yield from pop_with_stealing(d, s & 1, b, mutant))
    if mode == "queue":
        c = yield from atomic_add(d.qhead, s & 1, mutant)
        return c if c < d.nitems else -1
    c = yield from atomic_add(d.s_ctr, b, mutant)
    c += d.start[b]
    return c if c < d.start[b + 1] else -1


def warp(d, mode, s, b, ran, mutant):
    while True:
        item = yield from pop_item(d, mode, s, b, mutant)
        if item < 0:
            return
        ran.append(item)
        yield                                     # the item's work


def reset_next_parity(d, s, b, mutant):
    """Thread 0 of processor b at the start of step s (before __syncthreads)."""
    par = s & 1 if mutant == "reset_current_parity" else (s + 1) & 1
    d.ctr[par][b] = 0
    yield
    if b == 0:
        d.qhead[par] = 0
        yield


def run(lens, warps, mode, nsteps, seed, mutant=None, max_moves=1_000_000):
    """Returns, per step, the sorted list of items run, and the device state."""
    d = Dev(lens)
    rng = random.Random(seed)
    out = []
    for s in range(nsteps):
        for b in range(d.nbins):
            d.s_ctr[b] = 0                        # zeroed before the CTA's __syncthreads
        ran = []
        live = [warp(d, mode, s, b, ran, mutant) for b in range(d.nbins) for _ in range(warps)]
        live += [reset_next_parity(d, s, b, mutant) for b in range(d.nbins)]
        moves = 0
        while live:                               # the grid barrier ends the step
            i = rng.randrange(len(live))
            try:
                next(live[i])
            except StopIteration:
                live.pop(i)
            moves += 1
            assert moves <= max_moves, "a warp did not terminate"
        out.append(sorted(ran))
    return out, d


def instances(n, seed0):
    rng = random.Random(seed0)
    for k in range(n):
        nbins = rng.randint(1, 6)
        lens = [rng.choice([0, 0, 1, 2, 3, 5, 8]) for _ in range(nbins)]
        yield lens, rng.randint(1, 4), 100 + k


@pytest.mark.parametrize("mode", ["table", "queue", "steal"])
def test_every_item_runs_exactly_once_per_step(mode):
    for lens, warps, seed in instances(150, {"table": 1, "queue": 2, "steal": 3}[mode]):
        out, d = run(lens, warps, mode, 4, seed)
        want = list(range(sum(lens)))
        for s, ran in enumerate(out):
            assert ran == want, (mode, lens, warps, seed, s, ran)
        assert not d.gave_up_early, (lens, warps, seed)


def test_stealing_gives_up_only_when_every_counter_has_passed_its_items():
    """One processor holds all the work: every other warp steals from it, and
    the failed steals at its last items never use up the attempt bound."""
    for seed in range(40):
        lens = [0, 0, 0, 0, 0, 0, 13]
        out, d = run(lens, 4, "steal", 3, seed)
        assert all(ran == list(range(13)) for ran in out), seed
        assert not d.gave_up_early, seed


@pytest.mark.parametrize("mode,mutant", [
    ("steal", "reset_current_parity"),
    ("queue", "reset_current_parity"),
    ("table", "non_atomic_pop"),
    ("queue", "non_atomic_pop"),
    ("steal", "non_atomic_pop"),
    ("steal", "short_attempt_bound"),
])
def test_planted_dispatch_mistakes_are_caught(mode, mutant):
    caught = 0
    for lens, warps, seed in instances(150, 7):
        if sum(lens) == 0:
            continue
        out, d = run(lens, max(warps, 2), mode, 4, seed, mutant=mutant)
        want = list(range(sum(lens)))
        caught += any(ran != want for ran in out) or bool(d.gave_up_early)
    assert caught > 0, (mode, mutant)
