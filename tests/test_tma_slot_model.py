"""Host model of the TMA-staged step kernel's slot protocol, run on the CPU.

The model restates the item loop of `lb_step_kernel_tma`
(paper_1310_4218_gb300/csrc/lb_step_tma.cuh: `start_item`, `process_item_box`,
`mbar_wait`).  Each warp owns one shared-memory slot and one mbarrier
(arrival count 1).  For a boxed item, lane 0 arms the barrier with the box's
byte count (arrive.expect_tx) and issues the tensor copy, which signals
complete_tx on landing.  The warp waits on the parity of the copy's phase, then
flips its phase bit.  It reads the box into registers, and only then (its
`loaded()` hook) pops the next item and issues that copy into the same slot.
Items whose tile wraps the periodic boundary are not boxed: they read global
memory and call `loaded()` first.  At the end of the launch, a copy still in
flight is waited for.

The warp and the copy engine are generators that a seeded scheduler
interleaves.  A copy lands at a random later move, or a fixed number of clock
ticks after its issue.  The clock counts scheduler moves, and a wait gives up
after a limit on it, as the kernel's waits do on globaltimer.  The mbarrier
follows the
PTX rules.  A phase completes when its pending arrival count and its
transaction count are both zero.  try_wait.parity(P) is true once the phase of
parity P has completed, that is while the current phase's parity is not P.

Checked over many interleavings and item mixes:
- every read of the slot sees the box of the item being processed;
- no copy lands in the slot while the warp is reading it;
- no copy is in flight when the warp exits;
- every wait ends in time.
Planted mistakes (no phase flip after a wait, issuing the next copy before
the box is read, no wait at exit) must each be caught.
"""
import random

import pytest

BOX_BYTES = 12 * 3 * 96 * 4
READ_CHUNKS = 3                 # the box is read in several instructions


class Bar:
    """mbarrier with one expected arrival per phase."""

    def __init__(self):
        self.phase, self.pending, self.tx = 0, 1, 0

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.pending -= 1
        self._complete()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._complete()

    def _complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = 1

    def try_wait_parity(self, parity):
        return (self.phase & 1) != parity


class World:
    def __init__(self):
        self.bar = Bar()
        self.slot = None          # item whose box the slot holds
        self.reading = False
        self.in_flight = []       # issued copies (item id, issue time), oldest first
        self.clock = 0            # scheduler moves (the kernel reads globaltimer)
        self.violations = []
        self.warp_done = False
        self.timed_out = False


def start_item(w, item):
    """Returns (item id or None, boxed)."""
    if item is None:
        return None, 0
    c, boxed = item
    if not boxed:
        return c, 0
    w.bar.arrive_expect_tx(BOX_BYTES)           # lane 0 arms, then issues the copy
    w.in_flight.append((c, w.clock))
    yield
    return c, 1


def mbar_wait(w, parity, limit):
    t0 = w.clock
    while not w.bar.try_wait_parity(parity):
        if w.clock - t0 > limit:
            return False
        yield
    return True


def read_box(w, c):
    w.reading = True
    for _ in range(READ_CHUNKS):
        if w.slot != c:
            w.violations.append(("read of another box", c, w.slot))
        yield
    w.reading = False


def warp(w, steps, limit, mutant):
    phase, pending = 0, 0
    for items in steps:
        src = iter(items)
        cur = yield from start_item(w, next(src, None))
        pending = cur[1]
        while cur[0] is not None:
            c, boxed = cur
            if boxed:
                if not (yield from mbar_wait(w, phase, limit)):
                    w.timed_out = True
                    break
                if mutant != "no_phase_flip":
                    phase ^= 1
                pending = 0
                if mutant == "issue_before_read":
                    nxt = yield from start_item(w, next(src, None))
                yield from read_box(w, c)
                if mutant != "issue_before_read":
                    nxt = yield from start_item(w, next(src, None))   # loaded()
            else:
                nxt = yield from start_item(w, next(src, None))       # loaded() first
            yield                                                     # the solves
            pending = nxt[1]
            cur = nxt
        if w.timed_out:
            break
    if pending and mutant != "no_exit_wait":
        yield from mbar_wait(w, phase, limit)
    if w.in_flight:
        w.violations.append(("copy in flight at exit", list(w.in_flight)))
    w.warp_done = True


def engine(w, rng, p_land, delay):
    """Lands the oldest copy with probability p_land per move, or (delay set)
    exactly `delay` clock ticks after its issue."""
    while not w.warp_done:
        if w.in_flight and (w.clock - w.in_flight[0][1] >= delay if delay is not None
                            else rng.random() < p_land):
            c, _ = w.in_flight.pop(0)
            if w.reading:
                w.violations.append(("copy landed during reads", c))
            w.slot = c
            w.bar.complete_tx(BOX_BYTES)
        yield


def run(steps, seed, mutant=None, limit=10_000, p_land=0.3, delay=None, max_moves=1_000_000):
    w = World()
    rng = random.Random(seed)
    live = [warp(w, steps, limit, mutant), engine(w, random.Random(seed + 7), p_land, delay)]
    moves = 0
    while live:
        i = rng.randrange(len(live))
        try:
            next(live[i])
        except StopIteration:
            live.pop(i)
        moves += 1
        w.clock += 1
        assert moves <= max_moves, "the model did not terminate"
    return w


def item_mix(seed, nsteps=3, p_boxed=0.8):
    rng = random.Random(500 + seed)
    steps, c = [], 0
    for _ in range(nsteps):
        items = []
        for _ in range(rng.randint(0, 7)):
            items.append((c, 1 if rng.random() < p_boxed else 0))
            c += 1
        steps.append(items)
    return steps


@pytest.mark.parametrize("p_land", [0.05, 0.3, 0.9])
def test_every_read_sees_its_own_landed_box(p_land):
    for seed in range(200):
        w = run(item_mix(seed), seed, p_land=p_land)
        assert not w.violations, (seed, w.violations[:3])
        assert not w.timed_out and not w.in_flight, seed


def test_boxed_and_global_items_alternate_safely():
    """Runs of boxed items, wrap tiles in between, and empty steps."""
    for seed in range(100):
        for p_boxed in (0.0, 0.5, 1.0):
            w = run(item_mix(seed, nsteps=4, p_boxed=p_boxed), seed)
            assert not w.violations and not w.timed_out, (seed, p_boxed, w.violations[:3])


def test_phases_alternate_strictly_with_the_warps_items():
    """The barrier completes one phase per boxed item, so the warp's phase
    bit always names the copy it waits for."""
    steps = [[(n, 1) for n in range(9)], [(9, 1), (10, 0), (11, 1)]]
    w = run(steps, 3)
    assert not w.violations
    assert w.bar.phase == 11 and w.bar.pending == 1 and w.bar.tx == 0


def test_after_a_time_limit_the_copy_in_flight_lands_before_exit():
    """A copy that lands between one and two time limits after its issue: the
    warp's wait gives up (LB_ETIMEOUT in the kernel), and the wait at exit
    still sees the copy land, so none is in flight when the warp exits."""
    limit = 200
    for seed in range(50):
        w = run([[(0, 1), (1, 1)]], seed, limit=limit, delay=3 * limit // 2)
        assert w.timed_out and not w.violations, (seed, w.violations)


@pytest.mark.parametrize("mutant", ["no_phase_flip", "issue_before_read"])
def test_planted_slot_protocol_mistakes_are_caught(mutant):
    caught = 0
    for seed in range(100):
        w = run(item_mix(seed), seed, mutant=mutant)
        caught += bool(w.violations)
    assert caught > 0, mutant


def test_planted_missing_exit_wait_is_caught():
    limit = 200
    for seed in range(20):
        w = run([[(0, 1), (1, 1)]], seed, mutant="no_exit_wait", limit=limit,
                delay=3 * limit // 2)
        assert any(v[0] == "copy in flight at exit" for v in w.violations), seed
