"""Host model of the dataflow step schedule (lb_options.dataflow) under
seeded random interleavings of warps.

The dataflow kernel runs a launch's steps without a grid barrier.  Work
items of every step come from one queue (index i = step * nitems + item).
Before running item c at step s, a warp waits until every item in deps(c)
-- the items owning a column of c's closed 4-neighbourhood, c included --
has finished step s - 1 (done[d] >= s): the columns it reads are then
current (read after write), and every item that read c's columns at step
s - 1 has finished, so c may overwrite them in the ping-pong buffer (write
after read).  A warp's finished-item count and global-sum partial for a
step go into that step's slot (of K) when the warp moves on to a later
step or runs out of items; the flush that completes a step reduces it, in
step order, clears the slot and advances `reduced`; a warp starts an item
of step s >= K only once step s - K is reduced.  The warp that reduces
the launch's last step advances the device clock once every CTA has read
it.  A warp publishes its finished item's flag at the start of its next
iteration, before any wait (and at its exit).

The model checks, for every interleaving: each read sees the value of the
step before, no write lands before the previous step's readers are done,
no deadlock, every step reduced once and in order with every item's
contribution, and the clock advanced after every CTA read it.  Planted
protocol mistakes are caught."""
import random

import pytest


def make_grid(nx, ny, run, seed):
    """Columns of an nx x ny periodic grid cut into items: rows of VPs of
    random widths, each VP's columns taken in row-major runs of `run`."""
    rng = random.Random(seed)
    owner = [[-1] * nx for _ in range(ny)]
    items = []
    y = 0
    while y < ny:
        h = min(rng.randint(1, 3), ny - y)
        x = 0
        while x < nx:
            w = min(rng.randint(1, 5), nx - x)
            cols = [(i, j) for j in range(y, y + h) for i in range(x, x + w)]
            for k in range(0, len(cols), run):
                items.append(cols[k:k + run])
            x += w
        y += h
    for c, cols in enumerate(items):
        for (i, j) in cols:
            owner[j][i] = c
    deps, reads = [], []
    for c, cols in enumerate(items):
        nb = set()
        rd = set()
        for (i, j) in cols:
            for (di, dj) in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = (i + di) % nx, (j + dj) % ny
                nb.add(owner[jj][ii])
                rd.add((ii, jj))
        deps.append(sorted(nb))
        reads.append(sorted(rd))
    return items, deps, reads


class Model:
    def __init__(self, items, deps, reads, nsteps, K, nwarps, wpc, seed, mistake=None):
        self.items, self.deps, self.reads = items, deps, reads
        self.n, self.nsteps, self.K = len(items), nsteps, K
        self.mistake = mistake
        self.rng = random.Random(seed)
        self.qhead = 0
        self.done = [0] * self.n
        self.cnt = [0] * K
        self.mass = [[] for _ in range(K)]
        self.reduced = 0
        self.started = 0
        self.ncta = (nwarps + wpc - 1) // wpc
        self.clock_read = [False] * self.ncta
        self.clock_advanced = False
        self.hist = []
        cells = {c for cols in items for c in cols}
        # version[b][cell]: the step whose output buffer b holds (0: the input)
        self.version = [{x: 0 for x in cells}, {x: -1 for x in cells}]
        # readers of each cell at each step still to read it
        self.readers = {}
        for c, rd in enumerate(reads):
            for x in rd:
                self.readers.setdefault(x, []).append(c)
        self.pending = {}
        self.warps = [self.warp(w, w // wpc, w % wpc == 0) for w in range(nwarps)]

    def pending_reads(self, s, x):
        return self.pending.setdefault((s, x), len(self.readers[x]))

    # -- one warp; yields True after progress, False while spinning
    def warp(self, w, cta, first):
        if first:
            self.clock_read[cta] = True          # every CTA reads the clock first
            yield True
            self.started += 1
            yield True
        cur_s, my_cnt, my_mass = -1, 0, []
        pend = None                              # finished item, flag not yet published
        while True:
            i = self.qhead
            self.qhead += 1
            yield True
            if i >= self.nsteps * self.n:
                if pend is not None:
                    self.done[pend[0]] = pend[1] + 1
                    yield True
                yield from self.flush(cur_s, my_cnt, my_mass)
                return
            s, c = divmod(i, self.n)
            if pend is not None and self.mistake != "publish_after_waits":
                self.done[pend[0]] = pend[1] + 1   # before any wait
                pend = None
                yield True
            if s != cur_s and self.mistake != "flush_after_waits":
                yield from self.flush(cur_s, my_cnt, my_mass)
                cur_s, my_cnt, my_mass = s, 0, []
            if s >= self.K and self.mistake != "no_slot_wait":
                while self.reduced < s - self.K + 1:
                    yield False
            deps = self.deps[c]
            if self.mistake == "no_self_dep":
                deps = [d for d in deps if d != c]
            if self.mistake == "upwind_only":
                deps = deps[: max(1, len(deps) // 2)]
            for d in deps:
                while self.done[d] < s:
                    yield False
            if s != cur_s:                       # the late flush of the planted mistake
                yield from self.flush(cur_s, my_cnt, my_mass)
                cur_s, my_cnt, my_mass = s, 0, []
            if pend is not None:                 # the late publication of the planted mistake
                self.done[pend[0]] = pend[1] + 1
                pend = None
                yield True
            # read phase: every read cell holds step s's input, not yet overwritten
            src = s & 1
            for x in self.reads[c]:
                assert self.version[src][x] == s, ("stale or overwritten read", s, c, x)
                self.pending[(s, x)] = self.pending_reads(s, x) - 1
            yield True
            # write phase: no reader of the previous step still needs the old value
            dst = src ^ 1
            for x in self.items[c]:
                if s >= 1:
                    assert self.pending_reads(s - 1, x) == 0, ("write before read", s, c, x)
                self.version[dst][x] = s + 1
            yield True
            pend = (c, s)                        # published at the next iteration
            my_cnt += 1
            my_mass.append((s, c))
            yield True

    def flush(self, s, cnt, mass):
        if s < 0 or cnt == 0:
            return
        slot = s % self.K
        self.mass[slot].extend(mass)
        yield True
        prev = self.cnt[slot]
        self.cnt[slot] = prev + cnt
        yield True
        if prev + cnt == self.n:
            if self.mistake != "unordered_reduce":
                while self.reduced != s:
                    yield False
            got = sorted(self.mass[slot])
            assert got == [(s, c) for c in range(self.n)], ("incomplete step", s)
            self.hist.append(s)
            self.mass[slot] = []
            self.cnt[slot] = 0
            yield True
            if s == self.nsteps - 1:
                if self.mistake != "early_clock":
                    while self.started != self.ncta:
                        yield False
                assert all(self.clock_read), "clock advanced before every CTA read it"
                self.clock_advanced = True
            self.reduced = max(self.reduced, s + 1)
            yield True

    def run(self, max_idle=50000):
        # per-warp weights: some warps lag far behind the others, as a warp
        # of a CTA that starts late or keeps losing its issue slots would
        weight = {id(g): self.rng.choice([1.0, 1.0, 1.0, 0.01]) for g in self.warps}
        live = list(self.warps)
        idle = 0
        while live:
            g = self.rng.choices(live, weights=[weight[id(x)] for x in live])[0]
            try:
                progressed = next(g)
            except StopIteration:
                live.remove(g)
                idle = 0
                continue
            idle = 0 if progressed else idle + 1
            if idle > max_idle:
                raise AssertionError("deadlock")
        assert self.hist == list(range(self.nsteps)), ("steps reduced", self.hist)
        assert self.clock_advanced
        assert all(d == self.nsteps for d in self.done)


@pytest.mark.parametrize("seed", range(60))
def test_dataflow_schedule_is_safe_and_live(seed):
    items, deps, reads = make_grid(9, 7, 4, seed)
    m = Model(items, deps, reads, nsteps=6, K=2, nwarps=6, wpc=2, seed=seed)
    m.run()


@pytest.mark.parametrize("seed", range(20))
def test_one_slot_and_long_grids(seed):
    """K = 1 (a step's slot is reused by the next step) on a grid long in x,
    where far-apart items may run steps apart."""
    items, deps, reads = make_grid(24, 3, 3, seed)
    m = Model(items, deps, reads, nsteps=5, K=1, nwarps=8, wpc=2, seed=seed)
    m.run()


@pytest.mark.parametrize("mistake", ["no_self_dep", "upwind_only", "no_slot_wait",
                                     "unordered_reduce", "early_clock", "flush_after_waits",
                                     "publish_after_waits"])
def test_planted_protocol_mistakes_are_caught(mistake):
    caught = 0
    shapes = [((9, 7, 4), 2), ((24, 3, 3), 1), ((24, 3, 3), 2)]
    for seed in range(90):
        (nx, ny, run), K = shapes[seed % 3]
        items, deps, reads = make_grid(nx, ny, run, seed)
        m = Model(items, deps, reads, nsteps=6, K=K, nwarps=8, wpc=2, seed=1000 + seed,
                  mistake=mistake)
        try:
            m.run()
        except AssertionError:
            caught += 1
    assert caught > 0, mistake
