"""Host logic of the measure/rebalance loop (paper_1310_4218_gb300/schedule.py),
on the CPU: how a run of time steps is cut into launches at the k_c re-draw
boundaries (the load array C(i,j) changes between segments, Sec. VI-B), and
how many launches a rebalance period takes."""
import random

import pytest

pytest.importorskip("torch")
from paper_1310_4218_gb300.schedule import Schedule  # noqa: E402


def brute_force_segments(t0, t1, epoch_steps):
    """Group the steps t0..t1-1 into maximal runs of equal epoch index."""
    out = []
    for t in range(t0, t1):
        e = t // epoch_steps if epoch_steps else None
        if out and out[-1][2] == e:
            out[-1][1] += 1
        else:
            out.append([t, 1, e])
    return [tuple(s) for s in out]


@pytest.mark.parametrize("epoch_steps", [0, 1, 7, 50])
def test_segments_are_maximal_runs_within_one_kc_epoch(epoch_steps):
    sch = Schedule(None, period=10, epoch_steps=epoch_steps)
    rng = random.Random(epoch_steps)
    for _ in range(300):
        t0 = rng.randint(0, 400)
        t1 = t0 + rng.randint(0, 160)
        got = list(sch._segments(t0, t1))
        assert got == brute_force_segments(t0, t1, epoch_steps), (t0, t1)


def test_launches_per_period():
    # re-draws every 50 steps: a 10-step period never straddles one, a
    # 20-step period starting at 40 does (steps 40-49, then 50-59)
    assert Schedule(None, period=10, epoch_steps=50).launches_per_period(40) == 1
    assert Schedule(None, period=20, epoch_steps=50).launches_per_period(40) == 2
    assert Schedule(None, period=20, epoch_steps=50).launches_per_period(0) == 1
    # steps 30-149: 30-49, 50-99, 100-149; steps 30-159 add 150-159
    assert Schedule(None, period=120, epoch_steps=50).launches_per_period(30) == 3
    assert Schedule(None, period=130, epoch_steps=50).launches_per_period(30) == 4
    assert Schedule(None, period=10, epoch_steps=0).launches_per_period(37) == 1
