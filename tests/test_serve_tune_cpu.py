"""Host-side logic of the serving loop and the autotuner (no GPU): admission
under a memory budget, arrival order, and the convex coordinate descent."""
import math
import threading
import time

import numpy as np
import pytest

from paper_2002_04894_gb300 import serve, tune


class FakeExec:
    """Stand-in executor: sleeps in proportion to the request size and records
    how much reserved memory was in flight."""

    def __init__(self):
        self.lock = threading.Lock()
        self.order = []

    def __call__(self, req, t0):
        with self.lock:
            self.order.append(req.rid)
        time.sleep(0.002 + 1e-7 * len(req.charges))
        return serve.Result(req.rid, np.zeros(1), None, req.arrival, 0.0,
                            time.perf_counter() - t0, 0, 0)


def make_requests(sizes, gap=0.0):
    return [serve.Request(i, np.zeros((n, 3)), np.zeros(n), arrival=i * gap, p=8)
            for i, n in enumerate(sizes)]


def test_admission_respects_budget_and_slots():
    sizes = [20000, 50000, 1000, 300000, 8000, 120000, 4000, 70000]
    need = [serve.plan_bytes(n, serve.default_levels(n), 8) for n in sizes]
    budget = sorted(need)[-2] + sorted(need)[0]      # at most ~two big ones at a time
    res, adm = serve.run_schedule(make_requests(sizes), FakeExec(), budget, slots=3, realtime=False)
    assert [r.rid for r in res] == list(range(len(sizes)))
    assert adm.peak <= max(budget, max(need))
    assert adm.in_use == 0 and adm.active == 0


def test_oversized_request_runs_alone_and_does_not_starve():
    sizes = [1000, 5_000_000, 1000]
    res, adm = serve.run_schedule(make_requests(sizes), FakeExec(), budget=1 << 20, slots=4,
                                  realtime=False)
    assert len(res) == 3 and adm.in_use == 0


def test_arrival_order_and_realtime_admission():
    ex = FakeExec()
    reqs = make_requests([2000] * 6, gap=0.01)
    res, adm = serve.run_schedule(reqs, ex, budget=1 << 40, slots=2, realtime=True)
    assert ex.order == sorted(ex.order)               # admitted in arrival order
    for r in res:
        assert r.admitted >= r.arrival - 1e-3          # never before it arrives


def test_plan_bytes_grows_with_size_and_order():
    assert serve.plan_bytes(10 ** 6, 13, 12) > serve.plan_bytes(10 ** 5, 10, 12)
    assert serve.plan_bytes(10 ** 5, 10, 14) > serve.plan_bytes(10 ** 5, 10, 8)


def test_poisson_arrivals_rate():
    t = serve.poisson_arrivals(20000, 200.0, seed=0)
    assert np.all(np.diff(t) > 0)
    assert t[-1] / 20000 == pytest.approx(1 / 200.0, rel=0.03)


@pytest.mark.parametrize("start", [0, 3, 7, 12, 15])
def test_descend_finds_minimum_of_convex_response(start):
    f = lambda x: (x - 9) ** 2 + 0.5 * abs(x - 9) + 3
    x, best, memo = tune.descend(f, start, 0, 15)
    assert x == 9 and best == 3
    assert len(memo) <= abs(start - 9) + 3            # walks, does not scan


def test_descend_respects_bounds():
    x, _, _ = tune.descend(lambda v: -v, 5, 0, 8)     # monotone: stops at the edge
    assert x == 8


@pytest.mark.parametrize("tol,theta", [(1e-6, 0.5), (1e-4, 0.4), (1e-5, 0.6)])
def test_p_from_bound_meets_the_a_priori_bound(tol, theta):
    ps = tuple(range(2, 40))
    p = tune.p_from_bound(tol, theta, ps)
    assert theta ** (p + 1) / (1 - theta) ** 2 <= tol
    assert theta ** p / (1 - theta) ** 2 > tol        # and is the smallest such p


def test_pick_takes_the_fastest_trial_meeting_the_target():
    C = tune.Config
    trials = [(C(11, 12, 0.5), 5.19, 3.5e-7), (C(12, 12, 0.5), 5.29, 4.0e-7), (C(10, 12, 0.5), 6.24, 2.3e-7),
              (C(11, 12, 0.6), 3.52, 1.1e-5)]
    assert tune.pick(trials, 5e-7)[0] == C(11, 12, 0.5)     # not the most accurate, not the fastest overall
    assert tune.pick(trials, 1e-7)[0] == C(10, 12, 0.5)     # none meets it: the most accurate
    assert tune.pick(trials, 1e-4)[0] == C(11, 12, 0.6)


def test_levels_for_leaf():
    assert tune.levels_for_leaf(2_000_000, 122) == 14
    assert 2 ** tune.levels_for_leaf(100_000, 100) == pytest.approx(1000, rel=0.5)
