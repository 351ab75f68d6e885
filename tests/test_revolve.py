"""Host-side checks of the binomial checkpointing plan behind the discrete
adjoint (no GPU): its forward-step count equals both the closed form of
Griewank's revolve and an exhaustive dynamic program over all split points,
and the plan, executed symbolically, reverses every step exactly once in
order n-1 .. 0 with the right state in hand and never more slots than given."""
from functools import lru_cache
from math import comb

import numpy as np
import pytest

import paper_2502_09714_gb300 as dgpkg


@pytest.fixture(scope="module", autouse=True)
def lib():
    dgpkg.build()
    return dgpkg.load_library()


@lru_cache(None)
def _dp(n, s):
    """Least forward steps to reverse n steps with s free slots besides the
    retained start, by trying every first split point."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + _dp(n - m, s - 1) + _dp(m, s) for m in range(1, n))


def _closed(n, snapshots):
    s = snapshots - 1
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    t = 0
    while comb(s + 1 + t, t) < n:
        t += 1
    return t * n - comb(s + 1 + t, t - 1)


def _execute(n, snapshots, acts):
    slots = {0: 0}
    cur = None
    done = []
    advanced = 0
    for kind, a, b in acts.tolist():
        if kind == 0:                      # advance a -> b
            assert cur == a and b > a
            advanced += b - a
            cur = b
        elif kind == 1:                    # store slot a <- step b
            assert cur == b and 0 < a < snapshots
            slots[a] = b
        elif kind == 2:                    # restore slot a (step b)
            assert slots.get(a) == b
            cur = b
        else:                              # adjoint of step a
            assert cur == a
            done.append(a)
    assert done == list(range(n - 1, -1, -1))
    assert len(slots) <= snapshots
    return advanced


@pytest.mark.parametrize("snapshots", [1, 2, 3, 5, 8])
def test_cost_matches_closed_form_and_exhaustive_search(snapshots):
    for n in range(1, 70):
        c = dgpkg.revolve_cost(n, snapshots)
        assert c == _closed(n, snapshots) == _dp(n, snapshots - 1), (n, snapshots)


@pytest.mark.parametrize("n,snapshots", [(1, 1), (7, 1), (10, 3), (33, 4), (100, 6), (257, 9), (800, 40),
                                           (800, 801), (1500, 2), (16384, 10), (5000, 4096)])
def test_plan_reverses_every_step_once(n, snapshots):
    fw, acts = dgpkg.revolve_plan(n, snapshots)
    assert fw == dgpkg.revolve_cost(n, snapshots)
    assert _execute(n, snapshots, acts) == fw


def test_adjoint_workload_plan():
    """800 steps with 40 snapshots: C(42, 2) = 861 >= 800 steps at two
    repetitions, 2 x 800 - C(42, 1) = 1558 forward steps."""
    fw, _ = dgpkg.revolve_plan(800, 40)
    assert fw == 1558


def test_plan_rejects_bad_arguments():
    with pytest.raises(dgpkg.DGError):
        dgpkg.revolve_plan(0, 3)
    with pytest.raises(dgpkg.DGError):
        dgpkg.revolve_plan(10, 0)
    with pytest.raises(dgpkg.DGError):
        dgpkg.revolve_plan(1 << 20, 1)           # n (n - 1) / 2 forward steps: refused
    assert dgpkg.revolve_cost(0, 3) == -1
    assert np.isfinite(dgpkg.revolve_cost(1 << 20, 40))
