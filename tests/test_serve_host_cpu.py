"""Host logic of the request server that needs no GPU: the seeded Poisson
workload generator and the scale count used for admission estimates."""
import math

import numpy as np

from paper_1308_5706_gb300 import serve


def test_poisson_workload_invariants():
    reqs = serve.poisson_workload(rate=200.0, duration=5.0, seed=4)
    assert 700 < len(reqs) < 1300  # about rate x duration arrivals
    arrivals = [r.arrival for r in reqs]
    assert all(0.0 < a < 5.0 for a in arrivals)
    assert arrivals == sorted(arrivals)
    assert [r.rid for r in reqs] == list(range(len(reqs)))
    consumed = set()
    for r in reqs:
        assert 1 <= r.N <= r.L and r.lam in (2.0, 3.0)
        if r.kind == "analysis":
            assert 32 <= r.L <= 2048 and r.parent is None
        else:
            assert r.kind == "synthesis"
            par = reqs[r.parent]
            # a synthesis consumes an earlier analysis of the same configuration, once
            assert par.kind == "analysis" and par.arrival < r.arrival
            assert (par.L, par.N, par.lam) == (r.L, r.N, r.lam)
            assert r.parent not in consumed
            consumed.add(r.parent)
    kinds = [r.kind for r in reqs]
    assert 0.3 < kinds.count("synthesis") / len(kinds) < 0.5


def test_poisson_workload_is_seeded():
    a = serve.poisson_workload(rate=100.0, duration=2.0, seed=7)
    b = serve.poisson_workload(rate=100.0, duration=2.0, seed=7)
    c = serve.poisson_workload(rate=100.0, duration=2.0, seed=8)
    key = lambda rs: [(r.kind, r.L, r.N, r.lam, r.arrival, r.seed, r.parent) for r in rs]
    assert key(a) == key(b)
    assert key(a) != key(c)


def test_poisson_workload_fixed_band_limits_and_rate():
    Ls = (64, 128, 256)
    reqs = serve.poisson_workload(rate=400.0, duration=20.0, seed=1, Ls=Ls, N_range=(3, 3), lams=(2.0,))
    assert {r.L for r in reqs} == set(Ls) and {r.N for r in reqs} == {3}
    # inter-arrival times of a Poisson process: mean 1/rate, coefficient of variation 1
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() * 400.0 - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def test_jmax_is_the_smallest_exponent_reaching_L():
    for L in (2, 3, 16, 17, 100, 1024, 2048):
        for lam in (1.3, 1.7, 2.0, 3.0):
            J = serve.B_jmax(L, lam)
            assert lam ** J >= L * (1 - 1e-12)
            assert J == 0 or lam ** (J - 1) < L
            assert J == max(0, math.ceil(math.log(L) / math.log(lam) - 1e-12))
