"""Host logic of the serving stream (no GPU): the seeded request recipe of
config 5 and the work per request that sets the arrival rate of the
full-scale run."""
import numpy as np

from paper_1505_03271_gb300 import serving


def test_request_recipe_is_seeded_and_in_range():
    a = serving.make_requests(200, 2.0, 1000, 20000)
    b = serving.make_requests(200, 2.0, 1000, 20000)
    assert [(r.n, r.Ra, r.nsteps, r.arrival) for r in a] == [(r.n, r.Ra, r.nsteps, r.arrival) for r in b]
    assert all(r.n in serving.SIZES for r in a)
    assert all(1000 <= r.nsteps <= 20000 for r in a)
    assert all(1e4 <= r.Ra <= 1e8 for r in a)
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals at 2 per second: mean gap 0.5 s within sampling error
    assert abs(np.diff(t).mean() - 0.5) < 0.1
    assert {r.rid for r in a} == set(range(1, 201))


def test_mean_work_per_request():
    """E[N^2] E[steps] for N uniform on the five sizes and steps uniform on
    [lo, hi]: 279,347.2 cells x 10,500 steps for the configured stream."""
    sizes = serving.SIZES
    expect = sum(n * n for n in sizes) / len(sizes) * (1000 + 20000) / 2
    assert serving.mean_work() == expect
    assert abs(serving.mean_work() / 2.9331456e9 - 1) < 1e-9
