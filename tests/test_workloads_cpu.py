"""The seeded synthetic workloads have the sizes and structure of the five
measured configurations (grids, inputs, windows, horizons, the served
stream's ranges), and the same seed gives the same problems."""
import math

import numpy as np

import oracle
import workloads as W


def test_robot_lin_sizes():
    w = W.robot_lin()
    p = w.problem
    assert p.x_count == [41, 41] and p.n_states == 1681
    assert p.u_count == [5, 5] and p.n_inputs == 25
    assert p.sigma == [0.2, 0.2] and p.gamma == 0.0 and p.window is None   # dense rows
    assert w.horizon == 8 and w.spec.kind == W.REACH_AVOID


def test_unicycle_sizes_and_window():
    w = W.unicycle()
    p = w.problem
    assert p.x_count == [51, 51, 30] and p.n_states == 78030 and p.x_periodic == [0, 0, 1]
    assert p.n_inputs == 45 and w.horizon == 32 and w.spec.kind == W.REACH
    Wd, _ = oracle.window_shape(p)
    assert list(Wd) == [3, 3, 3]   # sigma 0.05, gamma 1e-6


def test_rooms7_and_traffic6_sizes():
    r = W.rooms7()
    assert r.problem.x_count == [9] * 7 and r.problem.n_states == 9 ** 7 == 4782969
    assert r.problem.n_inputs == 5 and r.problem.window == [3] * 7 and r.horizon == 10
    assert r.spec.kind == W.SAFETY
    t = W.traffic6()
    assert t.problem.x_count == [21] * 6 and t.problem.n_states == 21 ** 6 == 85766121
    assert t.problem.n_inputs == 4 and t.problem.window == [5] * 6 and t.horizon == 8
    assert t.problem.sigma == [0.5] * 6 and t.spec.kind == W.SAFETY


def test_served_stream_ranges_and_seed():
    reqs = W.served_stream(256)
    assert len(reqs) == 256
    dims = {w.problem.n for w in reqs}
    assert dims == {2, 3, 4}
    per_dim = {2: 20, 3: 17, 4: 15}
    for w in reqs:
        p = w.problem
        assert p.x_count == [per_dim[p.n]] * p.n
        assert 4 <= p.n_inputs <= 16
        assert 5 <= w.horizon <= 50
        assert p.gamma == 1e-3
        # the diagonal covariance entries lie in [0.05, 0.3]; sigma is their root
        assert all(math.sqrt(0.05) - 1e-12 <= s <= math.sqrt(0.3) + 1e-12 for s in p.sigma)
        assert w.spec.kind in (W.SAFETY, W.REACH_AVOID)
    kinds = [w.spec.kind for w in reqs]
    assert 0.3 < kinds.count(W.SAFETY) / len(kinds) < 0.7
    again = W.served_stream(256)
    assert all(np.array_equal(a.problem.params, b.problem.params) and a.horizon == b.horizon
               for a, b in zip(reqs, again))


def test_poisson_arrivals_rate():
    t = W.poisson_arrivals(4000, 100.0)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 100.0) < 10.0
