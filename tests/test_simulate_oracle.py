"""Pins of the oracle's closed-loop simulator (the Monte-Carlo validation of
Sec. 7: the synthesized controller run from initial states on the abstract
MDP) and of its counter-based generator.

The generator is checked against numpy's independent Philox4x64-10, the
simulator against what the value function fixes: the success frequency of
N runs is Binomial(N, V_0(x0)) under the synthesized policy, so it lies
within 4 binomial standard deviations of V_0; with a disturbance player
drawn at random the worst-case value is a lower bound; absorbing states and
the empty horizon give exact counts.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W


def _ctr_plus_one(c):
    c = [int(v) for v in c]
    for i in range(4):
        c[i] = (c[i] + 1) % 2**64
        if c[i]:
            break
    return c


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 9, 1], [123, 456]),
    ([2**64 - 1, 2**64 - 1, 3, 0], [2**63 + 5, 17]),       # carry across two words
    ([2**64 - 1] * 3 + [41], [2**64 - 1, 2**64 - 1]),     # carry into the last word
    ([12345, 0, 0, 0], [0x9E3779B97F4A7C15, 1]),
])
def test_philox_matches_numpy(ctr, key):
    """numpy's Philox returns, for counter c, the block of counter c + 1."""
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4).astype(np.uint64)
    assert np.array_equal(ref, oracle.philox4x64(_ctr_plus_one(ctr), key))


def test_philox_stream_matches_numpy():
    """Twenty consecutive blocks from one key: a shifted counter changes every word."""
    key = [2024, 7]
    bg = np.random.Philox(counter=np.zeros(4, np.uint64), key=np.array(key, np.uint64))
    ref = bg.random_raw(80).astype(np.uint64).reshape(20, 4)
    for i in range(20):
        assert np.array_equal(ref[i], oracle.philox4x64([i + 1, 0, 0, 0], key))


def _coarse_robot():
    w = W.robot_lin(n_per_dim=17, horizon=6)
    w.problem.x_eta = [10.0 / 16, 10.0 / 16]
    return w


def _binomial_z(counts, runs, V):
    fr = counts / runs
    sd = np.sqrt(np.maximum(V * (1 - V), 1e-300) / runs)
    return (fr - V) / sd


def test_simulated_frequency_matches_value_reach_avoid():
    w = _coarse_robot()
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    cand = [x for x in range(p.n_states) if mask[x] == 4 and 0.05 < r["V"][x] < 0.95]
    rng = np.random.default_rng(W.SEED)
    x0 = [cand[i] for i in rng.choice(len(cand), size=10, replace=False)]
    runs = 100_000
    c = oracle.simulate(p, s, w.horizon, r["pi"], x0, runs, seed=11)
    z = _binomial_z(c, runs, r["V"][x0])
    assert np.all(np.abs(z) < 4.0), z


def test_simulated_frequency_matches_value_safety_truncated():
    """Safety with a cut window (gamma > 0): the truncated mass loses runs,
    as it lowers V."""
    rng = np.random.default_rng(5)
    w = W.random_affine(rng, 2, [21, 19], 4, gamma=2e-2, kind=W.SAFETY, horizon=5)
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    x0 = [x for x in np.argsort(np.abs(r["V"] - 0.5))[:8]]
    runs = 50_000
    c = oracle.simulate(p, s, w.horizon, r["pi"], x0, runs, seed=3)
    z = _binomial_z(c, runs, r["V"][x0])
    assert np.all(np.abs(z) < 4.0), (z, r["V"][x0])


def test_simulated_frequency_three_dims_periodic():
    rng = np.random.default_rng(8)
    w = W.random_affine(rng, 3, [9, 8, 10], 3, gamma=1e-2, kind=W.REACH_AVOID, horizon=4, periodic=[0, 1, 0])
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    free = np.flatnonzero((mask == 4) & (r["V"] > 0.02) & (r["V"] < 0.98))
    x0 = list(free[:: max(1, len(free) // 8)][:8])
    runs = 40_000
    c = oracle.simulate(p, s, w.horizon, r["pi"], x0, runs, seed=99)
    z = _binomial_z(c, runs, r["V"][x0])
    assert np.all(np.abs(z) < 4.0), z


def test_random_disturbance_is_no_worse_than_the_game_value():
    """The policy secures V_0 against every disturbance sequence; drawn at
    random the disturbance does no worse, so frequencies stay above
    V_0 - 4 sd (and on the robot of Sec. 7 strictly above on average)."""
    w = W.robot_dist(horizon=5)
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    x0 = [x for x in np.argsort(np.abs(r["V"] - 0.5))[:6]]
    runs = 20_000
    c = oracle.simulate(p, s, w.horizon, r["pi"], x0, runs, seed=4)
    z = _binomial_z(c, runs, r["V"][x0])
    assert np.all(z > -4.0), z
    assert float(np.mean(c / runs - r["V"][x0])) > 0.0


def test_absorbing_states_and_empty_horizon_exact():
    w = _coarse_robot()
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    tgt, avd = int(np.flatnonzero(mask & 1)[0]), int(np.flatnonzero(mask & 2)[0])
    c = oracle.simulate(p, s, w.horizon, r["pi"], [tgt, avd], 1000, seed=1)
    assert list(c) == [1000, 0]
    # horizon 0: reach succeeds exactly on the target
    free = int(np.flatnonzero(mask == 4)[0])
    c0 = oracle.simulate(p, s, 0, np.zeros((0, p.n_states), np.uint16), [tgt, avd, free], 10, seed=1)
    assert list(c0) == [10, 0, 0]
    # safety, horizon 0: every safe state succeeds, the rest fail
    rng = np.random.default_rng(5)
    ws = W.random_affine(rng, 2, [21, 19], 4, gamma=2e-2, kind=W.SAFETY, horizon=5)
    ms = oracle.spec_mask(ws.problem, ws.spec)
    xs = [int(np.flatnonzero(ms & 4)[0]), int(np.flatnonzero((ms & 4) == 0)[0])]
    c1 = oracle.simulate(ws.problem, ws.spec, 0, np.zeros((0, ws.problem.n_states), np.uint16), xs, 7, seed=2)
    assert list(c1) == [7, 0]


def test_one_step_reach_counts_follow_the_row():
    """Horizon 1, the target one cell: a run succeeds exactly when its draw
    lands there, so the count is Binomial(N, T(target | x, pi_0(x)))."""
    p = dataclasses.replace(_coarse_robot().problem)
    x = 8 * 17 + 8
    spec = W.Spec(W.REACH_AVOID, targets=[([p.x_lb[0] + 9 * p.x_eta[0]] * 2, [p.x_lb[0] + 9 * p.x_eta[0]] * 2)],
                  avoids=[])
    r = oracle.synthesize(p, spec, 1)
    u = int(r["pi"][0, x])
    origin, probs = oracle.row(p, x, u)
    Wd, _ = oracle.window_shape(p)
    k = (9 - origin[0]) * Wd[1] + (9 - origin[1])
    pr = float(probs[k])
    assert pr == pytest.approx(r["V"][x], rel=1e-12)
    runs = 200_000
    c = oracle.simulate(p, spec, 1, r["pi"], [x], runs, seed=21)
    assert abs(c[0] / runs - pr) < 4.0 * np.sqrt(pr * (1 - pr) / runs)


def test_seeds_are_deterministic_and_distinct():
    w = _coarse_robot()
    p, s = w.problem, w.spec
    r = oracle.synthesize(p, s, w.horizon)
    x0 = [int(np.argmin(np.abs(r["V"] - 0.5)))]
    a = oracle.simulate(p, s, w.horizon, r["pi"], x0 * 3, 5000, seed=8)
    b = oracle.simulate(p, s, w.horizon, r["pi"], x0 * 3, 5000, seed=8)
    c = oracle.simulate(p, s, w.horizon, r["pi"], x0 * 3, 5000, seed=9)
    assert np.array_equal(a, b)
    assert len(set(a.tolist())) > 1           # different runs (run index in the counter)
    assert not np.array_equal(a, c)


def test_simulate_rejects_bad_states():
    w = _coarse_robot()
    r = oracle.synthesize(w.problem, w.spec, 2)
    with pytest.raises(ValueError):
        oracle.simulate(w.problem, w.spec, 2, r["pi"], [w.problem.n_states], 10, seed=1)
