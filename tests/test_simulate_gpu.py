"""GPU parity of the closed-loop simulator (the Monte-Carlo validation of
Sec. 7) through the C ABI: the CUDA runs against the oracle's runs on the
same policy, seed and initial states.

Both sides draw from Philox4x64-10 at the same counters and walk the same
FP64 cell masses in window order, so the success counts agree run for run;
the masses differ by rounding (two erfc implementations), which can flip a
run only when a draw falls within ~1e-15 of a cumulative mass boundary, so
the tests allow a total count difference of 2 per comparison.  The GPU's own
policy is checked against the oracle's V_0 by binomial bounds."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import load_engine

pytestmark = pytest.mark.gpu

FLIP = 2


@pytest.fixture(scope="module")
def amy():
    return load_engine()


def _starts(V, mask, k, lo=0.05, hi=0.95):
    """Up to k initial states whose value is neither near 0 nor near 1 (the
    states nearest V = 1/2 when there are none)."""
    idx = np.flatnonzero((mask & 4).astype(bool) & ((mask & 3) == 0) & (V > lo) & (V < hi))
    if idx.size == 0:
        idx = np.argsort(np.abs(V - 0.5))[:k]
    return [int(v) for v in idx[:: max(1, idx.size // k)][:k]]


def _coarse_robot():
    w = W.robot_lin(n_per_dim=17, horizon=6)
    w.problem.x_eta = [10.0 / 16, 10.0 / 16]
    return w


def _same_counts(amy, w, runs, seed, tmode="otf", prec="fp64", k=8):
    p, s = w.problem, w.spec
    ref = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    x0 = _starts(ref["V"], mask, k)
    want = oracle.simulate(p, s, w.horizon, ref["pi"], x0, runs, seed)
    with amy.amy_build(p, tmode=tmode, prec=prec) as h:
        got = amy.amy_simulate(h, s, w.horizon, ref["pi"], x0, runs, seed)
    assert int(np.abs(got - want).sum()) <= FLIP, (got, want)
    return x0, got, ref


def test_counts_match_oracle_robot_reach_avoid(amy):
    _same_counts(amy, _coarse_robot(), 20_000, seed=5)


@pytest.mark.parametrize("tmode,prec", [("stored_separable", "fp32"), ("stored_full", "fp64")])
def test_counts_do_not_depend_on_the_handle_mode(amy, tmode, prec):
    """The simulator computes its FP64 rows itself, so any handle of the
    problem gives the same counts."""
    _same_counts(amy, _coarse_robot(), 10_000, seed=6, tmode=tmode, prec=prec)


def test_counts_match_oracle_safety_truncated(amy):
    rng = np.random.default_rng(5)
    _same_counts(amy, W.random_affine(rng, 2, [21, 19], 4, gamma=2e-2, kind=W.SAFETY, horizon=5), 20_000, seed=3)


def test_counts_match_oracle_three_dims_periodic(amy):
    rng = np.random.default_rng(8)
    w = W.random_affine(rng, 3, [9, 8, 10], 3, gamma=1e-2, kind=W.REACH_AVOID, horizon=4, periodic=[0, 1, 0])
    _same_counts(amy, w, 10_000, seed=99)


def test_counts_match_oracle_disturbed_robot(amy):
    """The robot of Sec. 7 with its disturbance: the disturbance point is
    drawn uniformly each step (draw n), then the dims."""
    _same_counts(amy, W.robot_dist(horizon=5), 5_000, seed=4, tmode="otf", prec="fp32", k=6)


@pytest.mark.parametrize("kind,prm", [
    ("uniform", lambda n: [[0.45] * n]),
    ("beta", lambda n: [[2.0] * n, [3.0] * n, [-0.5] * n, [0.7] * n]),
    ("exponential", lambda n: [[3.0] * n]),
])
def test_counts_match_oracle_noise_kinds(amy, kind, prm):
    rng = np.random.default_rng(71)
    w = W.random_affine(rng, 2, [31, 27], 3, gamma=2e-2 if kind != "beta" else 1e-2, kind=W.REACH_AVOID,
                        horizon=4)
    p = dataclasses.replace(w.problem, noise=kind, noise_params=prm(2))
    _same_counts(amy, W.with_sizes(w, problem=p), 10_000, seed=12)


def test_counts_match_oracle_multiplicative_noise(amy):
    rng = np.random.default_rng(72)
    w = W.random_affine(rng, 2, [31, 27], 3, window=[7, 7], kind=W.REACH_AVOID, horizon=4)
    p = dataclasses.replace(w.problem, noise="mult_gaussian", noise_params=[[0.15] * 2])
    _same_counts(amy, W.with_sizes(w, problem=p), 10_000, seed=13)


def test_gpu_policy_frequencies_match_value(amy):
    """The GPU's own synthesized policy run on the GPU: frequencies within 4
    binomial standard deviations of the oracle's V_0."""
    w = _coarse_robot()
    p, s = w.problem, w.spec
    ref = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    x0 = _starts(ref["V"], mask, 10)
    runs = 200_000
    with amy.amy_build(p, tmode="otf", prec="fp32") as h:
        V, pi = amy.amy_synthesize(h, s, w.horizon, policy_all_steps=True)
        got = amy.amy_simulate(h, s, w.horizon, pi, x0, runs, seed=77)
    Vr = ref["V"][x0]
    z = (got / runs - Vr) / np.sqrt(Vr * (1 - Vr) / runs)
    assert np.all(np.abs(z) < 4.0), z


def test_device_buffers_match_host_buffers(amy):
    import torch
    w = _coarse_robot()
    p, s = w.problem, w.spec
    ref = oracle.synthesize(p, s, w.horizon)
    x0 = _starts(ref["V"], oracle.spec_mask(p, s), 8)
    with amy.amy_build(p, tmode="otf", prec="fp32") as h:
        host = amy.amy_simulate(h, s, w.horizon, ref["pi"], x0, 30_000, seed=1)
        pol = torch.from_numpy(ref["pi"].astype(np.int16)).cuda()
        xd = torch.tensor(x0, dtype=torch.int64, device="cuda")
        out = torch.full((len(x0),), -1, dtype=torch.int64, device="cuda")
        amy.amy_simulate(h, s, w.horizon, pol, xd, 30_000, seed=1, out=out)
        assert np.array_equal(out.cpu().numpy(), host)
        # runs are independent streams: the first runs of a longer batch are those of a shorter one
        again = amy.amy_simulate(h, s, w.horizon, ref["pi"], x0, 30_000, seed=1)
        assert np.array_equal(again, host)
        other = amy.amy_simulate(h, s, w.horizon, ref["pi"], x0, 30_000, seed=2)
        assert not np.array_equal(other, host)


def test_absorbing_states_and_empty_horizon(amy):
    w = _coarse_robot()
    p, s = w.problem, w.spec
    ref = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    tgt, avd = int(np.flatnonzero(mask & 1)[0]), int(np.flatnonzero(mask & 2)[0])
    free = int(np.flatnonzero(mask == 4)[0])
    with amy.amy_build(p, tmode="otf", prec="fp32") as h:
        c = amy.amy_simulate(h, s, w.horizon, ref["pi"], [tgt, avd], 1000, seed=1)
        assert list(c) == [1000, 0]
        c0 = amy.amy_simulate(h, s, 0, None, [tgt, avd, free], 10, seed=1)
        assert list(c0) == [10, 0, 0]
        assert amy.amy_simulate(h, s, w.horizon, ref["pi"], [], 10, seed=1).size == 0
        assert list(amy.amy_simulate(h, s, w.horizon, ref["pi"], [free], 0, seed=1)) == [0]


def test_bad_arguments_rejected(amy):
    import torch
    w = _coarse_robot()
    p, s = w.problem, w.spec
    ref = oracle.synthesize(p, s, w.horizon)
    free = int(np.flatnonzero(oracle.spec_mask(p, s) == 4)[0])
    with amy.amy_build(p, tmode="otf", prec="fp32") as h:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_simulate(h, s, w.horizon, ref["pi"], [p.n_states], 10, seed=1)
        assert "INVALID_ARG" in str(e.value)
        # device initial states out of range: the kernel checks and reports
        pol = torch.from_numpy(ref["pi"].astype(np.int16)).cuda()
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        with pytest.raises(amy.AmyError) as e:
            amy.amy_simulate(h, s, w.horizon, pol, torch.tensor([free, -3], dtype=torch.int64, device="cuda"),
                             10, seed=1, out=out)
        assert "INVALID_ARG" in str(e.value)
        # a policy entry naming no input at a live state
        bad = ref["pi"].copy()
        bad[0, free] = p.n_inputs
        with pytest.raises(amy.AmyError) as e:
            amy.amy_simulate(h, s, w.horizon, bad, [free], 10, seed=1)
        assert "INVALID_ARG" in str(e.value)
        with pytest.raises(amy.AmyError):
            amy.amy_simulate(h, s, w.horizon, ref["pi"], [free], -1, seed=1)
        # the handle is still usable
        assert amy.amy_simulate(h, s, w.horizon, ref["pi"], [free], 10, seed=1).size == 1
