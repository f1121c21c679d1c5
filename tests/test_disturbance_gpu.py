"""GPU parity of the disturbance player (the max-min game of the Remark in
Sec. 3; Algorithm 4's min over the disturbance grid before the max over
inputs): the CUDA path through the C ABI against the FP64 oracle, on the
paper's robot of Sec. 7 with its disturbance and on seeded random disturbed
systems, in every row mode and precision; window origins of (input,
disturbance) pairs bit-exact; the served and allocation-free paths."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import GAP, TOL, compare_synthesis, load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


@pytest.fixture(scope="module")
def robot_ref():
    w = W.robot_dist()
    return w, oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)


@pytest.mark.parametrize("tmode,prec", [("otf", "fp32"), ("otf", "fp32_kahan"), ("stored_separable", "fp32"),
                                        ("stored_factored", "fp32"), ("otf", "fp64"), ("stored_full", "fp64")])
def test_robot_dist_matches_oracle(amy, robot_ref, tmode, prec):
    """The paper's robot (41^2 states, 121 inputs, 11 disturbance points,
    13 x 13 windows, safety, horizon 8): V_0 and every pi_k."""
    w, ref = robot_ref
    with amy.amy_build(w.problem, tmode=tmode, prec=prec) as h:
        info = amy.amy_info(h)
        assert info["n_inputs"] == 121 and info["n_disturbances"] == 11
    st = compare_synthesis(amy, w, tmode, prec, ref=ref)
    assert st["policy_checked"] > 0


def test_robot_dist_tables_take_the_wide_2d_kernel(amy, robot_ref):
    """The robot's 13 x 13 windows with per-dimension tables: each input's
    value (min over its disturbance points) by k_sums_sep2 into per-state max
    keys, then k_collect_keys (backup kernel 9, two launches per backup), in
    FP32 and with Kahan over rows, against the oracle; repeated syntheses on
    one handle agree bit for bit (the keys are cleared between backups)."""
    w, ref = robot_ref
    for prec in ("fp32", "fp32_kahan"):
        with amy.amy_build(w.problem, tmode="stored_separable", prec=prec) as h:
            info = amy.amy_info(h)
            assert info["backup_kernel"] == 9 and info["backup_launch_kernels"] == 2
        compare_synthesis(amy, w, "stored_separable", prec, ref=ref)
    compare_synthesis(amy, w, "stored_separable", "fp32", v_store="u16", ref=ref)
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32") as h:
        a = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        b = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_robot_dist_reach_avoid_16bit(amy):
    w = W.robot_dist(kind=W.REACH_AVOID, horizon=6)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    compare_synthesis(amy, w, "otf", "fp32", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32", v_store="u16", ref=ref)
    st = compare_synthesis(amy, w, "otf", "fp32", v_store="bf16", ref=ref, bf16_over_ok=True)
    assert "bf16_over" not in st, st


def _disturbed(rng, n, per_dim, n_u, n_w, gamma=1e-2, window=None, kind=W.REACH_AVOID, horizon=3, periodic=None):
    """A seeded random affine system with an additive disturbance grid on
    [-0.5, 0.5] pushing every state dim by w * b (b random)."""
    base = W.random_affine(rng, n, per_dim, n_u, gamma=gamma, window=window, kind=kind, horizon=horizon,
                           periodic=periodic)
    p = base.problem
    rec = p.params.reshape(n_u, n * n + n)
    b = rng.normal(0.0, 0.4, size=n)
    wc = np.linspace(-0.5, 0.5, n_w) if n_w > 1 else np.zeros(1)
    As, cs = [], []
    for u in range(n_u):
        for wv in wc:
            As.append(rec[u, :n * n].reshape(n, n))
            cs.append(rec[u, n * n:] + wv * b)
    q = dataclasses.replace(p, params=W.affine_params(As, cs), w_lb=[-0.5], w_eta=[1.0 / max(n_w - 1, 1)],
                            w_count=[n_w], name=f"disturbed_{n}")
    return W.with_sizes(base, problem=q)


@pytest.mark.parametrize("n,per_dim,n_u,n_w,window,gamma,periodic", [
    (1, [31], 3, 4, None, 5e-2, None),
    (2, [13, 17], 4, 3, [3, 5], 0.0, None),
    (3, [7, 9, 8], 3, 5, None, 1e-2, [0, 0, 1]),
    (4, [5, 6, 5, 4], 2, 3, [3, 3, 3, 3], 0.0, None),
])
@pytest.mark.parametrize("kind", [W.SAFETY, W.REACH_AVOID])
def test_random_disturbed_every_mode(amy, n, per_dim, n_u, n_w, window, gamma, periodic, kind):
    rng = np.random.default_rng(900 + 10 * n + (kind == W.SAFETY))
    w = _disturbed(rng, n, per_dim, n_u, n_w, gamma=gamma, window=window, kind=kind, periodic=periodic)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for tmode in ["otf", "stored_separable", "stored_factored", "stored_full"]:
        compare_synthesis(amy, w, tmode, "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp64", ref=ref)


def test_disturbance_pair_rows_origins_exact(amy):
    """amy_query_rows takes the (input, disturbance) pair index u * n_w + w:
    window origins bit-exact against the oracle's rows, masses within
    rounding, for the robot in FP64 and FP32 tables."""
    w = W.robot_dist()
    p = w.problem
    rng = np.random.default_rng(17)
    xs = rng.integers(0, p.n_states, size=300)
    us = rng.integers(0, p.n_inputs, size=300)
    ws = rng.integers(0, p.n_disturbances, size=300)
    for tmode, prec, tol in [("otf", "fp64", 1e-13), ("stored_separable", "fp32", 2e-6)]:
        with amy.amy_build(p, tmode=tmode, prec=prec) as h:
            org, probs = amy.amy_query_rows(h, xs, us * p.n_disturbances + ws)
        for i in range(len(xs)):
            o_ref, pr_ref = oracle.row(p, int(xs[i]), int(us[i]), int(ws[i]))
            assert np.array_equal(o_ref, org[i]), (tmode, i)
            assert float(np.max(np.abs(pr_ref - probs[i]))) <= tol, (tmode, i)


def test_one_point_grid_equals_no_disturbance(amy):
    """A one-point disturbance grid gives the disturbance-free results bit for
    bit on the GPU as well (same means, same kernels' arithmetic)."""
    rng = np.random.default_rng(31)
    w = W.random_affine(rng, 2, [15, 12], 4, gamma=1e-2, horizon=4)
    q = dataclasses.replace(w.problem, w_lb=[0.0], w_eta=[1.0], w_count=[1])
    for tmode in ["otf", "stored_separable"]:
        with amy.amy_build(w.problem, tmode=tmode, prec="fp32") as h:
            a = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        with amy.amy_build(q, tmode=tmode, prec="fp32") as h:
            b = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_disturbance_served_and_noalloc(amy):
    """The served path (batched and plain) and the allocation-free entry point
    take disturbed problems too, with the allocating path's results."""
    import torch
    rng = np.random.default_rng(44)
    reqs = [_disturbed(rng, 2, [14, 11], 3, 3, horizon=5), _disturbed(rng, 3, [6, 7, 8], 2, 4, horizon=4)]
    direct = []
    for w in reqs:
        with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
            direct.append(amy.amy_synthesize(h, w.spec, w.horizon))
    for batched in (True, False):
        srv = amy.amy_server_create(batched=batched, max_slots=8)
        try:
            tk = [amy.amy_submit(srv, w) for w in reqs]
            for t, (Vd, pd) in zip(tk, direct):
                r = amy.amy_wait(srv, t)
                assert float(np.max(np.abs(r["V"] - Vd))) <= 2e-6
        finally:
            srv.close()
    for w, (Vd, pd) in zip(reqs, direct):
        n = w.problem.n_states
        V = torch.empty(n, dtype=torch.float32, device="cuda")
        P = torch.empty(n, dtype=torch.int16, device="cuda")
        amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V, P)
        torch.cuda.synchronize()
        assert float(np.max(np.abs(V.cpu().numpy() - Vd))) <= TOL["fp32"]


def test_disturbance_rejected_for_the_unicycle(amy):
    w = W.unicycle(nxy=11, horizon=2, target=(1.0, 2.0))
    q = dataclasses.replace(w.problem, w_lb=[0.0], w_eta=[1.0], w_count=[2])
    with pytest.raises(amy.AmyError) as e:
        amy.amy_build(q, tmode="otf", prec="fp32")
    assert "UNSUPPORTED" in str(e.value)


@pytest.mark.parametrize("periodic,window,n_w", [(None, [11, 9], 1), ([0, 1], [13, 15], 3), ([1, 1], [9, 11], 2),
                                                 (None, [15, 15], 2)])
def test_wide_2d_kernel_shapes(amy, periodic, window, n_w):
    """Kernel 9 on seeded 2-D systems with windows of 9 to 16 slots: the
    shared-memory form (no periodic dim) and the global-memory form (a
    periodic dim), with and without a disturbance grid, against the oracle."""
    rng = np.random.default_rng(700 + sum(window) + n_w)
    w = _disturbed(rng, 2, [23, 19], 3, n_w, gamma=0.0, window=window, kind=W.REACH_AVOID, horizon=4,
                   periodic=periodic)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for prec in ("fp32", "fp32_kahan"):
        with amy.amy_build(w.problem, tmode="stored_separable", prec=prec) as h:
            assert amy.amy_info(h)["backup_kernel"] == 9
        compare_synthesis(amy, w, "stored_separable", prec, ref=ref)


def test_wide_2d_kernel_in_captured_graphs(amy, robot_ref):
    """Device outputs run the horizon as a captured CUDA graph: replays of
    kernel 9 (its keys cleared by the collect kernel) give the host-output
    synthesis bit for bit."""
    import torch
    w, _ = robot_ref
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32") as h:
        Vh, Ph = amy.amy_synthesize(h, w.spec, w.horizon, policy_all_steps=True)
        V = torch.empty(w.problem.n_states, dtype=torch.float32, device="cuda")
        P = torch.empty((w.horizon, w.problem.n_states), dtype=torch.int16, device="cuda")
        for _ in range(3):
            amy.amy_synthesize(h, w.spec, w.horizon, V_out=V, policy_out=P, policy_all_steps=True)
            torch.cuda.synchronize()
            assert np.array_equal(V.cpu().numpy(), Vh)
            assert np.array_equal(P.cpu().numpy().view(np.uint16), Ph)
