"""GPU parity of systems given as text (Sec. 3: the right-hand side of the
difference equation written in the tool's configuration file), compiled at
build time with NVRTC into mean tables, against the FP64 oracle's own
expression evaluator: the paper's disturbed robot, the unicycle, a nonlinear
traffic ring with a saturating flow (per-dimension tables, the plane kernel)
and seeded random nonlinear systems, in every row mode and precision; window
origins bit-exact; text and built-in systems identical on the GPU; rebuilds
with new parameters; rejection of bad text."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import TOL, compare_rows, compare_synthesis, load_engine

pytestmark = pytest.mark.gpu

MODES = [("otf", "fp32"), ("otf", "fp32_kahan"), ("otf", "fp64"), ("stored_separable", "fp32_kahan"),
         ("stored_factored", "fp32"), ("stored_full", "fp64")]


@pytest.fixture(scope="module")
def amy():
    return load_engine()


def _text_unicycle(**kw):
    w = W.unicycle(**kw)
    p = dataclasses.replace(w.problem, sys_kind=W.EXPR,
                            exprs=["x0 + p0*u0*cos(x2)", "x1 + p0*u0*sin(x2)", "x2 + p0*u1"])
    return W.with_sizes(w, problem=p)


def _random_text(rng, n, per_dim, n_u, horizon=3, disturb=False):
    """A seeded nonlinear system: each component mixes its own coordinate,
    a neighbour through a bounded nonlinearity and the input."""
    base = W.random_affine(rng, n, per_dim, n_u, gamma=1e-2, kind=W.REACH_AVOID, horizon=horizon)
    exprs = []
    for d in range(n):
        a = float(rng.uniform(0.5, 0.9))
        b = float(rng.uniform(-0.6, 0.6))
        c = float(rng.uniform(0.3, 1.0))
        j = (d + 1) % n
        f = ["tanh", "sin", "atan"][d % 3]
        e = f"{a!r}*x{d} + {b!r}*{f}(x{j}) + {c!r}*u0*cos(p0*x{d})"
        if disturb:
            e += " + 0.3*w0"
        exprs.append(e)
    p = dataclasses.replace(base.problem, sys_kind=W.EXPR, params=np.array([0.7]), exprs=exprs,
                            name=f"text_random_{n}")
    if disturb:
        p = dataclasses.replace(p, w_lb=[-1.0], w_eta=[1.0], w_count=[3])
    return W.with_sizes(base, problem=p)


@pytest.mark.parametrize("tmode,prec", MODES)
def test_text_robot_matches_oracle(amy, tmode, prec):
    """The robot of Sec. 7 with its disturbance, given as text."""
    w = W.robot_dist_expr(n_per_dim=21, horizon=5)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    with amy.amy_build(w.problem, tmode=tmode, prec=prec) as h:
        assert amy.amy_info(h)["n_disturbances"] == 11
    compare_synthesis(amy, w, tmode, prec, ref=ref)


def test_text_equals_builtin_on_the_gpu(amy):
    """The text unicycle and the built-in one: identical values and policies
    (same FP64 operations, same CUDA cos and sin); the text robot and its
    affine records: equal to rounding."""
    pairs = [(W.robot_dist(n_per_dim=21, horizon=4), W.robot_dist_expr(n_per_dim=21, horizon=4)),
             (W.unicycle(nxy=15, nth=12, horizon=4, target=(1.0, 2.0)),
              _text_unicycle(nxy=15, nth=12, horizon=4, target=(1.0, 2.0)))]
    for a, b in pairs:
        for tmode, prec in [("otf", "fp64"), ("stored_factored", "fp32"), ("stored_separable", "fp32")]:
            with amy.amy_build(a.problem, tmode=tmode, prec=prec) as h:
                Va, Pa = amy.amy_synthesize(h, a.spec, a.horizon, policy_all_steps=True)
            with amy.amy_build(b.problem, tmode=tmode, prec=prec) as h:
                Vb, Pb = amy.amy_synthesize(h, b.spec, b.horizon, policy_all_steps=True)
            if a.problem.sys_kind == W.UNICYCLE:
                assert np.array_equal(Va, Vb) and np.array_equal(Pa, Pb), (a.problem.name, tmode)
            else:
                # the affine records' constants were computed with the host's
                # cos, the text's with CUDA's: equal to rounding
                assert float(np.max(np.abs(Va - Vb))) <= TOL[prec], (a.problem.name, tmode)


@pytest.mark.parametrize("tmode,prec", MODES)
def test_text_unicycle_matches_oracle(amy, tmode, prec):
    w = _text_unicycle(nxy=15, nth=12, horizon=4, target=(1.0, 2.0))
    compare_synthesis(amy, w, tmode, prec)


@pytest.mark.parametrize("n,per_dim,disturb", [(1, [41], False), (2, [23, 19], True), (3, [9, 8, 10], False),
                                               (4, [6, 5, 6, 5], True)])
def test_random_text_systems(amy, n, per_dim, disturb):
    rng = np.random.default_rng(400 + n)
    w = _random_text(rng, n, per_dim, 3, disturb=disturb)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for tmode, prec in MODES:
        compare_synthesis(amy, w, tmode, prec, ref=ref)


def test_text_rows_origins_exact(amy):
    for w in [W.robot_dist_expr(n_per_dim=21, horizon=2), _random_text(np.random.default_rng(9), 3, [9, 8, 10], 3)]:
        for tmode, prec, tol in [("otf", "fp64", 1e-13), ("stored_separable", "fp32", 2e-6)]:
            mism, worst = compare_rows(amy, w, tmode, prec, n_pairs=200, seed=5)
            assert mism == 0 and worst <= tol, (w.problem.name, tmode, mism, worst)


def test_text_traffic_tables_and_plane_kernel(amy):
    """A saturating traffic ring as text: component i reads three cells, so
    the per-dimension tables are small and the plane kernel (7) runs."""
    w = W.traffic_text(n_per_dim=6, horizon=2, capacity=3.0)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32_kahan") as h:
        assert amy.amy_info(h)["backup_kernel"] == 7
    compare_synthesis(amy, w, "stored_separable", "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32", ref=ref)
    compare_synthesis(amy, w, "stored_factored", "fp32", ref=ref)


def test_text_rebuild_with_new_parameters(amy):
    """amy_rebuild with new params refills the mean tables: the handle then
    gives what a fresh build with those params gives, and the oracle."""
    w = W.traffic_text(n_per_dim=6, horizon=2, capacity=3.0)
    w2 = W.with_sizes(w, problem=dataclasses.replace(w.problem, params=np.array([1.5])))
    ref2 = oracle.synthesize(w2.problem, w2.spec, w2.horizon)
    for tmode in ["stored_separable", "otf", "stored_factored"]:
        with amy.amy_build(w2.problem, tmode=tmode, prec="fp32") as h:
            V_fresh, _ = amy.amy_synthesize(h, w.spec, w.horizon)
        with amy.amy_build(w.problem, tmode=tmode, prec="fp32") as h:
            V1, _ = amy.amy_synthesize(h, w.spec, w.horizon)
            amy.amy_rebuild(h, np.array([1.5]))
            V2, _ = amy.amy_synthesize(h, w.spec, w.horizon)
        assert not np.array_equal(V1, V2)
        assert np.array_equal(V2, V_fresh), tmode
        assert float(np.max(np.abs(V2 - ref2["V"]))) <= TOL["fp32"], tmode


@pytest.mark.parametrize("exprs,err", [(["x0 +", "x1"], "INVALID_ARG"), (["x0", "y1"], "INVALID_ARG"),
                                       (["x0", "x2"], "INVALID_ARG"), (["x0", "p1"], "INVALID_ARG"),
                                       (["x0", "w0"], "INVALID_ARG"), (["x0", "exp(x1, x0)"], "INVALID_ARG"),
                                       (["x0", "x1; x0"], "INVALID_ARG")])
def test_bad_text_rejected(amy, exprs, err):
    w = W.robot_lin(n_per_dim=9, horizon=1)
    p = dataclasses.replace(w.problem, sys_kind=W.EXPR, params=np.array([1.0]), exprs=exprs)
    with pytest.raises(amy.AmyError) as e:
        amy.amy_build(p, tmode="otf", prec="fp32")
    assert err in str(e.value)


def test_text_not_served_or_noalloc(amy):
    import torch
    w = W.robot_dist_expr(n_per_dim=11, horizon=2)
    srv = amy.amy_server_create(batched=True, max_slots=4)
    try:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_submit(srv, w)
        assert "UNSUPPORTED" in str(e.value)
    finally:
        srv.close()
    V = torch.empty(w.problem.n_states, dtype=torch.float32, device="cuda")
    P = torch.empty(w.problem.n_states, dtype=torch.int16, device="cuda")
    with pytest.raises(amy.AmyError) as e:
        amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V, P)
    assert "UNSUPPORTED" in str(e.value)
