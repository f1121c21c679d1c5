"""Pins of the oracle's text systems (Sec. 3: the right-hand side of the
difference equation given as text in a configuration file).

The evaluator is checked against Python's own evaluation of the same
expressions -- Python floats are IEEE doubles and its math module calls the
same C library -- on seeded random expressions, and whole syntheses of text
systems against the oracle's built-in systems that the texts restate in the
same operation order (the affine robot, the unicycle and the paper's
disturbed robot): those must agree bit for bit.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workloads as W

_PY = {name: getattr(math, name) for name in
       ["sin", "cos", "tan", "asin", "acos", "atan", "sinh", "cosh", "tanh", "exp", "log", "log10", "sqrt",
        "fabs", "floor", "ceil", "atan2", "pow"]}
_PY["fmin"] = min
_PY["fmax"] = max


def _rand_expr(rng, depth, names):
    """A random expression whose every call stays inside its domain."""
    if depth == 0 or rng.random() < 0.25:
        r = rng.random()
        if r < 0.5:
            return str(rng.choice(names))
        v = float(rng.uniform(-3, 3))
        return repr(round(v, int(rng.integers(0, 17)))) if rng.random() < 0.5 else f"{abs(v):.6e}"
    a = _rand_expr(rng, depth - 1, names)
    b = _rand_expr(rng, depth - 1, names)
    k = int(rng.integers(0, 12))
    if k == 0:
        return f"({a} + {b})"
    if k == 1:
        return f"({a} - {b})"
    if k == 2:
        return f"{a} * {b}"
    if k == 3:
        return f"{a} / (fabs({b}) + 0.5)"
    if k == 4:
        return f"-{a}"
    if k == 5:
        f = str(rng.choice(["sin", "cos", "atan", "tanh", "fabs", "floor", "ceil"]))
        return f"{f}({a})"
    if k == 6:
        f = str(rng.choice(["exp", "sinh", "cosh"]))
        return f"{f}(tanh({a}))"
    if k == 7:
        f = str(rng.choice(["log", "log10", "sqrt"]))
        return f"{f}(fabs({a}) + 0.25)"
    if k == 8:
        f = str(rng.choice(["asin", "acos"]))
        return f"{f}(tanh({a}))"
    if k == 9:
        return f"pow(fabs({a}) + 0.5, tanh({b}))"
    if k == 10:
        f = str(rng.choice(["atan2", "fmin", "fmax"]))
        return f"{f}({a}, {b})"
    return f"tan(tanh({a}))"


def test_evaluator_matches_python_bitwise():
    rng = np.random.default_rng(W.SEED)
    names = ["x0", "x1", "x2", "u0", "u1", "w0", "p0", "p1"]
    for trial in range(300):
        exprs = [_rand_expr(rng, int(rng.integers(1, 6)), names) for _ in range(3)]
        x, u, w, prm = rng.normal(size=3), rng.normal(size=2), rng.normal(size=1), rng.normal(size=2)
        got = oracle.expr_eval(exprs, 3, 2, 1, prm, x, u, w)
        env = dict(_PY, x0=x[0], x1=x[1], x2=x[2], u0=u[0], u1=u[1], w0=w[0], p0=prm[0], p1=prm[1])
        for d in range(3):
            want = eval(exprs[d], {"__builtins__": {}}, env)
            assert got[d] == want or (math.isnan(got[d]) and math.isnan(want)), (trial, exprs[d], got[d], want)


def test_evaluator_precedence_and_literals():
    cases = [("1/2", 0.5), ("2*-3", -6.0), ("-2*3+4", -2.0), ("8/4/2", 1.0), ("8-4-2", 2.0),
             ("2*(3+4)", 14.0), ("- -x0", 1.5), ("+x0", 1.5), ("1e-3*1E3", 1.0), (".5+5.", 5.5),
             ("pow(2, 10)", 1024.0), ("fmin(x0, -1)", -1.0), ("atan2(1, 1)", math.atan2(1, 1))]
    for text, want in cases:
        assert oracle.expr_eval([text], 1, 0, 0, [], [1.5], [], [])[0] == want, text


@pytest.mark.parametrize("text", ["x0 +", "x1", "u0", "w0", "p0", "sin(x0", "sin x0", "foo(x0)", "x0 x0",
                                  "pow(x0)", "sin(x0, x0)", "x00", "1e", "3x0", "x0; x0", "x-1", "(((x0)"])
def test_evaluator_rejects(text):
    with pytest.raises(ValueError):
        oracle.expr_eval([text], 1, 0, 0, [], [1.0], [], [])


def test_deep_nesting_rejected_not_crashed():
    with pytest.raises(ValueError):
        oracle.expr_eval(["(" * 400 + "x0" + ")" * 400], 1, 0, 0, [], [1.0], [], [])
    assert oracle.expr_eval(["(" * 60 + "x0" + ")" * 60], 1, 0, 0, [], [1.0], [], [])[0] == 1.0
    long_sum = " + ".join(["x0"] * 2000)
    assert oracle.expr_eval([long_sum], 1, 0, 0, [], [0.5], [], [])[0] == 1000.0


def _same(a, b):
    assert float(np.ptp(a["V"])) > 1e-4  # not a constant value function
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["pi"], b["pi"])


def test_text_robot_equals_affine_robot():
    w = W.robot_lin(n_per_dim=17, horizon=5)
    w.problem.x_eta = [10.0 / 16, 10.0 / 16]
    p = w.problem
    q = dataclasses.replace(p, sys_kind=W.EXPR, params=np.zeros(0), exprs=["x0 + u0", "x1 + u1"])
    _same(oracle.synthesize(p, w.spec, w.horizon), oracle.synthesize(q, w.spec, w.horizon))


def test_text_unicycle_equals_builtin_unicycle():
    w = W.unicycle(nxy=15, nth=12, horizon=4, target=(1.0, 2.0))
    p = w.problem
    q = dataclasses.replace(p, sys_kind=W.EXPR, exprs=["x0 + p0*u0*cos(x2)", "x1 + p0*u0*sin(x2)", "x2 + p0*u1"])
    _same(oracle.synthesize(p, w.spec, w.horizon), oracle.synthesize(q, w.spec, w.horizon))
    # a row of the periodic heading dim: origins and masses identical
    for x, u in [(0, 0), (1000, 17), (2699, 44)]:
        a, b = oracle.row(p, x, u), oracle.row(q, x, u)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_text_disturbed_robot_equals_affine_records():
    """The paper's robot with its disturbance: the text system's game value
    and policy equal those of the per-(input, disturbance) affine records."""
    a = W.robot_dist(n_per_dim=21, horizon=4)
    b = W.robot_dist_expr(n_per_dim=21, horizon=4)
    _same(oracle.synthesize(a.problem, a.spec, a.horizon), oracle.synthesize(b.problem, b.spec, b.horizon))


def test_text_parameters_are_bound():
    w = W.robot_lin(n_per_dim=17, horizon=3)
    w.problem.x_eta = [10.0 / 16, 10.0 / 16]
    p = w.problem
    q1 = dataclasses.replace(p, sys_kind=W.EXPR, params=np.array([1.0, 0.0]), exprs=["p0*x0 + u0 + p1", "x1 + u1"])
    q2 = dataclasses.replace(q1, params=np.array([1.0, 0.25]))
    r0 = oracle.synthesize(p, w.spec, w.horizon)
    _same(r0, oracle.synthesize(q1, w.spec, w.horizon))
    assert not np.array_equal(r0["V"], oracle.synthesize(q2, w.spec, w.horizon)["V"])
    mu = oracle.mean(q2, 7, 3)
    uc = W.input_centres(p)[3]
    xc = [p.x_lb[0] + 0 * p.x_eta[0], p.x_lb[1] + 7 * p.x_eta[1]]
    assert mu[0] == 1.0 * xc[0] + uc[0] + 0.25 and mu[1] == xc[1] + uc[1]
