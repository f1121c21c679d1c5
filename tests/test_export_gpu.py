"""GPU checks of the PRISM export of the abstraction (the tool's PRISM export,
Sec. 2) through the C ABI.

The exported files are read back by an independent parser here and checked
against the oracle: every distribution sums to one (the sink takes the cut
mass), the rows equal the oracle's rows, the labels equal the oracle's spec
mask, and a plain bounded value iteration over the exported MDP -- written
here from the property the .props file states, sharing nothing with either
side -- gives the oracle's V_0."""
import dataclasses
import os

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


def _read(prefix):
    with open(prefix + ".tra") as f:
        S, Cn, T = (int(v) for v in f.readline().split())
        body = np.loadtxt(f, ndmin=2)
    assert body.shape == (T, 4)
    lab = {}
    with open(prefix + ".lab") as f:
        names = dict(item.split("=") for item in f.readline().split())
        names = {int(k): v.strip('"') for k, v in names.items()}
        for line in f:
            s, ids = line.split(":")
            lab[int(s)] = {names[int(i)] for i in ids.split()}
    with open(prefix + ".sta") as f:
        head = f.readline().strip()
        sta = [tuple(int(v) for v in line.split(":")[1].strip("()\n").split(",")) for line in f]
    with open(prefix + ".props") as f:
        prop = f.read().strip()
    return S, Cn, body, lab, head, sta, prop


def _bounded_vi(S, body, lab, prop, horizon):
    """Pmax of the bounded property by backward induction over the exported
    MDP, from the .props text and the labels alone."""
    src, ch, dst, pr = body[:, 0].astype(np.int64), body[:, 1].astype(np.int64), body[:, 2].astype(np.int64), body[:, 3]
    has = lambda name: np.array([name in lab.get(s, set()) for s in range(S)])
    if "G<=" in prop:
        good, stop_win, stop_lose = has("safe"), np.zeros(S, bool), ~has("safe")
        V = good.astype(float)
    else:
        tgt = has("target")
        avoid = has("avoid") if '!"avoid"' in prop else np.zeros(S, bool)
        stop_win, stop_lose = tgt, avoid & ~tgt
        V = tgt.astype(float)
    key = src * (int(ch.max()) + 1) + ch
    for _ in range(horizon):
        q = np.zeros(int(key.max()) + 1)
        np.add.at(q, key, pr * V[dst])
        best = np.full(S, -np.inf)
        np.maximum.at(best, src, q[key])
        V = np.where(stop_win, 1.0, np.where(stop_lose, 0.0, best))
    return V


def _cases():
    rng = np.random.default_rng(61)
    robot = W.robot_lin(n_per_dim=17, horizon=5)
    robot.problem.x_eta = [10.0 / 16, 10.0 / 16]
    safety = W.random_affine(rng, 2, [13, 11], 3, gamma=2e-2, kind=W.SAFETY, horizon=4)
    ring = W.random_affine(rng, 3, [6, 5, 7], 2, gamma=1e-2, kind=W.REACH_AVOID, horizon=3, periodic=[0, 1, 0])
    reach = W.random_affine(rng, 2, [12, 12], 3, gamma=1e-2, kind=W.REACH, horizon=4)
    uni = W.random_affine(rng, 2, [15, 13], 3, gamma=2e-2, kind=W.REACH_AVOID, horizon=4)
    uni = W.with_sizes(uni, problem=dataclasses.replace(uni.problem, noise="uniform", noise_params=[[0.4, 0.4]]))
    return [("robot", robot, "otf", "fp64", 1e-12), ("safety", safety, "stored_full", "fp64", 1e-12),
            ("ring", ring, "stored_separable", "fp32", 1e-5), ("reach", reach, "otf", "fp32", 1e-5),
            ("uniform", uni, "stored_factored", "fp64", 1e-12)]


@pytest.mark.parametrize("name,w,tmode,prec,tol", _cases())
def test_export_round_trip(amy, tmp_path, name, w, tmode, prec, tol):
    p, s = w.problem, w.spec
    prefix = str(tmp_path / name)
    with amy.amy_build(p, tmode=tmode, prec=prec) as h:
        T = amy.amy_export_prism(h, s, w.horizon, prefix)
    S, Cn, body, lab, head, sta, prop = _read(prefix)
    nx, nu = p.n_states, p.n_inputs
    assert S == nx + 1 and Cn == nx * nu + 1 and body.shape[0] == T
    assert head == "(" + ",".join(f"x{d}" for d in range(p.n)) + ")"
    # every choice's distribution sums to one
    key = body[:, 0].astype(np.int64) * (nu + 1) + body[:, 1].astype(np.int64)
    sums = np.zeros(int(key.max()) + 1)
    np.add.at(sums, key, body[:, 3])
    sum_tol = 1e-5 if prec == "fp32" else 1e-12
    assert np.all(np.abs(sums[np.unique(key)] - 1.0) < sum_tol)
    # states and labels
    for x in [0, nx // 3, nx - 1]:
        idx = np.unravel_index(x, p.x_count)
        assert sta[x] == tuple(int(v) for v in idx)
    assert sta[nx] == tuple([-1] * p.n)
    mask = oracle.spec_mask(p, s)
    for x in range(nx):
        names = lab[x]
        assert "init" in names
        assert ("target" in names) == bool(mask[x] & 1)
        assert ("avoid" in names) == bool(mask[x] & 2)
        if s.kind == W.SAFETY:
            assert ("safe" in names) == bool(mask[x] & 4)
    assert lab[nx] == {"sink"}
    # rows against the oracle's rows on sampled pairs
    rng = np.random.default_rng(3)
    Wd, _ = oracle.window_shape(p)
    rows = {}
    for a, b, c, v in body:
        if int(a) < nx:
            rows.setdefault((int(a), int(b)), {})[int(c)] = v
    for x, u in zip(rng.integers(0, nx, 40), rng.integers(0, nu, 40)):
        origin, probs = oracle.row(p, int(x), int(u))
        want = {}
        for slot, pr in enumerate(probs):
            if pr <= 0:
                continue
            k = np.unravel_index(slot, Wd)
            cell = []
            on = True
            for d in range(p.n):
                cd = int(origin[d] + k[d])
                if p.x_periodic[d]:
                    cd %= p.x_count[d]
                elif not 0 <= cd < p.x_count[d]:
                    on = False
                cell.append(cd)
            if on:
                t = int(np.ravel_multi_index(cell, p.x_count))
                want[t] = want.get(t, 0.0) + pr
        got = dict(rows[(int(x), int(u))])
        lost = got.pop(nx, 0.0)
        assert set(got) <= set(want), (name, x, u)
        for t, v in want.items():
            assert abs(got.get(t, 0.0) - v) <= (2e-6 if prec == "fp32" else 1e-13), (name, x, u, t)
        assert abs(lost - max(0.0, 1.0 - sum(want.values()))) <= (1e-5 if prec == "fp32" else 1e-12)
    # the property's bounded value iteration over the exported model is V_0
    ref = oracle.synthesize(p, s, w.horizon)
    V = _bounded_vi(S, body, lab, prop, w.horizon)
    assert float(np.max(np.abs(V[:nx] - ref["V"]))) <= tol, name
    assert V[nx] == 0.0


def test_export_property_text(amy, tmp_path):
    w = _cases()[0][1]
    with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
        amy.amy_export_prism(h, w.spec, 7, str(tmp_path / "a"))
        amy.amy_export_prism(h, W.Spec(W.SAFETY, safe=([-4.0, -4.0], [4.0, 4.0])), 3, str(tmp_path / "b"))
        amy.amy_export_prism(h, W.Spec(W.REACH, targets=[([3.0, 3.0], [5.0, 5.0])]), 2, str(tmp_path / "c"))
    assert open(tmp_path / "a.props").read().strip() == 'Pmax=? [ !"avoid" U<=7 "target" ]'
    assert open(tmp_path / "b.props").read().strip() == 'Pmax=? [ G<=3 "safe" ]'
    assert open(tmp_path / "c.props").read().strip() == 'Pmax=? [ F<=2 "target" ]'
    assert not os.path.exists(tmp_path / "a.tra.part")


def test_export_rejects(amy, tmp_path):
    w = W.robot_dist(horizon=2)
    with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_export_prism(h, w.spec, 2, str(tmp_path / "d"))
        assert "UNSUPPORTED" in str(e.value)
    w = _cases()[3][1]
    with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_export_prism(h, w.spec, 2, str(tmp_path / "no_such_dir" / "x"))
        assert "INVALID_ARG" in str(e.value)
        with pytest.raises(amy.AmyError):
            amy.amy_export_prism(h, w.spec, -1, str(tmp_path / "y"))
