"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints, closed forms evaluated independently (mpmath), adaptive
quadrature, brute-force path enumeration over all Markov policies, BFS in the
deterministic limit, Monte-Carlo simulation and exact symmetries.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import AFFINE, UNICYCLE, Problem, Spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _affine_problem(name, x_lb, x_eta, x_count, A_list, c_list, sigma, gamma=0.0, window=None,
                    u_lb=None, u_eta=None, u_count=None, periodic=None):
    n = len(x_count)
    nu = len(A_list)
    return Problem(
        name=name, x_lb=list(x_lb), x_eta=list(x_eta), x_count=list(x_count),
        x_periodic=list(periodic) if periodic else [0] * n,
        u_lb=u_lb or [0.0], u_eta=u_eta or [1.0], u_count=u_count or [nu],
        sys_kind=AFFINE, params=W.affine_params(A_list, c_list), sigma=list(sigma),
        gamma=gamma, window=window)


# --------------------------------------------------------------------------
# P11: the paper's own numbers (grid counts, memory of the stored robot row)
# --------------------------------------------------------------------------
def test_grid_counts_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for case in g["grids"]:
        nx = 1
        for lb, ub, eta in case["x"]:
            nx *= oracle.grid_count(lb, ub, eta)
        nu = 1
        for lb, ub, eta in case["u"]:
            nu *= oracle.grid_count(lb, ub, eta)
        assert nx * nu == case["pairs"], case["case"]


def test_robot_window_memory_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["memory"][0]
    s = math.sqrt(g["variance"])
    p = _affine_problem("robot", [-10, -10], [g["eta"]] * 2, [41, 41],
                        [np.eye(2)], [np.zeros(2)], [s, s], gamma=g["gamma"])
    Wd, xs = oracle.window_shape(p)
    assert list(Wd) == [13, 13]
    mib = g["pairs"] * (int(np.prod(Wd)) + 1) * 4 / 2 ** 20
    assert abs(mib - g["printed_MB"]) / g["printed_MB"] < 0.01


def test_cut_point_solves_density_equation():
    mpmath = pytest.importorskip("mpmath")
    for sigma, gamma in [(0.05, 1e-6), (0.866, 1e-3), (0.3, 0.5), (2.0, 1e-9)]:
        p = _affine_problem("cut", [0.0], [0.1], [11], [np.eye(1)], [np.zeros(1)], [sigma],
                            gamma=gamma)
        _, xs = oracle.window_shape(p)
        dens = mpmath.npdf(mpmath.mpf(xs[0]), 0, sigma)
        assert abs(float(dens) - gamma) <= 1e-12 * gamma


def test_gamma_above_peak_is_rejected():
    p = _affine_problem("cut", [0.0], [0.1], [11], [np.eye(1)], [np.zeros(1)], [0.1],
                        gamma=1.0 / (0.1 * math.sqrt(2 * math.pi)) * 1.0001)
    with pytest.raises(ValueError):
        oracle.window_shape(p)


# --------------------------------------------------------------------------
# P7: cell integrals against adaptive quadrature
# --------------------------------------------------------------------------
@pytest.mark.parametrize("npts", [3, 5])
def test_cell_masses_match_quadrature(npts):
    from scipy import integrate
    rng = np.random.default_rng(7)
    eta = [0.4, 0.7]
    sig = [0.35, 0.5]
    lb = [-0.4 * (npts // 2), -0.7 * (npts // 2)]
    for trial in range(3):
        c = rng.uniform(-0.3, 0.3, size=2)
        p = _affine_problem("quad", lb, eta, [npts, npts], [np.zeros((2, 2))], [c], sig)
        origin, probs = oracle.row(p, 0, 0)
        assert list(origin) == [0, 0]
        probs = probs.reshape(npts, npts)
        for i in range(npts):
            for j in range(npts):
                m = 1.0
                for d, k in ((0, i), (1, j)):
                    cc = lb[d] + k * eta[d]
                    f = lambda t, d=d: math.exp(-0.5 * ((t - c[d]) / sig[d]) ** 2) / (sig[d] * math.sqrt(2 * math.pi))
                    v, _ = integrate.quad(f, cc - eta[d] / 2, cc + eta[d] / 2, epsabs=1e-15, epsrel=1e-14, limit=200)
                    m *= v
                assert abs(probs[i, j] - m) <= 1e-13, (i, j, probs[i, j], m)


# --------------------------------------------------------------------------
# P4: row sums telescope to the Gaussian mass of the kept box
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["gamma", "explicit", "dense"])
def test_row_sums_equal_kept_box_mass(mode):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(11)
    w = W.random_affine(rng, 3, [9, 8, 7], 3, gamma=2e-2,
                        window=[3, 5, 3] if mode == "explicit" else None)
    p = w.problem
    if mode == "dense":
        p.gamma = 0.0
    Wd, xs = oracle.window_shape(p)
    for _ in range(12):
        x = int(rng.integers(p.n_states))
        u = int(rng.integers(p.n_inputs))
        origin, probs = oracle.row(p, x, u)
        mu = oracle.mean(p, x, u)
        total = mpmath.mpf(1)
        for d in range(p.n):
            kept = []
            for k in range(Wd[d]):
                s = origin[d] + k
                c = p.x_lb[d] + s * p.x_eta[d]
                ok = 0 <= s < p.x_count[d]
                if mode == "gamma" and not (c <= mu[d] + xs[d]):
                    ok = False
                if ok:
                    kept.append(s)
            if not kept:
                total = mpmath.mpf(0)
                break
            e_lo = mpmath.mpf(p.x_lb[d]) + kept[0] * mpmath.mpf(p.x_eta[d]) - mpmath.mpf(p.x_eta[d]) / 2
            e_hi = mpmath.mpf(p.x_lb[d]) + kept[-1] * mpmath.mpf(p.x_eta[d]) + mpmath.mpf(p.x_eta[d]) / 2
            sd = mpmath.mpf(p.sigma[d])
            total *= mpmath.ncdf(e_hi, mpmath.mpf(mu[d]), sd) - mpmath.ncdf(e_lo, mpmath.mpf(mu[d]), sd)
        assert abs(float(probs.sum()) - float(total)) <= 1e-14


def test_gamma_window_is_the_cut_region():
    """Kept slots are exactly the grid centres in [mu - xs, mu + xs] (Remark on the
    cutting region); the explicit window is centred on the nearest centre."""
    rng = np.random.default_rng(3)
    w = W.random_affine(rng, 2, [25, 23], 4, gamma=5e-2)
    p = w.problem
    Wd, xs = oracle.window_shape(p)
    for _ in range(40):
        x = int(rng.integers(p.n_states))
        u = int(rng.integers(p.n_inputs))
        origin, probs = oracle.row(p, x, u)
        mu = oracle.mean(p, x, u)
        probs = probs.reshape(Wd)
        for d in range(2):
            cut = [j for j in range(p.x_count[d])
                   if abs(p.x_lb[d] + j * p.x_eta[d] - mu[d]) <= xs[d] - 1e-9]
            slots = set(range(origin[d], origin[d] + Wd[d]))
            assert set(cut) <= slots
            # slots whose centre is clearly outside the cut carry zero mass
            for k in range(Wd[d]):
                c = p.x_lb[d] + (origin[d] + k) * p.x_eta[d]
                if abs(c - mu[d]) > xs[d] + 1e-9:
                    sl = [slice(None)] * 2
                    sl[d] = k
                    assert np.all(probs[tuple(sl)] == 0.0)
    pe = W.random_affine(rng, 2, [25, 23], 4, window=[5, 3]).problem
    for _ in range(40):
        x = int(rng.integers(pe.n_states))
        u = int(rng.integers(pe.n_inputs))
        origin, _ = oracle.row(pe, x, u)
        mu = oracle.mean(pe, x, u)
        for d, Wk in enumerate([5, 3]):
            centre = pe.x_lb[d] + (origin[d] + (Wk - 1) // 2) * pe.x_eta[d]
            assert abs(centre - mu[d]) <= 0.5 * pe.x_eta[d] + 1e-12


# --------------------------------------------------------------------------
# P5: closed form p^N for f == 0
# --------------------------------------------------------------------------
@pytest.mark.parametrize("window", [None, [5, 3]])
def test_zero_dynamics_safety_closed_form(window):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    eta = [0.5, 0.4]
    cnt = [9, 11]
    lb = [-2.0, -2.0]
    sig = [0.6, 0.45]
    p = _affine_problem("zero", lb, eta, cnt, [np.zeros((2, 2))] * 2, [np.zeros(2)] * 2, sig,
                        gamma=0.0, window=window)
    safe = ([-1.0, -1.2], [1.5, 1.0])
    spec = Spec(W.SAFETY, safe=safe)
    N = 5
    r = oracle.synthesize(p, spec, N)
    # mass of N(0, sig^2) over the safe cells inside the row's window, per dim
    pm = mpmath.mpf(1)
    for d in range(2):
        idx = [j for j in range(cnt[d]) if safe[0][d] <= lb[d] + j * eta[d] <= safe[1][d]]
        if window is not None:
            o = int(math.floor((0.0 - lb[d]) / eta[d] + 0.5)) - (window[d] - 1) // 2
            idx = [j for j in idx if o <= j < o + window[d]]
        lo = mpmath.mpf(lb[d]) + idx[0] * mpmath.mpf(eta[d]) - mpmath.mpf(eta[d]) / 2
        hi = mpmath.mpf(lb[d]) + idx[-1] * mpmath.mpf(eta[d]) + mpmath.mpf(eta[d]) / 2
        pm *= mpmath.ncdf(hi, 0, sig[d]) - mpmath.ncdf(lo, 0, sig[d])
    expect = float(pm ** N)
    V = r["V"].reshape(cnt)
    for i in range(cnt[0]):
        for j in range(cnt[1]):
            inside = all(safe[0][d] <= lb[d] + k * eta[d] <= safe[1][d] for d, k in ((0, i), (1, j)))
            assert abs(V[i, j] - (expect if inside else 0.0)) <= 1e-14


# --------------------------------------------------------------------------
# P6: brute force over all deterministic Markov policies and all paths
# --------------------------------------------------------------------------
def _chain_T(sig, eta, drifts):
    """Dense 5-cell chain T[x, u, x'] by mpmath cell integrals (mass off grid lost)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    T = np.zeros((5, len(drifts), 5))
    for x in range(5):
        for u, dr in enumerate(drifts):
            mu = mpmath.mpf(x * eta) + mpmath.mpf(dr)
            for y in range(5):
                lo = mpmath.mpf(y * eta) - mpmath.mpf(eta) / 2
                T[x, u, y] = float(mpmath.ncdf(lo + eta, mu, sig) - mpmath.ncdf(lo, mu, sig))
    return T


def _brute_force(T, kind, N, target, avoid, safe):
    nU = T.shape[1]
    free = [x for x in range(5) if (x in safe if kind == "safety" else (x not in target and x not in avoid))]
    # absorbing targets/avoids; safety: leaving S ends the run
    paths = np.array(list(itertools.product(range(5), repeat=N)), dtype=np.int64)  # x_1..x_N
    best = np.full(5, -1.0)
    n_dec = len(free) * N
    for pol_flat in itertools.product(range(nU), repeat=n_dec):
        pol = {}
        it = iter(pol_flat)
        for k in range(N):
            for x in free:
                pol[(k, x)] = next(it)
        for x0 in range(5):
            total = 0.0
            for path in paths:
                prob = 1.0
                cur = x0
                ok = None
                if kind == "safety" and cur not in safe:
                    ok = False
                if kind != "safety":
                    if cur in target:
                        ok = True
                    elif cur in avoid:
                        ok = False
                absorbed_at = 0 if ok is not None else None
                for k in range(N):
                    if ok is not None:
                        break
                    nxt = int(path[k])
                    prob *= T[cur, pol[(k, cur)], nxt]
                    cur = nxt
                    if kind == "safety":
                        if cur not in safe:
                            ok = False
                    else:
                        if cur in target:
                            ok = True
                        elif cur in avoid:
                            ok = False
                    if ok is not None:
                        absorbed_at = k + 1
                if ok is None:
                    ok = kind == "safety"
                    absorbed_at = N
                if ok:
                    # count each distinct absorbed prefix once: only the path whose
                    # remaining entries are all 0 represents the prefix
                    if absorbed_at < N and np.any(path[absorbed_at:] != 0):
                        continue
                    total += prob
            best[x0] = max(best[x0], total)
    return best


@pytest.mark.parametrize("sigfrac", [0.3, 1.0])
@pytest.mark.parametrize("kind,N,drifts", [("reach_avoid", 2, (-1, 0, 1)),
                                           ("reach_avoid", 3, (-1, 1)),
                                           ("safety", 2, (-1, 0, 1)),
                                           ("reach", 3, (0, 1))])
def test_brute_force_chain(sigfrac, kind, N, drifts):
    eta = 1.0
    sig = sigfrac * eta
    T = _chain_T(sig, eta, [d * eta for d in drifts])
    target, avoid, safe = {4}, ({0} if kind == "reach_avoid" else set()), {1, 2, 3}
    bf = _brute_force(T, kind, N, target, avoid, safe)
    p = _affine_problem("chain", [0.0], [eta], [5], [np.eye(1)] * len(drifts),
                        [np.array([d * eta]) for d in drifts], [sig], gamma=0.0,
                        u_lb=[0.0], u_eta=[1.0], u_count=[len(drifts)])
    if kind == "safety":
        spec = Spec(W.SAFETY, safe=([1.0], [3.0]))
    elif kind == "reach":
        spec = Spec(W.REACH, targets=[([4.0], [4.0])])
    else:
        spec = Spec(W.REACH_AVOID, targets=[([4.0], [4.0])], avoids=[([0.0], [0.0])])
    r = oracle.synthesize(p, spec, N)
    np.testing.assert_allclose(r["V"], bf, atol=1e-12, rtol=0)


def test_brute_force_policy_attains_max():
    """The oracle's policy evaluated by path enumeration reaches V_0."""
    eta, sig, N = 1.0, 0.6, 3
    drifts = (-1, 0, 1)
    T = _chain_T(sig, eta, drifts)
    p = _affine_problem("chain", [0.0], [eta], [5], [np.eye(1)] * 3,
                        [np.array([float(d)]) for d in drifts], [sig], gamma=0.0,
                        u_lb=[0.0], u_eta=[1.0], u_count=[3])
    spec = Spec(W.REACH_AVOID, targets=[([4.0], [4.0])], avoids=[([0.0], [0.0])])
    r = oracle.synthesize(p, spec, N)
    pi = r["pi"]
    # exact evaluation of the fixed policy by enumerating paths
    for x0 in range(5):
        total = 0.0
        for path in itertools.product(range(5), repeat=N):
            cur, prob, done = x0, 1.0, None
            if cur == 4:
                done = True
            elif cur == 0:
                done = False
            k_abs = 0
            for k in range(N):
                if done is not None:
                    break
                prob *= T[cur, pi[k, cur], path[k]]
                cur = path[k]
                if cur == 4:
                    done = True
                elif cur == 0:
                    done = False
                k_abs = k + 1
            if done and all(v == 0 for v in path[k_abs:]):
                total += prob
        assert abs(total - r["V"][x0]) <= 1e-12


# --------------------------------------------------------------------------
# The action values (the window sum of Algorithm 4 for every input at one
# state, the quantity the GPU tie check compares policies by): pinned to an
# independent transition matrix, to the pinned synthesis and to pinned rows.
# --------------------------------------------------------------------------
def test_action_values_match_independent_chain_matrix():
    """On the 5-cell chain, s_u(x) equals sum_x' T[x, u, x'] V(x') with T from
    mpmath cell integrals (P6's matrix), for arbitrary V_next."""
    eta, sig = 1.0, 0.7
    drifts = (-1, 0, 1)
    T = _chain_T(sig, eta, drifts)
    p = _affine_problem("chain", [0.0], [eta], [5], [np.eye(1)] * 3,
                        [np.array([float(d)]) for d in drifts], [sig], gamma=0.0,
                        u_lb=[0.0], u_eta=[1.0], u_count=[3])
    rng = np.random.default_rng(17)
    for _ in range(4):
        Vn = rng.uniform(0.0, 1.0, size=5)
        for x in range(5):
            av = oracle.action_values(p, Vn, x)
            np.testing.assert_allclose(av, T[x] @ Vn, atol=1e-13, rtol=0)


def _check_action_values_against_synthesis(p, s, N):
    """max_u s_u(V_{k+1}, x) is V_k(x) bit for bit and its lowest maximiser is
    pi_k(x), at every free state and step of the pinned synthesis."""
    r = oracle.synthesize(p, s, N, want_all=True)
    mask = oracle.spec_mask(p, s)
    free = (mask & 4) != 0 if s.kind == W.SAFETY else (mask & 3) == 0
    checked = 0
    for k in range(N):
        for x in np.flatnonzero(free):
            av = oracle.action_values(p, r["V_all"][k + 1], int(x))
            assert av.max() == r["V_all"][k][x], (k, x)
            assert int(np.flatnonzero(av == av.max())[0]) == int(r["pi"][k, x]), (k, x)
            checked += 1
    assert checked > 0


def test_action_values_agree_with_synthesis_chain():
    eta, sig = 1.0, 0.6
    p = _affine_problem("chain", [0.0], [eta], [5], [np.eye(1)] * 3,
                        [np.array([float(d)]) for d in (-1, 0, 1)], [sig], gamma=0.0,
                        u_lb=[0.0], u_eta=[1.0], u_count=[3])
    spec = Spec(W.REACH_AVOID, targets=[([4.0], [4.0])], avoids=[([0.0], [0.0])])
    _check_action_values_against_synthesis(p, spec, 3)


def test_action_values_agree_with_synthesis_and_rows_3d():
    """A random 3-D gamma-cut problem with a periodic dim: the same bit-exact
    agreement with the synthesis, and each s_u equals the sum over the pinned
    row (origin, probabilities) of probability x V at the wrapped / dropped
    cells, formed here in numpy."""
    rng = np.random.default_rng(33)
    w = W.random_affine(rng, 3, [7, 6, 8], 4, gamma=2e-2, periodic=[0, 0, 1], kind=W.REACH, horizon=3)
    p, s = w.problem, w.spec
    _check_action_values_against_synthesis(p, s, w.horizon)
    Wd, _ = oracle.window_shape(p)
    Vn = rng.uniform(0.0, 1.0, size=p.n_states)
    for x in rng.choice(p.n_states, size=40, replace=False):
        av = oracle.action_values(p, Vn, int(x))
        for u in range(p.n_inputs):
            origin, probs = oracle.row(p, int(x), u)
            acc = 0.0
            for t, (a, b, c) in enumerate(itertools.product(range(Wd[0]), range(Wd[1]), range(Wd[2]))):
                i, j, k = origin[0] + a, origin[1] + b, (origin[2] + c) % p.x_count[2]
                if not (0 <= i < p.x_count[0] and 0 <= j < p.x_count[1]):
                    assert probs[t] == 0.0
                    continue
                acc += probs[t] * Vn[(i * p.x_count[1] + j) * p.x_count[2] + k]
            assert abs(av[u] - acc) <= 1e-13, (x, u)


# --------------------------------------------------------------------------
# The disturbance player (the max-min game of the Remark in Sec. 3; Algorithm
# 3's "minimize with respect to W", Algorithm 4's inner min): pinned by brute
# force over controller and adversary strategies, and by exact reductions.
# --------------------------------------------------------------------------
def _chain_Tw(sig, drifts, pushes):
    """T[x, u, w, x'] of the 5-cell chain with mean x + drift_u + push_w (mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    T = np.zeros((5, len(drifts), len(pushes), 5))
    for x in range(5):
        for u, dr in enumerate(drifts):
            for w, pw in enumerate(pushes):
                mu = mpmath.mpf(x) + mpmath.mpf(dr) + mpmath.mpf(pw)
                for y in range(5):
                    T[x, u, w, y] = float(mpmath.ncdf(y + 0.5, mu, sig) - mpmath.ncdf(y - 0.5, mu, sig))
    return T


def _game_brute_force(T, kind, N, target, avoid, safe):
    """max over controller Markov policies of min over adversary Markov
    strategies (the adversary sees the state and step, hence the input) of
    the probability of the spec, by enumerating every path."""
    nU, nW = T.shape[1], T.shape[2]
    free = [x for x in range(5) if (x in safe if kind == "safety" else (x not in target and x not in avoid))]
    slots = [(k, x) for k in range(N) for x in free]

    def value(pol, adv, x0):
        # probability by forward propagation over the distribution of the state
        dist = np.zeros(5)
        dist[x0] = 1.0
        won = 0.0
        for k in range(N + 1):
            nxt = np.zeros(5)
            for x in range(5):
                pr = dist[x]
                if pr == 0.0:
                    continue
                if kind == "safety":
                    if x not in safe:
                        continue          # left S: lost
                    if k == N:
                        won += pr
                        continue
                else:
                    if x in target:
                        won += pr
                        continue
                    if x in avoid or k == N:
                        continue
                nxt += pr * T[x, pol[(k, x)], adv[(k, x)]]
            dist = nxt
        return won

    best = np.full(5, -1.0)
    for pf in itertools.product(range(nU), repeat=len(slots)):
        pol = dict(zip(slots, pf))
        worst = np.full(5, np.inf)
        for af in itertools.product(range(nW), repeat=len(slots)):
            adv = dict(zip(slots, af))
            for x0 in range(5):
                worst[x0] = min(worst[x0], value(pol, adv, x0))
        best = np.maximum(best, worst)
    return best


def _disturbed_chain(drifts, pushes, sig, gamma=0.0):
    As = [np.eye(1)] * (len(drifts) * len(pushes))
    cs = [np.array([float(d + pw)]) for d in drifts for pw in pushes]
    p = _affine_problem("dchain", [0.0], [1.0], [5], As, cs, [sig], gamma=gamma,
                        u_lb=[0.0], u_eta=[1.0], u_count=[len(drifts)])
    p.w_lb, p.w_eta, p.w_count = [0.0], [1.0], [len(pushes)]
    return p


@pytest.mark.parametrize("kind,N,safe", [("reach_avoid", 2, {1, 2, 3}), ("safety", 2, {1, 2, 3}),
                                         ("safety", 3, {1, 2})])
def test_disturbance_game_brute_force(kind, N, safe):
    drifts, pushes, sig = (0, 1), (0, -1), 0.7
    T = _chain_Tw(sig, drifts, pushes)
    target, avoid = {4}, ({0} if kind == "reach_avoid" else set())
    bf = _game_brute_force(T, kind, N, target, avoid, safe)
    p = _disturbed_chain(drifts, pushes, sig)
    if kind == "safety":
        lo, hi = min(safe), max(safe)
        spec = Spec(W.SAFETY, safe=([float(lo)], [float(hi)]))
    else:
        spec = Spec(W.REACH_AVOID, targets=[([4.0], [4.0])], avoids=[([0.0], [0.0])])
    r = oracle.synthesize(p, spec, N)
    np.testing.assert_allclose(r["V"], bf, atol=1e-12, rtol=0)


def test_disturbance_reductions():
    """A one-point disturbance grid, or disturbances that do not move the
    mean, give the disturbance-free values bit for bit; a larger disturbance
    grid can only lower the values (the min runs over a superset)."""
    rng = np.random.default_rng(71)
    w = W.random_affine(rng, 2, [11, 9], 3, gamma=5e-3, kind=W.REACH_AVOID, horizon=4)
    p, s, N = w.problem, w.spec, w.horizon
    ref = oracle.synthesize(p, s, N)
    import dataclasses
    p1 = dataclasses.replace(p, w_lb=[0.0], w_eta=[1.0], w_count=[1])
    r1 = oracle.synthesize(p1, s, N)
    assert np.array_equal(r1["V"], ref["V"]) and np.array_equal(r1["pi"], ref["pi"])
    rec = p.params.reshape(p.n_inputs, -1)
    p3 = dataclasses.replace(p, w_lb=[-1.0], w_eta=[1.0], w_count=[3], params=np.repeat(rec, 3, axis=0).reshape(-1))
    r3 = oracle.synthesize(p3, s, N)
    assert np.array_equal(r3["V"], ref["V"]) and np.array_equal(r3["pi"], ref["pi"])
    # genuine pushes of the mean: a superset of pushes can only lower V
    A = rec[:, :4].reshape(-1, 2, 2)
    c = rec[:, 4:]
    pushes_small, pushes_big = [0.0, 0.3], [0.0, 0.3, -0.4]
    vals = []
    for pushes in (pushes_small, pushes_big):
        As, cs = [], []
        for u in range(p.n_inputs):
            for pw in pushes:
                As.append(A[u])
                cs.append(c[u] + pw)
        q = dataclasses.replace(p, w_lb=[0.0], w_eta=[1.0], w_count=[len(pushes)], params=W.affine_params(As, cs))
        vals.append(oracle.synthesize(q, s, N)["V"])
    assert np.all(vals[1] <= vals[0] + 1e-15) and np.all(vals[0] <= ref["V"] + 1e-15)
    assert np.any(vals[1] < vals[0] - 1e-6)


def test_disturbance_action_values_are_min_over_w():
    """Each input's value is the min over the disturbance points of its window
    sums, formed here from the pinned rows (row(p, x, u, w))."""
    p = _disturbed_chain((0, 1, -1), (0, -1, 1), 0.6)
    rng = np.random.default_rng(5)
    Vn = rng.uniform(0.0, 1.0, size=5)
    for x in range(5):
        av = oracle.action_values(p, Vn, x)
        for u in range(3):
            sums = []
            for wv in range(3):
                o, pr = oracle.row(p, x, u, wv)
                sums.append(float(pr @ Vn))      # dense chain: window = the whole grid, origin 0
                assert o[0] == 0
            assert abs(av[u] - min(sums)) <= 1e-15


# --------------------------------------------------------------------------
# Other noise distributions (Sec. 6.2): uniform, exponential, beta (integer
# shapes) and multiplicative Gaussian, pinned to scipy's densities and CDFs.
# --------------------------------------------------------------------------
def _noise_dist(kind, prm, d, xd=0.0):
    """scipy.stats distribution of the noise of dim d (independent of the oracle)."""
    from scipy import stats
    if kind == "uniform":
        a = prm[0][d]
        return stats.uniform(loc=-a, scale=2 * a)
    if kind == "exponential":
        return stats.expon(scale=1.0 / prm[0][d])
    if kind == "beta":
        return stats.beta(prm[0][d], prm[1][d], loc=prm[2][d], scale=prm[3][d] - prm[2][d])
    if kind == "mult_gaussian":
        return stats.norm(scale=prm[0][d] * abs(xd))
    raise ValueError(kind)


NOISES = [("uniform", [[0.37, 0.61]]), ("exponential", [[2.5, 1.3]]),
          ("beta", [[2.0, 3.0], [3.0, 1.0], [-0.6, -0.2], [0.9, 1.1]]),
          ("beta", [[1.0, 4.0], [1.0, 2.0], [-0.5, -1.0], [0.5, 0.3]]),
          ("mult_gaussian", [[0.3, 0.45]])]


def _noise_problem(kind, prm, gamma=0.0, window=None, n=2, npts=9):
    lb, eta = -1.2, 0.3
    rng = np.random.default_rng(3)
    A = np.eye(n) * 0.8
    cs = [rng.uniform(-0.3, 0.3, size=n) for _ in range(2)]
    p = _affine_problem("noise", [lb] * n, [eta] * n, [npts] * n, [A, A], cs, [0.3] * n, gamma=gamma,
                        window=window, u_lb=[0.0], u_eta=[1.0], u_count=[2])
    p.noise, p.noise_params = kind, prm
    return p


@pytest.mark.parametrize("kind,prm", NOISES)
def test_noise_cell_masses_match_quadrature(kind, prm):
    """Dense rows: every cell mass equals the quadrature of scipy's density
    over the cell (a product over the two dims)."""
    from scipy import integrate
    p = _noise_problem(kind, prm)
    rng = np.random.default_rng(9)
    for _ in range(4):
        x, u = int(rng.integers(p.n_states)), int(rng.integers(2))
        origin, probs = oracle.row(p, x, u)
        mu = oracle.mean(p, x, u)
        xi = np.unravel_index(x, p.x_count)
        probs = probs.reshape(p.x_count)
        m = []
        for d in range(2):
            xd = p.x_lb[d] + xi[d] * p.x_eta[d]
            dist = _noise_dist(kind, prm, d, xd)
            row = []
            for j in range(p.x_count[d]):
                c = p.x_lb[d] + j * p.x_eta[d]
                lo, hi = c - p.x_eta[d] / 2 - mu[d], c + p.x_eta[d] / 2 - mu[d]
                if kind == "mult_gaussian" and xd == 0.0:
                    row.append(1.0 if lo <= 0.0 < hi else 0.0)
                    continue
                pts = [t for t in dist.support() if lo < t < hi]
                v, _ = integrate.quad(dist.pdf, lo, hi, points=pts or None, epsabs=1e-14, epsrel=1e-12, limit=200)
                row.append(v)
            m.append(np.array(row))
        np.testing.assert_allclose(probs, np.outer(m[0], m[1]), atol=2e-12, rtol=0)


@pytest.mark.parametrize("kind,prm", [nz for nz in NOISES if nz[0] != "mult_gaussian"])
def test_noise_cut_region_and_row_sums(kind, prm):
    """Gamma mode: the kept slots are exactly the grid centres inside the
    region where the density reaches gamma (the support for bounded
    supports; for the exponential the density level set, found by root
    finding), and each row sums to the distribution's mass over the kept
    cells (scipy's CDF)."""
    from scipy import optimize
    gamma = 0.05
    p = _noise_problem(kind, prm, gamma=gamma, n=2, npts=15)
    Wd, _ = oracle.window_shape(p)
    rng = np.random.default_rng(13)
    for _ in range(10):
        x, u = int(rng.integers(p.n_states)), int(rng.integers(2))
        origin, probs = oracle.row(p, x, u)
        mu = oracle.mean(p, x, u)
        probs = probs.reshape(Wd)
        total = 1.0
        for d in range(2):
            dist = _noise_dist(kind, prm, d)
            lo_s, hi_s = dist.support()
            if kind == "exponential":
                hi_s = optimize.brentq(lambda t: dist.pdf(t) - gamma, 1e-12, 100.0, xtol=1e-14)
            kept = [s for s in range(origin[d], origin[d] + Wd[d])
                    if 0 <= s < p.x_count[d] and mu[d] + lo_s - 1e-9 <= p.x_lb[d] + s * p.x_eta[d] <= mu[d] + hi_s + 1e-9]
            want = [s for s in range(p.x_count[d])
                    if mu[d] + lo_s + 1e-9 < p.x_lb[d] + s * p.x_eta[d] < mu[d] + hi_s - 1e-9]
            assert set(want) <= set(kept)
            if kept:
                e_lo = p.x_lb[d] + kept[0] * p.x_eta[d] - p.x_eta[d] / 2 - mu[d]
                e_hi = p.x_lb[d] + kept[-1] * p.x_eta[d] + p.x_eta[d] / 2 - mu[d]
                total *= dist.cdf(e_hi) - dist.cdf(e_lo)
            else:
                total = 0.0
        assert abs(float(probs.sum()) - total) <= 1e-12


def test_noise_uniform_chain_brute_force():
    """5-cell chain with uniform noise (half-width 0.8): the oracle's V_0
    equals brute force over all Markov policies and paths with T from
    scipy's uniform CDF."""
    from scipy import stats
    a, drifts, N = 0.8, (-1, 0, 1), 2
    T = np.zeros((5, 3, 5))
    dist = stats.uniform(loc=-a, scale=2 * a)
    for x in range(5):
        for u, dr in enumerate(drifts):
            for y in range(5):
                T[x, u, y] = dist.cdf(y + 0.5 - x - dr) - dist.cdf(y - 0.5 - x - dr)
    bf = _brute_force(T, "reach_avoid", N, {4}, {0}, set())
    p = _affine_problem("uchain", [0.0], [1.0], [5], [np.eye(1)] * 3, [np.array([float(d)]) for d in drifts],
                        [1.0], gamma=0.0, u_lb=[0.0], u_eta=[1.0], u_count=[3])
    p.noise, p.noise_params = "uniform", [[a]]
    spec = Spec(W.REACH_AVOID, targets=[([4.0], [4.0])], avoids=[([0.0], [0.0])])
    np.testing.assert_allclose(oracle.synthesize(p, spec, N)["V"], bf, atol=1e-14, rtol=0)


def test_noise_invalid_rejected():
    for kind, prm, gamma in [("beta", [[2.5], [2.0], [-1.0], [1.0]], 0.0),   # non-integer shape
                             ("uniform", [[0.2]], 10.0),                     # gamma above the flat density
                             ("exponential", [[1.0]], 2.0),                  # gamma above the peak
                             ("mult_gaussian", [[0.3]], 1e-3)]:              # multiplicative noise is uncut
        p = _affine_problem("bad", [0.0], [0.3], [9], [np.eye(1)], [np.zeros(1)], [0.3], gamma=gamma)
        p.noise, p.noise_params = kind, prm
        with pytest.raises(ValueError):
            oracle.window_shape(p) if kind != "mult_gaussian" else oracle.synthesize(p, Spec(W.SAFETY), 1)


# --------------------------------------------------------------------------
# P8: deterministic limit equals graph reachability (BFS)
# --------------------------------------------------------------------------
def _bfs_reach(n_states, succ, target, avoid, N):
    """States that reach `target` within N moves avoiding `avoid` (some input each step)."""
    good = set(target)
    for _ in range(N):
        new = set(good)
        for x in range(n_states):
            if x in good or x in avoid:
                continue
            if any(s in good for s in succ(x) if s is not None):
                new.add(x)
        good = new
    return good


def test_deterministic_limit_linear_shear():
    # x+ = A x + c_u on an integer lattice (eta = 1): A = [[1,1],[0,1]] shear, drifts
    n0, n1 = 9, 5
    drifts = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)]
    A = np.array([[1.0, 1.0], [0.0, 1.0]])
    p = _affine_problem("shear", [0.0, -2.0], [1.0, 1.0], [n0, n1], [A] * 5,
                        [np.array(d, float) for d in drifts], [1e-3, 1e-3], window=[3, 3],
                        u_count=[5])
    spec = Spec(W.REACH_AVOID, targets=[([7.0, 1.0], [8.0, 2.0])], avoids=[([3.0, -2.0], [4.0, -1.0])])
    N = 4
    r = oracle.synthesize(p, spec, N)

    def lin(i, j):
        return i * n1 + j

    def succ(x):
        i, j = divmod(x, n1)
        jc = j - 2  # centre value of dim 1
        out = []
        for di, dj in drifts:
            ni, njc = i + jc + di, jc + dj   # shear: x0 + x1, x1
            nj = njc + 2
            out.append(lin(ni, nj) if 0 <= ni < n0 and 0 <= nj < n1 else None)
        return out

    target = {lin(i, j) for i in range(n0) for j in range(n1) if 7 <= i <= 8 and 1 <= j - 2 <= 2}
    avoid = {lin(i, j) for i in range(n0) for j in range(n1) if 3 <= i <= 4 and -2 <= j - 2 <= -1}
    good = _bfs_reach(n0 * n1, succ, target, avoid, N)
    for x in range(n0 * n1):
        assert abs(r["V"][x] - (1.0 if x in good else 0.0)) <= 1e-12, x


def test_deterministic_limit_unicycle():
    # theta on 4 headings, tau*v in {0, 1} cells, tau*omega in {-pi/2, 0, pi/2}
    nxy, nth = 7, 4
    p = Problem(
        name="uni_det", x_lb=[0.0, 0.0, -math.pi], x_eta=[1.0, 1.0, math.pi / 2],
        x_count=[nxy, nxy, nth], x_periodic=[0, 0, 1],
        u_lb=[0.0, -5.0 * math.pi], u_eta=[10.0, 5.0 * math.pi], u_count=[2, 3],
        sys_kind=UNICYCLE, params=np.array([0.1]), sigma=[1e-3, 1e-3, 1e-3],
        gamma=0.0, window=[3, 3, 3])
    spec = Spec(W.REACH, targets=[([5.0, 5.0, -10.0], [6.0, 6.0, 10.0])])
    N = 6
    r = oracle.synthesize(p, spec, N)
    dirs = {0: (-1, 0), 1: (0, -1), 2: (1, 0), 3: (0, 1)}  # heading -pi, -pi/2, 0, pi/2

    def lin(i, j, k):
        return (i * nxy + j) * nth + k

    def succ(x):
        i, rem = divmod(x, nxy * nth)
        j, k = divmod(rem, nth)
        out = []
        for v in (0, 1):
            for dk in (-1, 0, 1):
                ni, nj = i + v * dirs[k][0], j + v * dirs[k][1]
                nk = (k + dk) % nth
                out.append(lin(ni, nj, nk) if 0 <= ni < nxy and 0 <= nj < nxy else None)
        return out

    target = {lin(i, j, k) for i in range(nxy) for j in range(nxy) for k in range(nth)
              if 5 <= i <= 6 and 5 <= j <= 6}
    good = _bfs_reach(nxy * nxy * nth, succ, target, set(), N)
    for x in range(nxy * nxy * nth):
        assert abs(r["V"][x] - (1.0 if x in good else 0.0)) <= 1e-12, x


# --------------------------------------------------------------------------
# P1-P3: range, masks, monotonicity in the horizon
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [W.SAFETY, W.REACH, W.REACH_AVOID])
def test_range_masks_monotone(kind):
    rng = np.random.default_rng(5)
    w = W.random_affine(rng, 2, [15, 13], 4, gamma=1e-3, kind=kind)
    p, s = w.problem, w.spec
    mask = oracle.spec_mask(p, s)
    prev = None
    for N in range(0, 6):
        V = oracle.synthesize(p, s, N)["V"]
        assert np.all(V >= 0.0) and np.all(V <= 1.0 + 1e-14)
        if kind == W.SAFETY:
            assert np.all(V[(mask & 4) == 0] == 0.0)
        else:
            assert np.all(V[(mask & 1) != 0] == 1.0)
            assert np.all(V[(mask & 2) != 0] == 0.0)
        if prev is not None:
            if kind == W.SAFETY:
                assert np.all(V <= prev + 1e-14)
            else:
                assert np.all(V >= prev - 1e-14)
        prev = V


def test_overlapping_target_and_avoid_rejected():
    rng = np.random.default_rng(1)
    w = W.random_affine(rng, 2, [9, 9], 2)
    s = Spec(W.REACH_AVOID, targets=[([0.0, 0.0], [1.0, 1.0])], avoids=[([0.5, 0.5], [2.0, 2.0])])
    with pytest.raises(ValueError):
        oracle.spec_mask(w.problem, s)


# --------------------------------------------------------------------------
# P10: symmetry of the 2-D robot under x1 <-> x2
# --------------------------------------------------------------------------
def test_robot_symmetry():
    w = W.robot_lin(n_per_dim=21, horizon=5)
    r = oracle.synthesize(w.problem, w.spec, w.horizon)
    V = r["V"].reshape(21, 21)
    assert np.max(np.abs(V - V.T)) <= 1e-14


# --------------------------------------------------------------------------
# P9: Monte-Carlo closed loop under the synthesized policy
# --------------------------------------------------------------------------
def test_monte_carlo_closed_loop():
    w = W.robot_lin(n_per_dim=17, horizon=6)
    p, s = w.problem, w.spec
    # coarser grid over the same box: step 10/16
    p.x_eta = [10.0 / 16, 10.0 / 16]
    r = oracle.synthesize(p, s, w.horizon)
    mask = oracle.spec_mask(p, s)
    rng = np.random.default_rng(W.SEED)
    Wd, _ = oracle.window_shape(p)
    rows = {}

    def row(x, u):
        key = (x, u)
        if key not in rows:
            origin, probs = oracle.row(p, x, u)
            idx = np.array([(origin[0] + a) * 17 + (origin[1] + b)
                            for a in range(Wd[0]) for b in range(Wd[1])], dtype=np.int64)
            keep = probs > 0
            pr = np.append(probs[keep], max(0.0, 1.0 - probs[keep].sum()))
            rows[key] = (np.append(idx[keep], -1), pr / pr.sum())
        return rows[key]

    cand = [x for x in range(p.n_states) if mask[x] == 4 and 0.05 < r["V"][x] < 0.95]
    starts = [cand[i] for i in rng.choice(len(cand), size=min(10, len(cand)), replace=False)]
    runs = 100000
    for x0 in starts:
        state = np.full(runs, x0, dtype=np.int64)
        alive = np.ones(runs, dtype=bool)
        success = np.zeros(runs, dtype=bool)
        for k in range(w.horizon):
            cur = state.copy()
            live = alive.copy()
            for x in np.unique(cur[live]):
                sel = live & (cur == x)
                m = mask[x]
                if m & 1:
                    success[sel] = True
                    alive[sel] = False
                    continue
                if m & 2:
                    alive[sel] = False
                    continue
                idx, pr = row(int(x), int(r["pi"][k, x]))
                nxt = idx[rng.choice(len(pr), size=int(sel.sum()), p=pr)]
                state[sel] = nxt
                lost = sel & (state < 0)
                alive[lost] = False
        fin = alive & ((mask[np.maximum(state, 0)] & 1) != 0) & (state >= 0)
        success |= fin
        freq = success.mean()
        v = r["V"][x0]
        sd = math.sqrt(max(v * (1 - v), 1e-12) / runs)
        assert abs(freq - v) <= 4.0 * sd + 1e-9, (x0, freq, v)
