"""Seeded synthetic problem descriptions shared by the tests and the benchmark.

This module only *describes* problems (grids, system parameters, noise,
cutting rule, specification boxes, request streams).  It holds none of the
method's arithmetic: no means, windows, cell masses or backups are computed
here, so both the CUDA path and the CPU oracle receive identical inputs.

The five workloads follow the paper's case studies (robot Sec. 7, room
temperature and road traffic Sec. 8) reshaped to the sizes the engine is
measured on:

  robot_lin    2-D x+ = x + u, dense rows, reach-avoid, horizon 8 (FP64)
  unicycle     3-D nonlinear unicycle, gamma = 1e-6, reach, horizon 32
  rooms7       7-room ring temperature network, window 3^7, safety, horizon 10
  served       stream of random linear 2-4-D problems (continuous batching)
  traffic6     6-D linear traffic ring, window 5^6, safety, horizon 8
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED = 20050619

AFFINE = "affine"        # mu = A_u x + c_u, A_u and c_u given per discrete input
UNICYCLE = "unicycle"    # mu = (x + tau v cos th, y + tau v sin th, th + tau w)
EXPR = "expr"            # mu_d = a C-syntax expression over x0.., u0.., w0.. and the params p0..

SAFETY = "safety"
REACH = "reach"
REACH_AVOID = "reach_avoid"

Box = Tuple[Sequence[float], Sequence[float]]


@dataclass
class Problem:
    """A finite-MDP abstraction request: grids, system, noise and cutting rule."""
    name: str
    x_lb: List[float]
    x_eta: List[float]
    x_count: List[int]
    x_periodic: List[int]
    u_lb: List[float]
    u_eta: List[float]
    u_count: List[int]
    sys_kind: str
    params: np.ndarray          # float64, layout per sys_kind
    sigma: List[float]          # per-dim noise standard deviation
    gamma: float = 0.0          # cutting threshold (0 = dense when window is None)
    window: Optional[List[int]] = None
    # disturbance grid (empty: none); with one, params holds (A, c) per
    # (input, disturbance) pair, disturbance fastest
    w_lb: List[float] = field(default_factory=list)
    w_eta: List[float] = field(default_factory=list)
    w_count: List[int] = field(default_factory=list)
    # noise distribution per dim: "gaussian" (sigma), "uniform" ([a]),
    # "exponential" ([rate]), "beta" ([alpha], [beta], [lo], [hi]; integer
    # shapes), "mult_gaussian" ([s]: std s * |x_d|); noise_params holds one
    # list of n values per parameter
    noise: str = "gaussian"
    noise_params: Optional[List[List[float]]] = None
    # sys_kind "expr": one expression per state dim (the text right-hand side
    # of Sec. 3); params are its p0, p1, ...
    exprs: Optional[List[str]] = None
    # noise "user": one density per dim in the variable t (Sec. 6.2: the user
    # gives the density and a box enclosing its support, noise_params
    # [[lo...], [hi...]]); it is normalised over the box
    noise_pdf: Optional[List[str]] = None

    @property
    def n(self) -> int:
        return len(self.x_count)

    @property
    def m(self) -> int:
        return len(self.u_count)

    @property
    def n_states(self) -> int:
        return int(np.prod(self.x_count, dtype=np.int64))

    @property
    def n_inputs(self) -> int:
        return int(np.prod(self.u_count, dtype=np.int64))

    @property
    def n_disturbances(self) -> int:
        return int(np.prod(self.w_count, dtype=np.int64)) if self.w_count else 1


@dataclass
class Spec:
    kind: str
    safe: Optional[Box] = None
    targets: List[Box] = field(default_factory=list)
    avoids: List[Box] = field(default_factory=list)


@dataclass
class Workload:
    problem: Problem
    spec: Spec
    horizon: int
    precision: str = "fp32"     # "fp64", "fp32", "fp32_kahan"
    tmode: str = "otf"          # "otf", "stored_full", "stored_factored"
    v_store: str = "native"     # "native", "bf16", "u16" (16-bit storage of V between backups)


def input_centres(p: Problem) -> np.ndarray:
    """All discrete input points in C order (last input dim fastest)."""
    axes = [p.u_lb[d] + np.arange(p.u_count[d], dtype=np.float64) * p.u_eta[d]
            for d in range(p.m)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


def affine_params(A_list: Sequence[np.ndarray], c_list: Sequence[np.ndarray]) -> np.ndarray:
    """Pack per-input (A_u, c_u) as [A_u row-major, c_u] for each u in order."""
    out = []
    for A, c in zip(A_list, c_list):
        out.append(np.asarray(A, dtype=np.float64).reshape(-1))
        out.append(np.asarray(c, dtype=np.float64).reshape(-1))
    return np.concatenate(out)


def linear_system_params(A: np.ndarray, B: np.ndarray, ucs: np.ndarray,
                         c0: Optional[np.ndarray] = None) -> np.ndarray:
    """x+ = A x + B u (+ c0): the same A for every input, c_u = B u (+ c0)."""
    n = A.shape[0]
    cs = []
    for u in ucs:
        c = B @ u
        if c0 is not None:
            c = c + c0
        cs.append(c)
    return affine_params([A] * len(ucs), cs)


# ---------------------------------------------------------------------------
# robot_lin: 2-D linear robot (shape of the paper's Sec. 7 robot example)
# ---------------------------------------------------------------------------
def robot_lin(n_per_dim: int = 41, horizon: int = 8, precision: str = "fp64") -> Workload:
    lb, eta = -5.0, 0.25
    p = Problem(
        name=f"robot_lin_{n_per_dim}",
        x_lb=[lb, lb], x_eta=[eta, eta], x_count=[n_per_dim, n_per_dim], x_periodic=[0, 0],
        u_lb=[-1.0, -1.0], u_eta=[0.5, 0.5], u_count=[5, 5],
        sys_kind=AFFINE, params=np.zeros(0), sigma=[0.2, 0.2], gamma=0.0, window=None)
    ucs = input_centres(p)
    p.params = linear_system_params(np.eye(2), np.eye(2), ucs)
    spec = Spec(REACH_AVOID, targets=[([3.0, 3.0], [5.0, 5.0])], avoids=[([-1.0, -1.0], [1.0, 1.0])])
    return Workload(p, spec, horizon, precision=precision, tmode="stored_full")


def disturbed_affine_params(A_of, c_of, ucs: np.ndarray, wcs: np.ndarray) -> np.ndarray:
    """Pack (A, c) per (input, disturbance) pair, disturbance fastest:
    A_of(u, w) and c_of(u, w) take the pair's centres."""
    As, cs = [], []
    for u in ucs:
        for w in wcs:
            As.append(A_of(u, w))
            cs.append(c_of(u, w))
    return affine_params(As, cs)


def disturbance_centres(p: Problem) -> np.ndarray:
    """All disturbance points in C order (last dim fastest)."""
    axes = [p.w_lb[d] + np.arange(p.w_count[d], dtype=np.float64) * p.w_eta[d] for d in range(len(p.w_count))]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


# ---------------------------------------------------------------------------
# robot_dist: the paper's 2-D robot of Sec. 7 with its bounded disturbance,
# x1+ = x1 + tau v1 cos(v2) + w, x2+ = x2 + tau v1 sin(v2) + w (the second
# line read with v1, like the first), tau = 10, X = [-10,10]^2 at 0.5,
# U = [-1,1]^2, W = [-1,1] at 0.2, Sigma = diag(0.75, 0.75), gamma = 1e-3
# (13 x 13 windows), safety in X for 8 steps.  Inputs at 0.2 give the
# 41^2 x 11^2 = 203401 state-input pairs of the paper's safety rows.
# ---------------------------------------------------------------------------
def robot_dist(n_per_dim: int = 41, u_step: float = 0.2, w_step: float = 0.2, horizon: int = 8,
               kind: str = SAFETY) -> Workload:
    lo, hi = -10.0, 10.0
    eta = (hi - lo) / (n_per_dim - 1)
    nu1 = int(round(2.0 / u_step)) + 1
    nw = int(round(2.0 / w_step)) + 1
    tau = 10.0
    p = Problem(
        name=f"robot_dist_{n_per_dim}",
        x_lb=[lo, lo], x_eta=[eta, eta], x_count=[n_per_dim, n_per_dim], x_periodic=[0, 0],
        u_lb=[-1.0, -1.0], u_eta=[u_step, u_step], u_count=[nu1, nu1],
        sys_kind=AFFINE, params=np.zeros(0), sigma=[math.sqrt(0.75)] * 2, gamma=1e-3, window=None,
        w_lb=[-1.0], w_eta=[w_step], w_count=[nw])
    p.params = disturbed_affine_params(
        lambda u, w: np.eye(2),
        lambda u, w: np.array([tau * u[0] * math.cos(u[1]) + w[0], tau * u[0] * math.sin(u[1]) + w[0]]),
        input_centres(p), disturbance_centres(p))
    if kind == SAFETY:
        spec = Spec(SAFETY, safe=([lo, lo], [hi, hi]))
    else:
        spec = Spec(REACH_AVOID, targets=[([5.0, 5.0], [10.0, 10.0])], avoids=[([-2.0, -2.0], [2.0, 2.0])])
    return Workload(p, spec, horizon, precision="fp32", tmode="otf")


def robot_dist_expr(n_per_dim: int = 41, u_step: float = 0.2, w_step: float = 0.2, horizon: int = 8,
                    kind: str = SAFETY) -> Workload:
    """The robot of Sec. 7 given as text, as the tool's configuration file
    gives it: x1+ = x1 + tau nu1 cos(nu2) + w, x2+ = x2 + tau nu1 sin(nu2) + w
    (the same system as robot_dist, whose affine records restate it per
    input and disturbance point)."""
    w = robot_dist(n_per_dim, u_step, w_step, horizon, kind)
    p = replace(w.problem, name=f"robot_dist_expr_{n_per_dim}", sys_kind=EXPR, params=np.array([10.0]),
                exprs=["x0 + (p0*u0*cos(u1) + w0)", "x1 + (p0*u0*sin(u1) + w0)"])
    return replace(w, problem=p)


# ---------------------------------------------------------------------------
# unicycle: 3-D nonlinear unicycle, theta periodic
# ---------------------------------------------------------------------------
def unicycle(nxy: int = 51, nth: int = 30, horizon: int = 32, precision: str = "fp32",
             tmode: str = "stored_factored", target=(8.0, 10.0)) -> Workload:
    p = Problem(
        name=f"unicycle_{nxy}x{nxy}x{nth}",
        x_lb=[0.0, 0.0, -math.pi], x_eta=[0.2, 0.2, 2.0 * math.pi / nth],
        x_count=[nxy, nxy, nth], x_periodic=[0, 0, 1],
        u_lb=[0.0, -1.0], u_eta=[0.25, 0.25], u_count=[5, 9],
        sys_kind=UNICYCLE, params=np.array([0.1]), sigma=[0.05, 0.05, 0.05],
        gamma=1e-6, window=None)
    lo, hi = target
    spec = Spec(REACH, targets=[([lo, lo, -10.0], [hi, hi, 10.0])])
    return Workload(p, spec, horizon, precision=precision, tmode=tmode)


# ---------------------------------------------------------------------------
# rooms7: 7-room circular temperature network, one shared heater input
# ---------------------------------------------------------------------------
def rooms7(n_per_dim: int = 9, horizon: int = 10, n_rooms: int = 7,
           tmode: str = "otf") -> Workload:
    eta_c, beta, theta, Te, Th = 0.1, 0.022, 0.05, -1.0, 50.0
    lo, hi = 19.0, 21.0
    step = (hi - lo) / (n_per_dim - 1)
    nus = [0.0, 0.15, 0.3, 0.45, 0.6]
    A_list, c_list = [], []
    for nu in nus:
        A = np.zeros((n_rooms, n_rooms))
        for i in range(n_rooms):
            A[i, i] = 1.0 - 2.0 * eta_c - beta - theta * nu
            A[i, (i - 1) % n_rooms] += eta_c
            A[i, (i + 1) % n_rooms] += eta_c
        A_list.append(A)
        c_list.append(np.full(n_rooms, beta * Te + theta * Th * nu))
    p = Problem(
        name=f"rooms{n_rooms}_{n_per_dim}",
        x_lb=[lo] * n_rooms, x_eta=[step] * n_rooms, x_count=[n_per_dim] * n_rooms,
        x_periodic=[0] * n_rooms,
        u_lb=[0.0], u_eta=[0.15], u_count=[5],
        sys_kind=AFFINE, params=affine_params(A_list, c_list),
        sigma=[0.02] * n_rooms, gamma=0.0, window=[3] * n_rooms)
    spec = Spec(SAFETY, safe=([lo] * n_rooms, [hi] * n_rooms))
    return Workload(p, spec, horizon, precision="fp32_kahan", tmode=tmode)


# ---------------------------------------------------------------------------
# traffic6: 6-D linear traffic ring, two binary on-ramp lights
# ---------------------------------------------------------------------------
def traffic6(n_per_dim: int = 21, horizon: int = 8, n_cells: int = 6, window: int = 5,
             v_store: str = "native", wrap: bool = True) -> Workload:
    A = np.zeros((n_cells, n_cells))
    for i in range(n_cells):
        A[i, i] = 0.6
        if wrap or i - 1 >= 0:
            A[i, (i - 1) % n_cells] = 0.25
        if wrap or i + 1 < n_cells:
            A[i, (i + 1) % n_cells] = 0.05
    B = np.zeros((n_cells, 2))
    B[0, 0] = 6.0
    B[2 % n_cells, 1] = 8.0
    p = Problem(
        name=f"traffic{n_cells}_{n_per_dim}",
        x_lb=[0.0] * n_cells, x_eta=[1.0] * n_cells, x_count=[n_per_dim] * n_cells,
        x_periodic=[0] * n_cells,
        u_lb=[0.0, 0.0], u_eta=[1.0, 1.0], u_count=[2, 2],
        sys_kind=AFFINE, params=np.zeros(0), sigma=[0.5] * n_cells, gamma=0.0,
        window=[window] * n_cells)
    p.params = linear_system_params(A, B, input_centres(p))
    safe_hi = float(min(18.0, n_per_dim - 1 - 2))
    spec = Spec(SAFETY, safe=([0.0] * n_cells, [safe_hi] * n_cells))
    return Workload(p, spec, horizon, precision="fp32_kahan", tmode="otf", v_store=v_store)


def traffic_text(n_per_dim: int = 21, horizon: int = 8, n_cells: int = 6, window: int = 5,
                 capacity: float = 12.0) -> Workload:
    """A nonlinear traffic ring given as text: each cell keeps 0.6 of its
    vehicles, takes 0.25 of its upstream neighbour's -- at most the capacity
    p0 (a saturating flow) -- and 0.05 of its downstream one's; two inputs
    feed cells 0 and 2.  Component i reads x_{i-1}, x_i, x_{i+1} only."""
    base = traffic6(n_per_dim, horizon, n_cells, window)
    exprs = []
    for i in range(n_cells):
        up, dn = (i - 1) % n_cells, (i + 1) % n_cells
        e = f"0.6*x{i} + 0.25*fmin(x{up}, p0) + 0.05*x{dn}"
        if i == 0:
            e += " + 6*u0"
        if i == 2 % n_cells:
            e += " + 8*u1"
        exprs.append(e)
    p = replace(base.problem, name=f"traffic_text{n_cells}_{n_per_dim}", sys_kind=EXPR,
                params=np.array([capacity]), exprs=exprs)
    return replace(base, problem=p)


# ---------------------------------------------------------------------------
# served: stream of random linear problems (2-4 dims)
# ---------------------------------------------------------------------------
def _random_box(rng, lo, hi, frac_lo, frac_hi):
    lbs, ubs = [], []
    for a, b in zip(lo, hi):
        w = (b - a) * rng.uniform(frac_lo, frac_hi)
        s = rng.uniform(a, b - w)
        lbs.append(float(s))
        ubs.append(float(s + w))
    return lbs, ubs


def _boxes_overlap(b1: Box, b2: Box) -> bool:
    return all(l1 <= u2 and l2 <= u1 for l1, u1, l2, u2 in zip(b1[0], b1[1], b2[0], b2[1]))


def served_request(rng: np.random.Generator, idx: int) -> Workload:
    """One request of the served stream (random stable linear system)."""
    n = int(rng.integers(2, 5))
    per_dim = {2: 20, 3: 17, 4: 15}[n]
    lo, hi = -5.0, 5.0
    eta = (hi - lo) / (per_dim - 1)
    A = rng.standard_normal((n, n))
    rad = max(abs(np.linalg.eigvals(A)))
    A = A * (rng.uniform(0.5, 0.9) / rad)
    if rng.uniform() < 0.5:
        m = 1
        ucount = [int(rng.integers(4, 17))]
    else:
        m = 2
        k = int(rng.integers(2, 5))
        ucount = [k, k]
    ulb = [-1.0] * m
    ueta = [2.0 / (c - 1) for c in ucount]
    B = rng.normal(0.0, 0.5, size=(n, m))
    var = rng.uniform(0.05, 0.3, size=n)
    sigma = [float(math.sqrt(v)) for v in var]
    p = Problem(
        name=f"served_{idx}_n{n}",
        x_lb=[lo] * n, x_eta=[eta] * n, x_count=[per_dim] * n, x_periodic=[0] * n,
        u_lb=ulb, u_eta=ueta, u_count=ucount,
        sys_kind=AFFINE, params=np.zeros(0), sigma=sigma, gamma=1e-3, window=None)
    p.params = linear_system_params(A, B, input_centres(p))
    if rng.uniform() < 0.5:
        spec = Spec(SAFETY, safe=_random_box(rng, [lo] * n, [hi] * n, 0.6, 0.9))
    else:
        while True:
            t = _random_box(rng, [lo] * n, [hi] * n, 0.10, 0.25)
            a = _random_box(rng, [lo] * n, [hi] * n, 0.10, 0.25)
            if not _boxes_overlap(t, a):
                break
        spec = Spec(REACH_AVOID, targets=[t], avoids=[a])
    horizon = int(rng.integers(5, 51))
    return Workload(p, spec, horizon, precision="fp32", tmode="otf")


def served_stream(n_requests: int = 256, seed: int = SEED) -> List[Workload]:
    rng = np.random.default_rng(seed)
    return [served_request(rng, i) for i in range(n_requests)]


def poisson_arrivals(n: int, rate_per_s: float, seed: int = SEED + 1) -> np.ndarray:
    """Arrival offsets in seconds of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


# ---------------------------------------------------------------------------
# small problems used by parity tests
# ---------------------------------------------------------------------------
def random_affine(rng: np.random.Generator, n: int, per_dim: Sequence[int], n_u: int,
                  gamma: float = 1e-3, window: Optional[List[int]] = None,
                  periodic: Optional[List[int]] = None, kind: str = REACH_AVOID,
                  horizon: int = 4) -> Workload:
    lo, hi = -3.0, 3.0
    etas = [(hi - lo) / (c - 1) if c > 1 else 1.0 for c in per_dim]
    A = rng.standard_normal((n, n))
    A = A * (rng.uniform(0.6, 1.0) / max(abs(np.linalg.eigvals(A))))
    B = rng.normal(0.0, 0.6, size=(n, 1))
    p = Problem(
        name=f"rand_affine_n{n}",
        x_lb=[lo] * n, x_eta=etas, x_count=list(per_dim),
        x_periodic=list(periodic) if periodic else [0] * n,
        u_lb=[-1.0], u_eta=[2.0 / max(n_u - 1, 1)], u_count=[n_u],
        sys_kind=AFFINE, params=np.zeros(0),
        sigma=[float(s) for s in rng.uniform(0.15, 0.5, size=n)],
        gamma=gamma if window is None else 0.0, window=window)
    p.params = linear_system_params(A, B, input_centres(p))
    if kind == SAFETY:
        spec = Spec(SAFETY, safe=([lo + 0.5] * n, [hi - 0.5] * n))
    elif kind == REACH:
        spec = Spec(REACH, targets=[([1.0] * n, [3.0] * n)])
    else:
        spec = Spec(REACH_AVOID, targets=[([1.0] * n, [3.0] * n)],
                    avoids=[([-1.5] * n, [-0.2] * n)])
    return Workload(p, spec, horizon, precision="fp32")


def with_sizes(w: Workload, **kw) -> Workload:
    return replace(w, **kw)
