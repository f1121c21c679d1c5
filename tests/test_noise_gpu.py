"""GPU parity of the noise distributions of Sec. 6.2 (uniform, exponential,
beta with integer shapes, multiplicative Gaussian): the CUDA path through the
C ABI against the FP64 oracle in every row mode and precision, window origins
bit-exact, and the Gaussian default unchanged."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import compare_rows, compare_synthesis, load_engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amy():
    return load_engine()


NOISES = [
    ("uniform", lambda n: [[0.45] * n], 2e-2, None),
    ("exponential", lambda n: [[3.0] * n], 5e-2, None),
    ("beta", lambda n: [[2.0] * n, [3.0] * n, [-0.5] * n, [0.7] * n], 1e-2, None),
    ("beta", lambda n: [[1.0] * n, [1.0] * n, [-0.4] * n, [0.4] * n], 1e-2, None),
    ("mult_gaussian", lambda n: [[0.15] * n], 0.0, None),            # dense rows
    ("mult_gaussian", lambda n: [[0.15] * n], 0.0, "explicit"),      # explicit odd windows
]


def _noisy(kind, prm, gamma, win, n, per_dim, seed, kind_spec=W.REACH_AVOID, horizon=4):
    rng = np.random.default_rng(seed)
    window = [5] * n if win == "explicit" else None
    w = W.random_affine(rng, n, per_dim, 3, gamma=gamma if gamma > 0 else 0.0, window=window,
                        kind=kind_spec, horizon=horizon)
    p = dataclasses.replace(w.problem, noise=kind, noise_params=prm(n), name=f"{kind}_{n}")
    if gamma == 0.0 and window is None:
        p.gamma = 0.0
    return W.with_sizes(w, problem=p)


@pytest.mark.parametrize("kind,prm,gamma,win", NOISES)
@pytest.mark.parametrize("n,per_dim", [(2, [31, 27]), (3, [8, 9, 7])])
def test_noise_kinds_every_mode(amy, kind, prm, gamma, win, n, per_dim):
    w = _noisy(kind, prm, gamma, win, n, per_dim, seed=70 + n)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for tmode in ["otf", "stored_separable", "stored_factored", "stored_full"]:
        compare_synthesis(amy, w, tmode, "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32", ref=ref)
    compare_synthesis(amy, w, "otf", "fp64", ref=ref)
    compare_synthesis(amy, w, "stored_full", "fp64", ref=ref)


@pytest.mark.parametrize("kind,prm,gamma,win", NOISES)
def test_noise_rows_origins_exact(amy, kind, prm, gamma, win):
    """Window origins bit-exact and masses within rounding (FP64 on the fly,
    FP32 tables) against the oracle's rows."""
    w = _noisy(kind, prm, gamma, win, 3, [8, 9, 7], seed=91)
    for tmode, prec, tol in [("otf", "fp64", 1e-13), ("stored_separable", "fp32", 2e-6)]:
        mism, worst = compare_rows(amy, w, tmode, prec, n_pairs=128, seed=3)
        assert mism == 0 and worst <= tol, (kind, tmode, mism, worst)


def test_noise_high_d_plane_kernel(amy):
    """Uniform noise on the 6-D traffic ring (tables: the plane kernel) and
    multiplicative noise on a 4-D ring with explicit windows."""
    w = W.traffic6(n_per_dim=6, horizon=2)
    p = dataclasses.replace(w.problem, noise="uniform", noise_params=[[0.8] * 6])
    w = W.with_sizes(w, problem=p)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    with amy.amy_build(w.problem, tmode="stored_separable", prec="fp32_kahan") as h:
        assert amy.amy_info(h)["backup_kernel"] == 7
    compare_synthesis(amy, w, "stored_separable", "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp32_kahan", ref=ref)
    w4 = W.rooms7(n_per_dim=5, horizon=3, n_rooms=4)
    p4 = dataclasses.replace(w4.problem, noise="mult_gaussian", noise_params=[[1e-3] * 4])
    w4 = W.with_sizes(w4, problem=p4)
    ref4 = oracle.synthesize(w4.problem, w4.spec, w4.horizon, want_all=True)
    for tmode in ["stored_separable", "otf"]:
        compare_synthesis(amy, w4, tmode, "fp32_kahan", ref=ref4)


def test_noise_invalid_rejected(amy):
    base = W.random_affine(np.random.default_rng(2), 2, [9, 9], 3, gamma=1e-2).problem
    bad = [dataclasses.replace(base, noise="beta", noise_params=[[2.5, 2.0], [2.0, 2.0], [-1, -1], [1, 1]]),
           dataclasses.replace(base, noise="uniform", noise_params=[[0.2, 0.2]], gamma=10.0),
           dataclasses.replace(base, noise="exponential", noise_params=[[1.0, 1.0]], gamma=2.0),
           dataclasses.replace(base, noise="mult_gaussian", noise_params=[[0.2, 0.2]]),
           dataclasses.replace(base, noise="uniform", noise_params=[[-0.3, 0.3]])]
    for p in bad:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_build(p, tmode="otf", prec="fp32")
        assert "INVALID_ARG" in str(e.value), p.noise


USER_DENSITIES = [
    ("bump", "exp(-t*t/(2*0.3*0.3))", -1.2, 1.2),
    ("triangle", "fmax(0, 0.5 - fabs(t - 0.1))", -0.4, 0.6),
    ("two humps", "exp(-(t - 0.35)*(t - 0.35)/0.02) + 0.5*exp(-(t + 0.3)*(t + 0.3)/0.05)", -1.0, 1.0),
]


@pytest.mark.parametrize("name,pdf,lo,hi", USER_DENSITIES)
@pytest.mark.parametrize("n,per_dim", [(2, [31, 27]), (3, [8, 9, 7])])
def test_user_densities_every_mode(amy, name, pdf, lo, hi, n, per_dim):
    """The user's density and support box (Sec. 6.2), tabulated at build time
    (NVRTC) on both sides with the same quadrature and interpolation, in every
    row mode and precision, against the oracle."""
    rng = np.random.default_rng(80 + n)
    w = W.random_affine(rng, n, per_dim, 3, gamma=1e-2, kind=W.REACH_AVOID, horizon=4)
    p = dataclasses.replace(w.problem, noise="user", noise_params=[[lo] * n, [hi] * n], noise_pdf=[pdf] * n,
                            name=f"user_{name}_{n}")
    w = W.with_sizes(w, problem=p)
    ref = oracle.synthesize(w.problem, w.spec, w.horizon, want_all=True)
    for tmode in ["otf", "stored_separable", "stored_factored", "stored_full"]:
        compare_synthesis(amy, w, tmode, "fp32_kahan", ref=ref)
    compare_synthesis(amy, w, "otf", "fp64", ref=ref)
    compare_synthesis(amy, w, "stored_full", "fp64", ref=ref)
    for tmode, prec, tol in [("otf", "fp64", 1e-13), ("stored_separable", "fp32", 2e-6)]:
        mism, worst = compare_rows(amy, w, tmode, prec, n_pairs=128, seed=4)
        assert mism == 0 and worst <= tol, (name, tmode, mism, worst)


def test_user_density_rejected(amy):
    base = W.random_affine(np.random.default_rng(2), 2, [9, 9], 3, gamma=1e-2).problem
    for pdf, lo, hi in [("t", -1.0, 1.0), ("0", -1.0, 1.0), ("exp(t", -1.0, 1.0), ("x0", -1.0, 1.0),
                        ("1", 1.0, 1.0)]:
        p = dataclasses.replace(base, noise="user", noise_params=[[lo, lo], [hi, hi]], noise_pdf=[pdf, "1"])
        with pytest.raises(amy.AmyError) as e:
            amy.amy_build(p, tmode="otf", prec="fp32")
        assert "INVALID_ARG" in str(e.value), pdf
    p = dataclasses.replace(base, noise="user", noise_params=[[-1, -1], [1, 1]], noise_pdf=["1", "1"])
    srv = amy.amy_server_create(batched=True, max_slots=4)
    try:
        with pytest.raises(amy.AmyError) as e:
            amy.amy_submit(srv, W.with_sizes(W.random_affine(np.random.default_rng(2), 2, [9, 9], 3), problem=p))
        assert "UNSUPPORTED" in str(e.value)
    finally:
        srv.close()
    import torch
    V = torch.empty(81, dtype=torch.float32, device="cuda")
    P = torch.empty(81, dtype=torch.int16, device="cuda")
    w = W.with_sizes(W.random_affine(np.random.default_rng(2), 2, [9, 9], 3), problem=p)
    with pytest.raises(amy.AmyError) as e:
        amy.amy_synthesize_noalloc(w.problem, w.spec, w.horizon, V, P)
    assert "UNSUPPORTED" in str(e.value)
