"""Pins of the oracle's user densities (Sec. 6.2: the user supplies the
density of the noise and a box enclosing its support).

The oracle integrates the density with the 8-point Gauss-Legendre rule per
knot interval and interpolates the normalised CDF between knots by cubic
Hermite polynomials.  Pinned here against closed forms: the rule integrates
polynomials up to degree 15 exactly; a constant density gives the built-in
uniform noise's masses and values, a (t - lo)(hi - t) density the built-in
beta(2, 2)'s (cubic CDF: exact), a beta(2, 3) and a Gaussian density agree
with the built-in kinds within the interpolation error; densities are
normalised over the box; invalid ones are refused.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("deg", list(range(16)))
def test_gauss_legendre_exact_to_degree_15(deg):
    a, b = -0.7, 1.3
    text = "1" if deg == 0 else "*".join(["t"] * deg)
    want = (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
    assert oracle.gauss_legendre8(text, a, b) == pytest.approx(want, rel=1e-13, abs=1e-15)


def test_gauss_legendre_is_not_exact_at_degree_16():
    a, b = 0.0, 1.0
    got = oracle.gauss_legendre8("*".join(["t"] * 16), a, b)
    assert abs(got - 1.0 / 17.0) > 1e-12


def test_cdf_of_constant_density_is_linear():
    ts = np.linspace(-1.5, 1.5, 61)
    got = oracle.user_cdf("3.5", -1.0, 1.0, ts)
    assert np.max(np.abs(got - np.clip((ts + 1.0) / 2.0, 0.0, 1.0))) < 1e-15


def test_cdf_of_quadratic_density_is_exact():
    """(t - lo)(hi - t) on [lo, hi]: the beta(2, 2) CDF, a cubic, exactly."""
    lo, hi = -0.4, 0.8
    ts = np.linspace(lo - 0.1, hi + 0.1, 97)
    z = np.clip((ts - lo) / (hi - lo), 0.0, 1.0)
    want = 3 * z ** 2 - 2 * z ** 3
    got = oracle.user_cdf(f"(t - ({lo}))*({hi} - t)", lo, hi, ts)
    assert np.max(np.abs(got - want)) < 1e-14


def test_cdf_of_gaussian_density():
    s = 0.3
    ts = np.linspace(-1.0, 1.0, 41)
    got = oracle.user_cdf(f"exp(-t*t/(2*{s}*{s}))", -8 * s, 8 * s, ts)
    want = np.array([0.5 * math.erfc(-t / (s * math.sqrt(2))) for t in ts])
    assert np.max(np.abs(got - want)) < 1e-10


def _grid_problem(noise, prm, pdf=None, window=None):
    rng = np.random.default_rng(52)
    w = W.random_affine(rng, 2, [25, 21], 3, gamma=0.0, window=window or [9, 7], kind=W.REACH_AVOID, horizon=4)
    p = dataclasses.replace(w.problem, noise=noise, noise_params=prm, noise_pdf=pdf)
    return W.with_sizes(w, problem=p)


def _rows(p, pairs):
    return [oracle.row(p, x, u) for x, u in pairs]


def test_constant_density_is_the_uniform_noise():
    a = 0.35
    wu = _grid_problem("uniform", [[a, a]])
    wd = _grid_problem("user", [[-a, -a], [a, a]], pdf=["1", "2.5"])
    pairs = [(0, 0), (100, 1), (260, 2), (524, 0)]
    for (oa, pa), (ob, pb) in zip(_rows(wu.problem, pairs), _rows(wd.problem, pairs)):
        assert np.array_equal(oa, ob) and np.max(np.abs(pa - pb)) < 1e-14
    ra = oracle.synthesize(wu.problem, wu.spec, wu.horizon)
    rb = oracle.synthesize(wd.problem, wd.spec, wd.horizon)
    assert np.max(np.abs(ra["V"] - rb["V"])) < 1e-13
    sure = np.minimum(ra["gap"], rb["gap"]) > 1e-9
    assert np.array_equal(ra["pi"][sure], rb["pi"][sure])


@pytest.mark.parametrize("alpha,beta,dens,tol", [(2, 2, "(t - ({lo}))*({hi} - t)", 1e-13),
                                                  (2, 3, "(t - ({lo}))*({hi} - t)*({hi} - t)", 1e-9),
                                                  (1, 4, "({hi} - t)*({hi} - t)*({hi} - t)", 1e-9)])
def test_polynomial_densities_are_the_beta_noise(alpha, beta, dens, tol):
    lo, hi = -0.5, 0.7
    wb = _grid_problem("beta", [[alpha] * 2, [beta] * 2, [lo] * 2, [hi] * 2])
    text = dens.format(lo=lo, hi=hi)
    wd = _grid_problem("user", [[lo] * 2, [hi] * 2], pdf=[text, text])
    pairs = [(0, 0), (77, 1), (300, 2), (500, 1)]
    for (oa, pa), (ob, pb) in zip(_rows(wb.problem, pairs), _rows(wd.problem, pairs)):
        assert np.array_equal(oa, ob) and np.max(np.abs(pa - pb)) < tol


def test_gaussian_density_is_the_gaussian_noise():
    wg = _grid_problem("gaussian", None)
    s = wg.problem.sigma
    pdf = [f"exp(-t*t/(2*{v!r}*{v!r}))" for v in s]
    wd = _grid_problem("user", [[-8 * v for v in s], [8 * v for v in s]], pdf=pdf)
    pairs = [(0, 0), (140, 1), (333, 2), (520, 0)]
    for (oa, pa), (ob, pb) in zip(_rows(wg.problem, pairs), _rows(wd.problem, pairs)):
        assert np.array_equal(oa, ob) and np.max(np.abs(pa - pb)) < 1e-9


def test_density_normalised_over_the_box():
    a = 0.35
    w1 = _grid_problem("user", [[-a, -a], [a, a]], pdf=["exp(-t)", "1 + t*t"])
    w2 = _grid_problem("user", [[-a, -a], [a, a]], pdf=["7*exp(-t)", "0.5*(1 + t*t)"])
    for (oa, pa), (ob, pb) in zip(_rows(w1.problem, [(10, 1), (400, 2)]), _rows(w2.problem, [(10, 1), (400, 2)])):
        assert np.array_equal(oa, ob) and np.max(np.abs(pa - pb)) < 1e-14


@pytest.mark.parametrize("pdf,lo,hi", [("t", -1.0, 1.0), ("0", -1.0, 1.0), ("1", 1.0, 1.0), ("x0", -1.0, 1.0),
                                       ("exp(t", -1.0, 1.0), ("log(t)", -1.0, 1.0)])
def test_invalid_densities_refused(pdf, lo, hi):
    with pytest.raises(ValueError):
        oracle.user_cdf(pdf, lo, hi, [0.0])
