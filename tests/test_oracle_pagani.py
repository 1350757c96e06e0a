"""Pins of the PAGANI oracle (oracle/pagani_oracle.c) against things other than itself: exact
integrals of monomials on [-1, 1]^d (the Genz-Malik rule of degree 7 and its embedded degree-5
rule), exact integrals of polynomial integrands on boxes, Gaussian closed forms, the split axis
of integrands that vary along one axis only, and the adaptive driver against the Genz closed
forms."""
import itertools
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2302_05730_gb300 import workloads as W

sys.path.insert(0, os.path.dirname(__file__))
from closed_forms import exact   # noqa: E402


def _monomial_exact(e):
    """int over [-1, 1]^d of prod x_i^e_i."""
    out = 1.0
    for k in e:
        out *= 0.0 if k % 2 else 2.0 / (k + 1)
    return out


def _rule(U, cls, w, e):
    vals = np.prod(U ** np.asarray(e, dtype=float), axis=1)
    return sum(w[k - 1] * vals[cls == k].sum() for k in range(1, 6))


@pytest.mark.parametrize("d", [2, 3, 5, 8])
def test_point_count_and_classes(d):
    U, cls, w7, w5 = oracle.gm_rule(d)
    assert U.shape == (1 + 4 * d + 2 * d * (d - 1) + 2 ** d, d)
    assert list(np.bincount(cls, minlength=6)[1:]) == [1, 2 * d, 2 * d, 2 * d * (d - 1), 2 ** d]
    # fully symmetric: every class is closed under sign changes and axis permutations of its radii
    for k in range(1, 6):
        pts = U[cls == k]
        assert np.allclose(pts.sum(axis=0), 0.0, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_rules_integrate_every_monomial_up_to_their_degree(d):
    U, cls, w7, w5 = oracle.gm_rule(d)
    for e in itertools.product(range(8), repeat=d):
        deg = sum(e)
        if deg > 7:
            continue
        ref = _monomial_exact(e)
        assert abs(_rule(U, cls, w7, e) - ref) <= 1e-12 * 2 ** d, (e, _rule(U, cls, w7, e), ref)
        if deg <= 5:
            assert abs(_rule(U, cls, w5, e) - ref) <= 1e-12 * 2 ** d, (e, "deg5")


@pytest.mark.parametrize("d", [6, 8, 10])
def test_rules_on_sampled_monomials_in_higher_dimension(d):
    U, cls, w7, w5 = oracle.gm_rule(d)
    rng = np.random.default_rng(d)
    for _ in range(200):
        deg = int(rng.integers(0, 8))
        e = np.zeros(d, dtype=int)
        for _ in range(deg):
            e[rng.integers(0, d)] += 1
        ref = _monomial_exact(e)
        assert abs(_rule(U, cls, w7, e) - ref) <= 1e-11 * 2 ** d, (e,)
        if deg <= 5:
            assert abs(_rule(U, cls, w5, e) - ref) <= 1e-11 * 2 ** d, (e, "deg5")


def test_degrees_are_tight():
    """Degree 8 (resp. 6) monomials are not integrated exactly: the rules have exactly the
    stated degrees, so a mistake that made them trivially exact would show."""
    U, cls, w7, w5 = oracle.gm_rule(3)
    assert abs(_rule(U, cls, w7, (8, 0, 0)) - _monomial_exact((8, 0, 0))) > 1e-3
    assert abs(_rule(U, cls, w7, (4, 4, 0)) - _monomial_exact((4, 4, 0))) > 1e-3
    assert abs(_rule(U, cls, w5, (6, 0, 0)) - _monomial_exact((6, 0, 0))) > 1e-3


@pytest.mark.parametrize("d", [2, 5, 8])
def test_region_mapping_is_exact_for_polynomials(d):
    rng = np.random.default_rng(40 + d)
    for _ in range(5):
        lo = rng.uniform(0.0, 0.5, d)
        ln = rng.uniform(0.05, 0.5, d)
        vol = float(np.prod(ln))
        I, E, ax = oracle.pagani_evaluate(W.ADDITION, d, W.paper_params(W.ADDITION, d), lo, ln)
        ref = vol * float(np.sum(lo + ln / 2))
        assert abs(I - ref) <= 1e-13 * abs(ref) and E <= 1e-13 * abs(ref)
        I, E, ax = oracle.pagani_evaluate(W.CONSTANT, d, W.constant_params(d, 2.5), lo, ln)
        assert abs(I - 2.5 * vol) <= 1e-13 * 2.5 * vol and E <= 1e-13 * 2.5 * vol
        # a constant has no preferred axis: the longest side is split
        assert ax == int(np.argmax(ln))


def test_gaussian_on_small_boxes_against_closed_form():
    """exp(-sum a_i^2 (x_i - u_i)^2) over a box is a product of erf differences; on boxes small
    against 1/a the degree-7 rule is accurate to many digits, and its error estimate is not
    smaller than its actual error."""
    d = 4
    rng = np.random.default_rng(7)
    a = rng.uniform(2.0, 6.0, d)
    u = rng.uniform(0.3, 0.7, d)
    par = np.concatenate([a, u])
    for h in (0.2, 0.1, 0.05):
        lo = u - h * rng.uniform(0.2, 0.8, d)
        ln = np.full(d, h)
        ref = 1.0
        for i in range(d):
            ref *= math.sqrt(math.pi) / (2 * a[i]) * (math.erf(a[i] * (lo[i] + ln[i] - u[i])) -
                                                      math.erf(a[i] * (lo[i] - u[i])))
        I, E, ax = oracle.pagani_evaluate(W.GAUSSIAN, d, par, lo, ln)
        assert abs(I - ref) <= max(E, 1e-15 * ref), (h, I, ref, E)
        assert abs(I - ref) <= 1e-3 * ref * (h / 0.2) ** 6


def test_split_axis_follows_the_varying_axis():
    d = 5
    for k in range(d):
        a = np.full(d, 0.5)
        a[k] = 12.0
        par = np.concatenate([a, np.full(d, 0.31)])
        I, E, ax, fourth = oracle.pagani_evaluate(W.GAUSSIAN, d, par, np.zeros(d), np.ones(d), want_fourth=True)
        assert ax == k and np.argmax(fourth) == k


@pytest.mark.parametrize("fid,d", [(W.GAUSSIAN, 2), (W.GAUSSIAN, 3), (W.PRODUCT_PEAK, 2), (W.OSCILLATORY, 3),
                                   (W.C0, 2), (W.CORNER_PEAK, 3)])
def test_adaptive_driver_converges_to_closed_form(fid, d):
    par = W.genz_params(fid, d, seed=3)
    ref = exact(fid, par[:d], par[d:])
    tol = 1e-6
    r = oracle.pagani_integrate(fid, d, par, tol, max_iters=60, max_regions=1 << 20, init_split=2)
    assert r["status"] == 0, r
    assert r["error"] <= tol * abs(r["estimate"]) * 1.000001
    # the error estimate is a heuristic (not a bound); the true error stays well inside 10 tol
    assert abs(r["estimate"] - ref) <= 10.0 * tol * abs(ref), (r, ref)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_lower_degree_rules_are_exact_to_their_degree_and_no_further(d):
    """R3a (centre and +-l2 e_i) and R3b (centre and +-l3 e_i) integrate every monomial of degree
    <= 3 exactly, R1 (the centre) every one of degree <= 1; none is exact one degree higher."""
    U, cls, w7, w5 = oracle.gm_rule(d)
    Wr = oracle.gm_rules(d)
    assert np.allclose(Wr[0], w7) and np.allclose(Wr[1], w5)
    for e in itertools.product(range(4), repeat=d):
        deg = sum(e)
        if deg > 3:
            continue
        ref = _monomial_exact(e)
        for r in (2, 3):
            assert abs(_rule(U, cls, Wr[r], e) - ref) <= 1e-12 * 2 ** d, (r, e)
        if deg <= 1:
            assert abs(_rule(U, cls, Wr[4], e) - ref) <= 1e-12 * 2 ** d, (4, e)
    e4 = (4,) + (0,) * (d - 1)
    e2 = (2,) + (0,) * (d - 1)
    for r in (2, 3):
        assert abs(_rule(U, cls, Wr[r], e4) - _monomial_exact(e4)) > 1e-3 * 2 ** d
    assert abs(_rule(U, cls, Wr[4], e2) - _monomial_exact(e2)) > 1e-3 * 2 ** d


def test_error_estimate_properties():
    """E is never below |R7 - R5|; it equals it when the differences of successive degrees fall
    at least fourfold, and is the largest difference otherwise; a cubic is integrated with E = 0."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        R = rng.normal(size=5)
        E = oracle.pagani_error(R)
        d7 = abs(R[0] - R[1])
        d5 = max(abs(R[1] - R[2]), abs(R[1] - R[3]))
        d3 = max(abs(R[2] - R[4]), abs(R[3] - R[4]))
        assert E >= d7
        assert E in (d7, max(d7, d5, d3))
    # geometric decay by 8 per degree: the asymptotic branch
    R = np.array([1.0, 1.0 + 1e-6, 1.0 + 1e-6 + 8e-6, 1.0 + 1e-6 - 8e-6, 1.0 + 1e-6 + 8e-6 + 64e-6])
    assert oracle.pagani_error(R) == pytest.approx(1e-6, rel=1e-9)
    # decay by 2 only: the conservative branch
    R = np.array([1.0, 1.0 + 1e-6, 1.0 + 1e-6 + 2e-6, 1.0 + 1e-6, 1.0 + 1e-6 + 2e-6 + 4e-6])
    assert oracle.pagani_error(R) == pytest.approx(max(2e-6, 6e-6, 6e-6 - 2e-6), rel=1e-9)
    # the rules on a cubic: R7 = R5 = R3a = R3b exactly, so E = 0 whatever R1 gives
    d = 3
    U, cls, _, _ = oracle.gm_rule(d)
    Wr = oracle.gm_rules(d)
    R = np.array([_rule(U, cls, Wr[r], (2, 1, 0)) + 3.0 * _rule(U, cls, Wr[r], (2, 0, 0)) for r in range(5)])
    assert oracle.pagani_error(R) <= 1e-13


@pytest.mark.parametrize("fid,d,tol", [(W.GAUSSIAN, 4, 1e-4), (W.GAUSSIAN, 5, 1e-3), (W.C0, 4, 1e-3),
                                       (W.CORNER_PEAK, 4, 1e-4), (W.PRODUCT_PEAK, 4, 1e-5)])
def test_adaptive_error_estimate_covers_the_true_error(fid, d, tol):
    """The five-rule estimate at convergence is not below the true error against the closed form
    (the two-rule |R7 - R5| alone fell below it on the d = 8 Gaussian)."""
    par = W.genz_params(fid, d, seed=0)
    ref = exact(fid, par[:d], par[d:])
    r = oracle.pagani_integrate(fid, d, par, tol, max_iters=60, max_regions=1 << 22, init_split=2)
    assert r["status"] == 0, r
    assert abs(r["estimate"] - ref) <= r["error"], (r, ref)
