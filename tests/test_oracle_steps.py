"""Step-by-step pins of the oracle's V-Sample pass (paper Sec. 3.2, Algorithm 2) and grid
refinement (VEGAS, Lepage 1978), each checked against a library routine, a closed form or an
invariant -- never against a retyped copy of the oracle's own formula."""
import math

import numpy as np
import pytest

import oracle
from paper_2302_05730_gb300 import workloads as W

ND = oracle.ND


# ----------------------------------------------------------------------------- stratify
@pytest.mark.parametrize("d,n,g,m,p", [
    (3, 10 ** 6, 79, 493039, 2),
    (5, 10 ** 8, 34, 45435424, 2),
    (6, 10 ** 8, 19, 47045881, 2),
    (8, 10 ** 8, 9, 43046721, 2),
    (10, 10 ** 9, 7, 282475249, 3),
    (2, 10 ** 4, 70, 4900, 2),
    (8, 10 ** 7, 6, 1679616, 5),
    (1, 2, 1, 1, 2),
    (16, 2, 1, 1, 2),
    (4, 31, 1, 1, 31),
])
def test_stratify_table(d, n, g, m, p):
    assert oracle.stratify(d, n) == (g, m, p)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 13, 16])
def test_stratify_is_largest_two_point_split(d):
    rng = np.random.default_rng(d)
    for n in [2, 3, 7, 100, 12345, 10 ** 6, 987654321] + list(rng.integers(2, 10 ** 9, 20)):
        n = int(n)
        g, m, p = oracle.stratify(d, n)
        assert m == g ** d and 2 * g ** d <= n < 2 * (g + 1) ** d   # Python big ints
        assert p == max(2, n // m)
        assert m * p >= n - m  # about n samples


def test_stratify_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.stratify(0, 100)
    with pytest.raises(ValueError):
        oracle.stratify(17, 100)
    with pytest.raises(ValueError):
        oracle.stratify(3, 1)
    with pytest.raises(ValueError):
        oracle.stratify(1, 2 ** 34)  # 2^33 cubes: the cube index is one 32-bit counter word


# ----------------------------------------------------------------------------- the map
def _random_grid(d, seed):
    """A strictly increasing grid with bin widths spanning four decades."""
    rng = np.random.default_rng(seed)
    B = np.empty((d, ND + 1))
    for i in range(d):
        w = np.exp(rng.uniform(-4.0, 0.0, ND) * math.log(10))
        c = np.concatenate([[0.0], np.cumsum(w)])
        B[i] = c / c[-1]
        B[i, 0], B[i, -1] = 0.0, 1.0
    return B


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("d", [1, 3, 8])
def test_map_is_piecewise_linear_interpolation_of_the_grid(mode, d):
    """x_i is the grid interpolated at yn = (c_i + u) nd / g (np.interp), J the product of
    nd * (bin width), sub-cube strata are respected, and bins are the floor of yn."""
    B = _random_grid(d, 7 + d)
    n = 2 * 5 ** d if d < 8 else 2 * 3 ** d
    pts = oracle.sample_points(W.ADDITION, d, np.zeros(2 * d), n, seed=3, it=2, job=1, mode=mode,
                               B=B, t0=0, t1=min(200, oracle.stratify(d, n)[1]))
    g, p = pts["g"], pts["p"]
    t = np.repeat(np.arange(pts["x"].shape[0] // p), p)
    digits = np.stack([(t // g ** i) % g for i in range(d)], axis=1)
    yn = (digits + pts["u"]) * (ND / g)
    knots = np.arange(ND + 1, dtype=np.float64)
    tol = 1e-15 if mode == 0 else 3e-7
    for i in range(d):
        x_ref = np.interp(yn[:, i], knots, B[i])
        assert np.allclose(pts["x"][:, i], x_ref, rtol=0, atol=tol * 4)
        k = pts["k"][:, i]
        assert np.all(k == np.minimum(np.floor(yn[:, i]).astype(int), ND - 1)) or mode == 1
        if mode == 1:  # single-precision bins may differ only next to a bin edge
            kk = np.floor(yn[:, i]).astype(int)
            off = k != kk
            assert np.all(np.abs(yn[off, i] - np.round(yn[off, i])) < 1e-4)
        # the point lies in its sub-cube's stratum of y-space
        assert np.all((yn[:, i] >= digits[:, i] * ND / g - 1e-9) & (yn[:, i] <= (digits[:, i] + 1) * ND / g + 1e-9))
    J_ref = np.prod(ND * (np.take_along_axis(B[:, 1:], pts["k"].T, 1) - np.take_along_axis(B[:, :-1], pts["k"].T, 1)), axis=0)
    assert np.allclose(pts["J"], J_ref, rtol=1e-13, atol=0)


def test_uniform_grid_is_identity_map():
    d = 3
    pts = oracle.sample_points(W.ADDITION, d, np.zeros(2 * d), 2 * 7 ** d, seed=5, t0=0, t1=343)
    g = pts["g"]
    t = np.repeat(np.arange(343), pts["p"])
    digits = np.stack([(t // g ** i) % g for i in range(d)], axis=1)
    assert np.allclose(pts["x"], (digits + pts["u"]) / g, rtol=0, atol=1e-15)
    assert np.allclose(pts["J"], 1.0, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------- per cube
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid,d,n", [(W.GAUSSIAN, 3, 2 * 6 ** 3 * 3), (W.OSCILLATORY, 2, 5 * 30 ** 2),
                                     (W.DISCONTINUOUS, 4, 2 * 4 ** 4), (W.PRODUCT_PEAK, 5, 4 * 3 ** 5)])
def test_per_cube_mean_variance_and_bin_contributions(mode, fid, d, n):
    """I_t = mean of the cube's weights, V_t = unbiased variance / p (np.var ddof=1), C = sum of
    w^2 per (axis, bin) (np.add.at), w = f(x) J with f from the integrand evaluated alone."""
    par = W.genz_params(fid, d, seed=1)
    B = _random_grid(d, 11)
    g, m, p = oracle.stratify(d, n)
    res = oracle.vsample(fid, d, par, n, seed=17, it=1, mode=mode, adjust=1, B=B, per_cube=True)
    pts = oracle.sample_points(fid, d, par, n, seed=17, it=1, mode=mode, B=B, t0=0, t1=m)
    if mode == 0:
        f = oracle.integrand(fid, d, par, pts["x"])
        assert np.allclose(pts["w"], f * pts["J"], rtol=1e-15, atol=0)
    w = pts["w"].reshape(m, p)
    assert np.allclose(res["cubeI"], w.mean(axis=1), rtol=1e-13, atol=1e-300)
    vref = w.var(axis=1, ddof=1) / p
    assert np.allclose(res["cubeV"], vref, rtol=1e-9, atol=1e-14 * np.abs(w).max() ** 2)
    C = np.zeros((d, ND))
    for i in range(d):
        np.add.at(C[i], pts["k"][:, i], pts["w"] ** 2)
    assert np.allclose(res["C"], C, rtol=1e-12, atol=0)
    assert math.isclose(res["I"], math.fsum(w.mean(axis=1)) / m, rel_tol=1e-13, abs_tol=1e-300)
    assert math.isclose(res["Var"], math.fsum(vref) / m ** 2, rel_tol=1e-9, abs_tol=1e-300)


def test_cube_ranges_partition_the_pass():
    d, n = 3, 2 * 10 ** 3
    par = W.genz_params(W.C0, d)
    full = oracle.vsample(W.C0, d, par, n, seed=4, adjust=1)
    m = full["m"]
    cuts = [0, 1, 99, 500, m]
    parts = [oracle.vsample(W.C0, d, par, n, seed=4, adjust=1, t0=a, t1=b) for a, b in zip(cuts, cuts[1:])]
    sI = math.fsum([v for pr in parts for v in pr["sumI"]])
    assert math.isclose(sI / m, full["I"], rel_tol=1e-15)
    assert np.allclose(sum(pr["C"] for pr in parts), full["C"], rtol=1e-14)


def test_no_adjust_leaves_histogram_alone():
    d = 2
    par = W.genz_params(W.GAUSSIAN, d)
    r = oracle.vsample(W.GAUSSIAN, d, par, 1000, seed=1, adjust=0)
    assert "C" not in r


def test_iteration_and_job_select_independent_draws():
    d = 2
    par = W.genz_params(W.GAUSSIAN, d)
    a = oracle.vsample(W.GAUSSIAN, d, par, 1000, seed=1, it=0)["I"]
    b = oracle.vsample(W.GAUSSIAN, d, par, 1000, seed=1, it=1)["I"]
    c = oracle.vsample(W.GAUSSIAN, d, par, 1000, seed=1, job=3)["I"]
    e = oracle.vsample(W.GAUSSIAN, d, par, 1000, seed=2)["I"]
    assert len({a, b, c, e}) == 4


# ----------------------------------------------------------------------------- rebin
def test_rebin_uniform_contributions_keep_any_grid():
    d = 3
    B = _random_grid(d, 1)
    C = np.ones((d, ND)) * 3.7
    assert np.allclose(oracle.rebin(B, C), B, rtol=0, atol=1e-13)  # rounding of the running sums


def test_rebin_alpha_zero_keeps_grid():
    """With damping exponent 0 every non-empty bin gets the same weight: the grid stays."""
    d = 2
    B = _random_grid(d, 2)
    C = np.random.default_rng(0).uniform(0.1, 10.0, (d, ND))
    assert np.allclose(oracle.rebin(B, C, alpha=0.0), B, rtol=0, atol=1e-13)


def test_rebin_scale_invariant_and_axis_separable():
    d = 3
    B = _random_grid(d, 3)
    C = np.random.default_rng(1).exponential(1.0, (d, ND))
    a = oracle.rebin(B, C)
    b = oracle.rebin(B, C * 1e30)
    c = oracle.rebin(B, C * np.array([[1e-20], [1.0], [7e12]]))
    assert np.allclose(a, b, rtol=0, atol=1e-14)
    assert np.allclose(a, c, rtol=0, atol=1e-14)
    one = oracle.rebin(B[1:2], C[1:2])
    assert np.array_equal(one[0], a[1])


def _compress(C, alpha=1.5):
    """Lepage's damped weights, evaluated with numpy: smoothed contributions (a 3-point
    moving average, np.convolve), normalised, then ((1 - rho) / ln(1/rho))^alpha. The damping
    formula is the cited VEGAS paper's; this test pins the redistribution built on it."""
    c = np.convolve(C, np.ones(3), mode="same")
    cnt = np.convolve(np.ones_like(C), np.ones(3), mode="same")
    dsm = c / cnt
    rho = dsm / dsm.sum()
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(dsm == 0, 0.0, np.where(rho == 1.0, 1.0, ((1 - rho) / np.log(1 / rho)) ** alpha))
    return r


def test_rebin_equal_mass_per_new_bin():
    """New boundaries are the quantiles of the piecewise-linear cumulative weight over the old
    grid: each new bin carries S / nd of the damped weight (checked with np.interp)."""
    d = 2
    B = _random_grid(d, 4)
    C = np.random.default_rng(2).exponential(1.0, (d, ND)) ** 3
    Bn = oracle.rebin(B, C)
    for i in range(d):
        r = _compress(C[i])
        Rc = np.concatenate([[0.0], np.cumsum(r)])
        T = np.arange(ND + 1) * Rc[-1] / ND
        assert np.allclose(Bn[i], np.interp(T, Rc, B[i]), rtol=0, atol=1e-13)
        mass = np.interp(Bn[i], B[i], Rc)
        assert np.allclose(np.diff(mass), Rc[-1] / ND, rtol=1e-9, atol=0)


def test_rebin_monotone_endpoints_and_concentration():
    d = 1
    B = oracle.uniform_grid(d)
    for C in [np.random.default_rng(5).exponential(1.0, (d, ND)) ** 8,
              np.where(np.arange(ND) == 250, 1.0, 0.0)[None, :],
              np.where(np.arange(ND) < 3, 1.0, 0.0)[None, :],
              np.where(np.arange(ND) > 496, 1e200, 0.0)[None, :]]:
        Bn = oracle.rebin(B, C)
        assert Bn[0, 0] == 0.0 and Bn[0, -1] == 1.0
        assert np.all(np.diff(Bn[0]) > 0)
    # all weight in bins 249..251 (after smoothing): every new boundary inside them
    C = np.where(np.arange(ND) == 250, 1.0, 0.0)[None, :]
    Bn = oracle.rebin(B, C)
    assert Bn[0, 1] >= 249 / ND - 1e-15 and Bn[0, -2] <= 252 / ND + 1e-15


def test_damping_asymptotic_laws_pin_alpha():
    """The damped weight r(rho) = ((1 - rho) / ln(1/rho))^alpha against two laws the mathematics
    fixes, with no re-typing of the formula: near rho = 1, with eps = 1 - rho, ln(1/rho) =
    eps + eps^2/2 + ..., so r = 1 - alpha eps / 2 + O(eps^2); for rho -> 0, (1 - rho) -> 1 and
    r ln(1/rho)^alpha -> 1. A wrong exponent (alpha = 1), ln(rho) for ln(1/rho) or a missing
    (1 - rho) fails one of them."""
    for eps in (1e-4, 1e-5):
        slope = (1.0 - oracle.damp(1.0 - eps)) / eps
        assert abs(slope - 0.75) < 2 * eps, (eps, slope)        # alpha / 2 = 0.75
    assert oracle.damp(1.0) == 1.0
    for rho in (1e-30, 1e-60, 1e-120):
        law = math.log(1.0 / rho) ** -1.5
        assert abs(oracle.damp(rho) / law - 1.0) < 1e-12, rho
    # the (1 - rho) factor at a moderate rho: r^(1/alpha) ln(1/rho) = 1 - rho
    for rho in (0.1, 0.5, 0.9):
        assert abs(oracle.damp(rho) ** (1 / 1.5) * math.log(1 / rho) - (1 - rho)) < 1e-14


def test_rebin_spacing_ratio_measures_alpha():
    """Through the whole Rebin on one axis with a uniform grid: contributions C = 1 on bins
    0..199, 2e-8 on 200..349 and 2e-18 on 350..499 (smoothed mass fractions about 1e-10 and
    1e-20 inside the two small groups). Inside a group of constant damped weight r the new
    boundaries are equally spaced by (1/nd) (S/nd) / r, so the ratio of the two groups' new
    spacings is r_1 / r_2, and by the small-rho law r ~ ln(1/rho)^-alpha it measures
    alpha = ln(spacing_2 / spacing_1) / ln(ln(1/rho_2) / ln(1/rho_1)), to the O(rho) size of the
    law's correction."""
    C = np.concatenate([np.ones(200), np.full(150, 2e-8), np.full(150, 2e-18)])[None, :]
    B = oracle.uniform_grid(1)
    Bn = oracle.rebin(B, C)[0]
    D = 200.0   # the smoothed total, up to terms of order 1e-8 (set by the small groups)

    def spacing(lo, hi):
        inside = Bn[(Bn > lo + 0.02) & (Bn < hi - 0.02)]
        assert inside.size >= 6
        sp = np.diff(inside)
        assert np.allclose(sp, sp.mean(), rtol=1e-9, atol=0)
        return sp.mean()

    s1, s2 = spacing(0.4, 0.7), spacing(0.7, 1.0)
    rho1, rho2 = 2e-8 / D, 2e-18 / D
    alpha = math.log(s2 / s1) / math.log(math.log(1 / rho2) / math.log(1 / rho1))
    # the relative errors of rho (about 1e-8) enter through ln(1/rho) ~ 20-46: below 1e-9 in alpha
    assert abs(alpha - 1.5) < 1e-8, alpha


def test_rebin_empty_contributions_keep_grid():
    d = 2
    B = _random_grid(d, 9)
    C = np.zeros((d, ND))
    C[1] = 1.0
    C[1, 10] = 50.0
    Bn = oracle.rebin(B, C)
    assert np.array_equal(Bn[0], B[0])
    assert not np.array_equal(Bn[1], B[1])


# ----------------------------------------------------------------------------- combination
def test_combination_is_inverse_variance_weighting():
    d, n = 2, 5000
    par = W.genz_params(W.GAUSSIAN, d)
    est, sig, chi2, iI, iV = oracle.integrate(W.GAUSSIAN, d, par, n, itmax=6, iter_adjust=3, seed=8)
    w = 1.0 / iV
    assert math.isclose(est, np.average(iI, weights=w), rel_tol=1e-13)
    assert math.isclose(sig, math.sqrt(1.0 / w.sum()), rel_tol=1e-13)
    assert math.isclose(chi2, float(np.sum(w * (iI - est) ** 2)) / 5, rel_tol=1e-10)


def test_combination_single_iteration_and_zero_variance():
    d = 2
    est, sig, chi2, iI, iV = oracle.integrate(W.GAUSSIAN, d, W.genz_params(W.GAUSSIAN, d), 400,
                                              itmax=1, iter_adjust=0, seed=1)
    assert est == iI[0] and chi2 == 0.0 and math.isclose(sig, math.sqrt(iV[0]))
    # f = 0 everywhere: every per-iteration variance is exactly zero
    est, sig, chi2, iI, iV = oracle.integrate(W.CONSTANT, d, np.zeros(2 * d), 400, itmax=3,
                                              iter_adjust=1, seed=1)
    assert est == 0.0 and sig == 0.0 and chi2 == 0.0
