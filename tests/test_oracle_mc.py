"""Statistical and exact pins of the oracle's whole m-Cubes run: closed-form integrals of the
Genz families (paper Sec. 5, Eq. 1-6), brute-force Gauss-Legendre quadrature at d <= 2,
exactness on constant integrands, the addition integrand (Sec. 5.3), z-score and chi^2
calibration over seeds."""
import math

import numpy as np
import pytest

import oracle
from closed_forms import exact
from paper_2302_05730_gb300 import workloads as W

FAMILIES = [W.OSCILLATORY, W.PRODUCT_PEAK, W.CORNER_PEAK, W.GAUSSIAN, W.C0, W.DISCONTINUOUS]


def _gauss_legendre_2d(f, d, panels=200, order=10):
    """Composite tensor Gauss-Legendre on [0,1]^d (d = 1 or 2), numpy's leggauss nodes."""
    z, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0.0, 1.0, panels + 1)
    h = np.diff(edges)[:, None]
    x1 = (edges[:-1, None] + h * (z[None, :] + 1) / 2).ravel()
    w1 = (h * w[None, :] / 2).ravel()
    if d == 1:
        return float(np.dot(w1, f(x1[:, None])))
    X, Y = np.meshgrid(x1, x1, indexing="ij")
    WW = np.outer(w1, w1).ravel()
    return float(np.dot(WW, f(np.stack([X.ravel(), Y.ravel()], axis=1))))


@pytest.mark.parametrize("fid", FAMILIES + [W.ADDITION])
@pytest.mark.parametrize("d", [1, 2])
def test_integrand_matches_closed_form_by_quadrature(fid, d):
    """Brute force: tensor Gauss-Legendre of the oracle's integrand equals the closed form.
    The discontinuous family has a jump and C0 a kink at x = u, so for them u is put on a panel
    edge (Gauss-Legendre then converges spectrally on every panel)."""
    par = W.genz_params(fid, d, seed=5) if fid != W.ADDITION else W.paper_params(fid, d)
    if fid in (W.DISCONTINUOUS, W.C0):
        par[d:] = np.round(par[d:] * 200) / 200
    f = lambda X: oracle.integrand(fid, d, par, X)
    q = _gauss_legendre_2d(f, d, panels=200 if d == 2 else 2000)
    ref = exact(fid, par[:d], par[d:])
    scale = 1.0 if fid == W.OSCILLATORY else abs(ref)
    assert abs(q - ref) <= 1e-11 * scale, (q, ref)


@pytest.mark.parametrize("fid", FAMILIES)
def test_paper_integrands_at_known_points(fid):
    """Values of the paper's f1..f6 at points where they reduce to elementary numbers."""
    d = 8
    par = W.paper_params(fid, d)
    half = np.full((1, d), 0.5)
    zero = np.zeros((1, d))
    v = oracle.integrand(fid, d, par, np.vstack([half, zero]))
    if fid == W.OSCILLATORY:
        assert math.isclose(v[0], math.cos(0.5 * 36), rel_tol=1e-14) and v[1] == 1.0
    elif fid == W.PRODUCT_PEAK:
        assert math.isclose(v[0], 2500.0 ** 8, rel_tol=1e-14)
        assert math.isclose(v[1], (1 / (1 / 2500 + 0.25)) ** 8, rel_tol=1e-14)
    elif fid == W.CORNER_PEAK:
        assert math.isclose(v[0], (1 + 18.0) ** -9, rel_tol=1e-14) and v[1] == 1.0
    elif fid == W.GAUSSIAN:
        assert v[0] == 1.0 and math.isclose(v[1], math.exp(-625 * 8 * 0.25), rel_tol=1e-13)
    elif fid == W.C0:
        assert v[0] == 1.0 and math.isclose(v[1], math.exp(-40.0), rel_tol=1e-14)
    elif fid == W.DISCONTINUOUS:
        assert v[0] == 0.0 and v[1] == 1.0   # x_1 = 1/2 >= 4/10 is cut away
        x = np.full((1, d), 0.3)
        assert math.isclose(oracle.integrand(fid, d, par, x)[0], math.exp(0.3 * sum(range(5, 13))), rel_tol=1e-14)


CASES = [
    (W.OSCILLATORY, 3, 2 * 10 ** 5), (W.PRODUCT_PEAK, 3, 2 * 10 ** 5), (W.CORNER_PEAK, 4, 2 * 10 ** 5),
    (W.GAUSSIAN, 3, 2 * 10 ** 5), (W.C0, 4, 2 * 10 ** 5), (W.DISCONTINUOUS, 3, 2 * 10 ** 5),
    (W.GAUSSIAN, 5, 10 ** 5), (W.PRODUCT_PEAK, 5, 10 ** 5),
]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid,d,n", CASES)
def test_estimate_within_error_of_closed_form(fid, d, n, mode):
    par = W.genz_params(fid, d, seed=2)
    est, sig, chi2, iI, iV = oracle.integrate(fid, d, par, n, itmax=6, iter_adjust=3, seed=11, mode=mode)
    ref = exact(fid, par[:d], par[d:])
    assert abs(est - ref) < 5 * sig, (est, ref, sig)
    assert sig < 0.05 * abs(ref) or fid == W.OSCILLATORY


@pytest.mark.parametrize("d", [1, 2])
def test_mc_matches_brute_force_quadrature_low_dim(d):
    """d <= 2: the m-Cubes estimate agrees with composite Gauss-Legendre within 4 sigma for every
    family (quadrature of the oracle integrand, independent of the sampler). At d = 1 the jump
    of the discontinuous family sits in a single sub-cube whose two samples cannot estimate its
    variance (both often land on one side), so that case is bounded by that cube's weight, I/m."""
    for fid in FAMILIES:
        par = W.genz_params(fid, d, seed=9)
        if fid in (W.DISCONTINUOUS, W.C0):
            par[d:] = np.round(par[d:] * 200) / 200
        q = _gauss_legendre_2d(lambda X: oracle.integrand(fid, d, par, X), d, panels=200)
        n = 4 * 10 ** 4
        est, sig, *_ = oracle.integrate(fid, d, par, n, itmax=5, iter_adjust=3, seed=21)
        m = oracle.stratify(d, n)[1]
        slack = abs(q) / m if (fid == W.DISCONTINUOUS and d == 1) else 0.0
        assert abs(est - q) < 4.5 * sig + slack, (fid, est, q, sig)


@pytest.mark.parametrize("mode", [0, 1])
def test_constant_integrand_is_exact(mode):
    """f = c on the uniform grid: every sample weight is c up to the rounding of J, so the
    estimate is c and the variance is zero up to rounding. The per-cube variance comes from
    S2 - S1^2/p (Algorithm 2 accumulates squares), whose rounding floor is a few eps * c^2 per
    cube: Var <= 8 eps c^2 / ((p - 1) m)."""
    c = 3.25
    eps = np.finfo(np.float64).eps
    for d in [1, 3, 7]:
        n = 3000
        g, m, p = oracle.stratify(d, n)
        est, sig, chi2, iI, iV = oracle.integrate(W.CONSTANT, d, W.constant_params(d, c), n,
                                                  itmax=3, iter_adjust=0, seed=2, mode=mode)
        assert np.all(np.abs(iI - c) <= 1e-13 * c)
        assert np.all(iV <= 8 * eps * c * c / ((p - 1) * m))
        assert abs(est - c) <= 1e-13 * c


def test_constant_integrand_on_adapted_grid_stays_unbiased():
    """Any grid integrates to one (the map's Jacobian has unit mean): a constant integrand on a
    grid adapted to a Gaussian still estimates c within its error."""
    d, c = 3, 2.0
    B = oracle.adapted_grid(W.GAUSSIAN, d, W.genz_params(W.GAUSSIAN, d), 2 * 10 ** 4, 3, seed=1)
    est, sig, *_ = oracle.integrate(W.CONSTANT, d, W.constant_params(d, c), 10 ** 5, itmax=2,
                                    iter_adjust=0, seed=5, B=B)
    assert abs(est - c) < 5 * sig and sig > 0


@pytest.mark.parametrize("d", [5, 6, 7, 8])
def test_addition_integrand(d):
    est, sig, *_ = oracle.integrate(W.ADDITION, d, W.paper_params(W.ADDITION, d), 10 ** 5,
                                    itmax=4, iter_adjust=2, seed=d)
    assert abs(est - d / 2) < 5 * sig and sig < 1e-3


def test_z_scores_and_chi2_are_calibrated():
    """Over 40 seeds: z = (estimate - exact)/sigma has mean ~ 0 and spread ~ 1; frozen-grid
    chi^2/dof averages ~ 1 (the error estimate of the method is honest)."""
    d = 2
    par = W.genz_params(W.GAUSSIAN, d, seed=3)
    ref = exact(W.GAUSSIAN, par[:d], par[d:])
    zs, chis = [], []
    for s in range(40):
        est, sig, chi2, *_ = oracle.integrate(W.GAUSSIAN, d, par, 2000, itmax=5, iter_adjust=0, seed=100 + s)
        zs.append((est - ref) / sig)
        chis.append(chi2)
    zs = np.array(zs)
    assert abs(zs.mean()) < 0.6 and 0.6 < zs.std() < 1.5
    assert 0.6 < np.mean(chis) < 1.5


def test_variance_drops_after_adjustment():
    """VEGAS importance sampling: after grid-adjusting iterations the per-iteration variance of
    a separable peak falls by orders of magnitude relative to the uniform grid."""
    d = 3
    par = W.gaussian_params(d, 10.0)
    est, sig, chi2, iI, iV = oracle.integrate(W.GAUSSIAN, d, par, 10 ** 5, itmax=4, iter_adjust=4, seed=0)
    assert iV[2] < iV[0] / 30


def test_config1_gaussian_reference_value():
    """d = 3 Gaussian a_i = 10, u_i = 1/2: closed form, and the oracle's 10-iteration run."""
    d = 3
    par = W.gaussian_params(d, 10.0)
    ref = exact(W.GAUSSIAN, par[:d], par[d:])
    assert math.isclose(ref, (math.sqrt(math.pi) / 10 * math.erf(5.0)) ** 3, rel_tol=1e-15)
    est, sig, chi2, *_ = oracle.integrate(W.GAUSSIAN, d, par, 10 ** 6, itmax=10, iter_adjust=5, seed=0)
    assert abs(est - ref) < 4 * sig and sig / ref < 1e-4


def test_double_gaussian_closed_form_and_mc():
    """Two mirrored Gaussian peaks: Gauss-Legendre of the oracle integrand at d = 2 equals the sum
    of two Gaussian closed forms; the oracle's m-Cubes run at d = 4 finds it within error."""
    d = 2
    par = W.double_gaussian_params(d, a=6.0, u=0.3)
    q = _gauss_legendre_2d(lambda X: oracle.integrand(W.DOUBLE_GAUSSIAN, d, par, X), d, panels=200)
    ref = exact(W.DOUBLE_GAUSSIAN, par[:d], par[d:])
    assert abs(q - ref) <= 1e-11 * ref
    d = 4
    par = W.double_gaussian_params(d, a=6.0, u=0.3)
    est, sig, *_ = oracle.integrate(W.DOUBLE_GAUSSIAN, d, par, 2 * 10 ** 5, itmax=6, iter_adjust=3, seed=3)
    assert abs(est - exact(W.DOUBLE_GAUSSIAN, par[:d], par[d:])) < 5 * sig


@pytest.mark.parametrize("d", [2, 3])
def test_rotated_gaussian_against_multivariate_normal_box_probability(d):
    """exp(-(x-c)^T M (x-c)) over the unit cube: scipy's multivariate normal CDF (box probability
    by inclusion-exclusion) against quadrature of the oracle integrand (d = 2) and the oracle's
    m-Cubes run (d = 3)."""
    from closed_forms import rotated_gaussian_exact
    par = W.rotated_gaussian_params(d, seed=1, lam_min=1.0, lam_max=60.0)
    M = par[:d * d].reshape(d, d)
    c = par[d * d:]
    ref = rotated_gaussian_exact(M, c)
    if d == 2:
        q = _gauss_legendre_2d(lambda X: oracle.integrand(W.ROTATED_GAUSSIAN, d, par, X), d, panels=100)
        assert abs(q - ref) <= 1e-9 * ref
    est, sig, *_ = oracle.integrate(W.ROTATED_GAUSSIAN, d, par, 2 * 10 ** 5, itmax=6, iter_adjust=3, seed=5)
    assert abs(est - ref) < 5 * sig and sig < 1e-2 * ref
