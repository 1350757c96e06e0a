"""Pins of the coupling-flow oracle (oracle/flow.py) against things other than itself: numerical
derivatives and Jacobian determinants, quadrature of the density, torch's bfloat16 conversion,
invertibility, and the identity at zero output weights."""
import numpy as np
import pytest

from oracle import flow as F


def _raw(rng, n, K, scale=1.5):
    return rng.normal(0.0, scale, (n, 2 * K + 1))


def _params(rng, d, L, H, K, scale=0.3):
    p = rng.normal(0.0, scale, F.n_params(d, L, H, K))
    return p


@pytest.mark.parametrize("K", [1, 4, 16])
def test_piecewise_quadratic_cdf_is_a_cdf(K):
    rng = np.random.default_rng(K)
    raw = _raw(rng, 1, K)
    xs = np.linspace(0.0, 1.0, 20001)
    y, q = F.pq_cdf(xs, np.repeat(raw, xs.size, axis=0), K)
    assert abs(y[0]) < 1e-14 and abs(y[-1] - 1.0) < 1e-12
    assert np.all(np.diff(y) >= -1e-15)
    assert np.all(q > 0)
    # pdf integrates to 1 (trapezoid; exact for piecewise-linear pdf up to kinks between nodes)
    assert abs(np.trapezoid(q, xs) - 1.0) < 1e-6
    # pdf is the derivative of the CDF (central differences, away from bin edges)
    h = 1e-7
    xm = rng.uniform(0.01, 0.99, 200)
    yp, _ = F.pq_cdf(xm + h, np.repeat(raw, 200, axis=0), K)
    ym, _ = F.pq_cdf(xm - h, np.repeat(raw, 200, axis=0), K)
    _, qm = F.pq_cdf(xm, np.repeat(raw, 200, axis=0), K)
    assert np.allclose((yp - ym) / (2 * h), qm, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("K", [2, 16])
def test_piecewise_quadratic_inverse(K):
    rng = np.random.default_rng(10 + K)
    raw = _raw(rng, 500, K, 2.0)
    x = rng.uniform(0, 1, 500)
    y, q = F.pq_cdf(x, raw, K)
    x2, q2 = F.pq_inverse(y, raw, K)
    assert np.allclose(x2, x, rtol=0, atol=1e-12)
    assert np.allclose(q2, q, rtol=1e-10)


def test_masks_transform_every_axis():
    for d in range(2, 17):
        for L in (2, 4, 6):
            seen = set()
            for A, B in F.masks(d, L):
                assert len(A) + len(B) == d and set(A).isdisjoint(B) and len(B) > 0 and len(A) > 0
                seen |= set(B.tolist())
            assert seen == set(range(d))


def test_identity_at_zero_output_layer():
    d, L, H, K = 5, 4, 16, 8
    rng = np.random.default_rng(1)
    p = _params(rng, d, L, H, K)
    for lay in F.unpack(p, d, L, H, K):     # views into p
        lay["W3"][...] = 0.0
        lay["b3"][...] = 0.0
    x = rng.uniform(0, 1, (100, d))
    z, logq = F.forward(p, x, d, L, H, K)
    assert np.allclose(z, x, atol=1e-14) and np.allclose(logq, 0.0, atol=1e-13)


@pytest.mark.parametrize("d,L", [(2, 2), (4, 4), (8, 4), (7, 3)])
def test_flow_inverse_and_log_det(d, L):
    H, K = 12, 6
    rng = np.random.default_rng(d * 10 + L)
    p = _params(rng, d, L, H, K)
    x = rng.uniform(0.02, 0.98, (40, d))
    z, logq = F.forward(p, x, d, L, H, K)
    x2, logq2 = F.inverse(p, z, d, L, H, K)
    assert np.allclose(x2, x, atol=1e-10)
    assert np.allclose(logq2, logq, atol=1e-9)
    # log q is log |det dz/dx| (finite-difference Jacobian, numpy determinant)
    Jm = F.grad_x_fd(p, x, d, L, H, K)
    det = np.linalg.det(Jm)
    assert np.all(det > 0)
    assert np.allclose(np.log(det), logq, atol=1e-5)
    # z lies in the unit cube
    assert z.min() >= 0.0 and z.max() <= 1.0


def test_flow_density_integrates_to_one():
    d, L, H, K = 2, 4, 16, 8
    rng = np.random.default_rng(3)
    p = _params(rng, d, L, H, K, 0.5)
    n = 600
    g = (np.arange(n) + 0.5) / n
    X = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    _, logq = F.forward(p, X, d, L, H, K)
    assert abs(np.mean(np.exp(logq)) - 1.0) < 2e-3   # midpoint rule on a 600^2 grid


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 10, 10000), rng.normal(0, 1e-30, 100), [0.0, -0.0, 1.0, 65504.0]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.bf16(v), ref)


def test_finite_difference_gradient_is_consistent_and_descends():
    d, L, H, K = 4, 2, 8, 4
    rng = np.random.default_rng(5)
    p = _params(rng, d, L, H, K, 0.4)
    x = rng.uniform(0, 1, (64, d))
    w = np.exp(-20 * np.sum((x - 0.3) ** 2, axis=1)) ** 2
    for kind in ("variance", "kl"):
        g1 = F.grad_fd(p, x, w, d, L, H, K, kind, eps=1e-5)
        g2 = F.grad_fd(p, x, w, d, L, H, K, kind, eps=2e-6)
        assert np.allclose(g1, g2, rtol=1e-5, atol=1e-8 * np.abs(g1).max())
        l0 = F.loss(p, x, w, d, L, H, K, kind)
        l1 = F.loss(p - 1e-3 * g1 / np.abs(g1).max(), x, w, d, L, H, K, kind)
        assert l1 < l0
