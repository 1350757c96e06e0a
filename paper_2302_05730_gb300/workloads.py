"""Seeded synthetic inputs for the m-Cubes benchmark integrands.

This module only draws and names integrand parameters; it holds none of the method's
arithmetic. Both the CUDA path and the CPU oracle receive the arrays it returns, so tests and
the benchmark feed the two sides the same inputs.

The integrand families are the Genz families behind the paper's benchmark integrands
(Sec. 5, Eq. 1-6); parameters are a[0..d-1] followed by u[0..d-1]. The random parameter
recipe (a_i ~ U[5, 15], u_i ~ U[0.2, 0.8]) stands in for a seeded draw of Genz test
problems; the paper's own fixed-parameter f1..f6 are available as well.
"""
from __future__ import annotations

import numpy as np

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, ADDITION, CONSTANT = range(8)
DOUBLE_GAUSSIAN, ROTATED_GAUSSIAN = 8, 9

NAMES = {
    OSCILLATORY: "oscillatory",
    PRODUCT_PEAK: "product_peak",
    CORNER_PEAK: "corner_peak",
    GAUSSIAN: "gaussian",
    C0: "c0",
    DISCONTINUOUS: "discontinuous",
    ADDITION: "addition",
    CONSTANT: "constant",
    DOUBLE_GAUSSIAN: "double_gaussian",
    ROTATED_GAUSSIAN: "rotated_gaussian",
}
BY_NAME = {v: k for k, v in NAMES.items()}

# The six Genz families of the d = 5, 6, 8 benchmark at 1e8 samples per iteration.
GENZ6 = (OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS)


def genz_params(fid: int, d: int, seed: int = 0, a_range=(5.0, 15.0), u_range=(0.2, 0.8)):
    """Seeded Genz parameters: a_i ~ U[a_range], u_i ~ U[u_range] (one stream per family, d, seed)."""
    rng = np.random.default_rng([0xC0FFEE, int(seed), int(fid), int(d)])
    a = rng.uniform(a_range[0], a_range[1], size=d)
    u = rng.uniform(u_range[0], u_range[1], size=d)
    return np.concatenate([a, u])


def paper_params(fid: int, d: int):
    """Fixed parameters of the paper's f1..f6 (Sec. 5, Eq. 1-6) and the addition integrand."""
    i = np.arange(1, d + 1, dtype=np.float64)
    if fid == OSCILLATORY:       # f1 = cos(sum i x_i)
        a, u = i, np.zeros(d)
    elif fid == PRODUCT_PEAK:    # f2 = prod (1/50^2 + (x_i - 1/2)^2)^-1
        a, u = np.full(d, 50.0), np.full(d, 0.5)
    elif fid == CORNER_PEAK:     # f3 = (1 + sum i x_i)^(-d-1)
        a, u = i, np.zeros(d)
    elif fid == GAUSSIAN:        # f4 = exp(-625 sum (x_i - 1/2)^2)
        a, u = np.full(d, 25.0), np.full(d, 0.5)
    elif fid == C0:              # f5 = exp(-10 sum |x_i - 1/2|)
        a, u = np.full(d, 10.0), np.full(d, 0.5)
    elif fid == DISCONTINUOUS:   # f6 = exp(sum (i+4) x_i) if x_i < (3+i)/10 on every axis
        a, u = i + 4.0, (3.0 + i) / 10.0
    elif fid == ADDITION:
        a, u = np.zeros(d), np.zeros(d)
    else:
        raise ValueError(fid)
    return np.concatenate([a, u])


def gaussian_params(d: int, a: float, u: float = 0.5):
    """Isotropic Gaussian exp(-sum a^2 (x_i - u)^2)."""
    return np.concatenate([np.full(d, float(a)), np.full(d, float(u))])


def constant_params(d: int, c: float):
    p = np.zeros(2 * d)
    p[0] = c
    return p


def batch_jobs(n_jobs: int = 4096, seed: int = 0, dmin: int = 2, dmax: int = 8,
               nmin: float = 1e4, nmax: float = 1e7):
    """Independent Gaussian integrations of uneven size: d ~ U{dmin..dmax},
    a_i ~ U[5, 25], u_i ~ U[0.2, 0.8], samples per iteration log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng([0xBA7C4, int(seed)])
    jobs = []
    for j in range(n_jobs):
        d = int(rng.integers(dmin, dmax + 1))
        a = rng.uniform(5.0, 25.0, size=d)
        u = rng.uniform(0.2, 0.8, size=d)
        n = int(round(float(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))))
        jobs.append(dict(fid=GAUSSIAN, d=d, params=np.concatenate([a, u]), ncall=n))
    return jobs


def double_gaussian_params(d: int, a: float = 10.0, u: float = 0.25):
    """exp(-a^2 |x - u 1|^2) + exp(-a^2 |x - (1-u) 1|^2): centres u 1 and (1-u) 1."""
    return np.concatenate([np.full(d, float(a)), np.full(d, float(u))])


def rotated_gaussian_params(d: int, seed: int = 0, lam_min: float = 1.0, lam_max: float = 400.0, centre: float = 0.5):
    """exp(-(x - c)^T Q diag(lam) Q^T (x - c)) with Q from the QR factorisation of a seeded Gaussian
    matrix and lam = linspace(lam_min, lam_max, d). Parameters: M = Q diag(lam) Q^T (d x d,
    row-major), then c (d)."""
    rng = np.random.default_rng([0x507A7E, int(seed), int(d)])
    Q, R = np.linalg.qr(rng.normal(size=(d, d)))
    Q = Q * np.sign(np.diag(R))
    lam = np.linspace(lam_min, lam_max, d)
    M = (Q * lam) @ Q.T
    M = (M + M.T) / 2.0
    return np.concatenate([M.ravel(), np.full(d, float(centre))])
