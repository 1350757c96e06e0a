"""Closed-form integrals over [0,1]^d of the Genz families used by the benchmark integrands
(paper Sec. 5, Eq. 1-6) -- independent of the oracle; used to pin it.

Each family integrates in closed form because it is a product of one-dimensional factors, or
(oscillatory, corner peak) a function of a linear form whose d-fold integral has a known
expression:
  oscillatory    Re[ e^{i 2 pi u_1} prod_i (e^{i a_i} - 1) / (i a_i) ]
  product peak   prod_i a_i (atan(a_i (1 - u_i)) + atan(a_i u_i))
  corner peak    1/(d! prod a_i) * sum_{S subset [d]} (-1)^{|S|} / (1 + sum_{i in S} a_i)
  Gaussian       prod_i sqrt(pi)/(2 a_i) (erf(a_i (1 - u_i)) + erf(a_i u_i))
  C0             prod_i (2 - e^{-a_i u_i} - e^{-a_i (1 - u_i)}) / a_i
  discontinuous  prod_i (e^{a_i min(u_i,1)} - 1) / a_i     (cut on every axis)
  addition       d / 2
  constant       c
"""
from fractions import Fraction
from itertools import combinations
from math import atan, erf, exp, factorial, pi, sqrt
import cmath

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, ADDITION, CONSTANT = range(8)
DOUBLE_GAUSSIAN, ROTATED_GAUSSIAN = 8, 9


def _corner_exact(a):
    d = len(a)
    fa = [Fraction(v) for v in a]
    total = Fraction(0)
    for r in range(d + 1):
        for S in combinations(range(d), r):
            total += Fraction((-1) ** r) / (1 + sum((fa[i] for i in S), Fraction(0)))
    den = Fraction(factorial(d))
    for v in fa:
        den *= v
    return total / den


def exact(fid, a, u):
    a = [float(v) for v in a]
    u = [float(v) for v in u]
    d = len(a)
    if fid == OSCILLATORY:
        z = cmath.exp(2j * pi * u[0])
        for ai in a:
            z *= (cmath.exp(1j * ai) - 1.0) / (1j * ai)
        return z.real
    if fid == PRODUCT_PEAK:
        v = 1.0
        for ai, ui in zip(a, u):
            v *= ai * (atan(ai * (1.0 - ui)) + atan(ai * ui))
        return v
    if fid == CORNER_PEAK:
        return float(_corner_exact(a))
    if fid == GAUSSIAN:
        v = 1.0
        for ai, ui in zip(a, u):
            v *= sqrt(pi) / (2.0 * ai) * (erf(ai * (1.0 - ui)) + erf(ai * ui))
        return v
    if fid == C0:
        v = 1.0
        for ai, ui in zip(a, u):
            v *= (2.0 - exp(-ai * ui) - exp(-ai * (1.0 - ui))) / ai
        return v
    if fid == DISCONTINUOUS:
        v = 1.0
        for ai, ui in zip(a, u):
            v *= (exp(ai * min(ui, 1.0)) - 1.0) / ai
        return v
    if fid == ADDITION:
        return d / 2.0
    if fid == CONSTANT:
        return a[0]
    if fid == DOUBLE_GAUSSIAN:   # two Gaussians, centres u and 1 - u
        return exact(GAUSSIAN, a, u) + exact(GAUSSIAN, a, [1.0 - v for v in u])
    raise ValueError(fid)


def rotated_gaussian_exact(M, c):
    """int_[0,1]^d exp(-(x-c)^T M (x-c)) dx = pi^{d/2} / sqrt(det M) * P(X in [0,1]^d) for
    X ~ N(c, (2M)^-1); the box probability from scipy's multivariate normal CDF by
    inclusion-exclusion over the 2^d corners."""
    import itertools
    import numpy as np
    from scipy.stats import multivariate_normal
    M = np.asarray(M, dtype=float)
    c = np.asarray(c, dtype=float)
    d = len(c)
    cov = np.linalg.inv(2.0 * M)
    mvn = multivariate_normal(mean=c, cov=cov, abseps=1e-12, releps=1e-10, maxpts=10 ** 7)
    prob = 0.0
    for corner in itertools.product([0, 1], repeat=d):
        sign = (-1) ** (d - sum(corner))
        prob += sign * mvn.cdf(np.array(corner, dtype=float))
    return float(np.pi ** (d / 2) / np.sqrt(np.linalg.det(M)) * prob)


def paper_params(fid, d):
    """Fixed parameters of the paper's benchmark integrands f1..f6 (Sec. 5, Eq. 1-6)."""
    idx = list(range(1, d + 1))
    if fid == OSCILLATORY:       # f1 = cos(sum i x_i)
        return [float(i) for i in idx], [0.0] * d
    if fid == PRODUCT_PEAK:      # f2 = prod (1/50^2 + (x_i - 1/2)^2)^-1
        return [50.0] * d, [0.5] * d
    if fid == CORNER_PEAK:       # f3 = (1 + sum i x_i)^(-d-1)
        return [float(i) for i in idx], [0.0] * d
    if fid == GAUSSIAN:          # f4 = exp(-625 sum (x_i - 1/2)^2)
        return [25.0] * d, [0.5] * d
    if fid == C0:                # f5 = exp(-10 sum |x_i - 1/2|)
        return [10.0] * d, [0.5] * d
    if fid == DISCONTINUOUS:     # f6 = exp(sum (i+4) x_i) if x_i < (3+i)/10
        return [float(i + 4) for i in idx], [(3 + i) / 10.0 for i in idx]
    if fid == ADDITION:
        return [0.0] * d, [0.0] * d
    raise ValueError(fid)
