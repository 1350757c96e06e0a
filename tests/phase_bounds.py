"""Rounding bound on the oscillatory family's FP64 bin contributions.

The family is cos(phi) with phi = 2 pi u_1 + sum a_i x_i (paper Eq. 1). Any FP64 evaluation of phi
-- the oracle's left-to-right sum in radians, a kernel's sum in turns over folded table entries --
carries an absolute error of a few eps times the size of its terms, and two valid evaluations
differ by that much. A sample's contribution w^2 = (J cos phi)^2 then moves by at most
2 |w| |J| |delta phi|, which is large relative to w^2 near the zeros of cos. Where one sample
dominates a bin (very uneven grids give Jacobians over many orders of magnitude) and sits near a
zero, that is above 1e-12 of the bin's C; this module sums the bound over each bin's samples so
that a per-bin tolerance can include it.
"""
import numpy as np

import oracle

EPS = np.finfo(np.float64).eps
ND = 500


def oscillatory_c_bound(d, par, n, seed, it, job, B, chunk=1 << 16):
    """Per bin (d x ND): the sum over the bin's samples of 2 |w| |J| delta_phi, with
    delta_phi = 2 (d + 4) eps (2 pi |u_1| + sum_i |a_i| (x_i + 3 Delta_i)) (Delta_i the sample's bin
    width on axis i: the folded table entries' share)."""
    from concurrent.futures import ThreadPoolExecutor
    g, m, p = oracle.stratify(d, n)
    a, u = np.abs(np.asarray(par[:d], dtype=np.float64)), np.asarray(par[d:], dtype=np.float64)
    widths = np.diff(np.asarray(B, dtype=np.float64), axis=1)

    def one(t0):
        sp = oracle.sample_points(0, d, par, n, seed, it=it, job=job, mode=0, B=B, t0=t0, t1=min(m, t0 + chunk))
        x, k, J, w = sp["x"], sp["k"], sp["J"], sp["w"]
        dk = widths[np.arange(d)[None, :], k]
        dphi = 2 * (d + 4) * EPS * (2 * np.pi * abs(u[0]) + np.abs(x) @ a + 3 * dk @ a)
        b = 2 * np.abs(w) * np.abs(J) * dphi
        return np.stack([np.bincount(k[:, i], weights=b, minlength=ND) for i in range(d)])

    with ThreadPoolExecutor(max_workers=8) as ex:
        parts = list(ex.map(one, range(0, m, chunk)))
    return np.sum(parts, axis=0)
