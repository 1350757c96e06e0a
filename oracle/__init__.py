"""m-Cubes CPU oracle -- test infrastructure only.

A plain FP64 C restatement of one m-Cubes iteration (paper Sec. 3.2, Algorithm 2), the VEGAS
grid refinement it relies on (Lepage 1978), the benchmark integrands (Sec. 5, Eq. 1-6 and the
addition integrand), Philox4x32-10 (Salmon et al., SC'11), and the PAGANI region evaluation
(Sec. 3.1) with the Genz-Malik degree-7/5 rule and a simple adaptive driver, wrapped with ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package. The CUDA library never loads it and shares
no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

ND = 500
DMAX = 16

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, ADDITION, CONSTANT = range(8)
DOUBLE_GAUSSIAN, ROTATED_GAUSSIAN = 8, 9

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcubes_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "pagani_oracle.c")]
_LIB = os.path.join(_HERE, "libmcubes_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_philox4x32_10.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
            L.orc_stratify.argtypes = [i32, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
            L.orc_integrand.argtypes = [i32, i32, dp, dp, i32]
            L.orc_integrand.restype = ctypes.c_double
            L.orc_integrand_many.argtypes = [i32, i32, dp, i64, dp, dp]
            L.orc_vsample.argtypes = [i32, i32, dp, i64, u64, i32, u32, i32, i32, dp, i64, i64,
                                      dp, dp, dp, dp, dp, dp]
            L.orc_rebin.argtypes = [i32, dp, dp, ctypes.c_double, dp]
            L.orc_damp.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_damp.restype = ctypes.c_double
            L.orc_uniform_grid.argtypes = [i32, dp]
            L.orc_integrate.argtypes = [i32, i32, dp, i64, i32, i32, u64, u32, i32, dp, dp, dp, dp]
            L.orc_adapted_grid.argtypes = [i32, i32, dp, i64, i32, u64, u32, i32, dp]
            L.orc_sample_points.argtypes = [i32, i32, dp, i64, u64, i32, u32, i32, dp, i64, i64,
                                            dp, dp, ctypes.POINTER(ctypes.c_int32), dp, dp]
            L.orc_gm_count.argtypes = [i32]
            L.orc_gm_count.restype = i32
            L.orc_gm_weights.argtypes = [i32, dp, dp]
            L.orc_gm_rules.argtypes = [i32, dp]
            L.orc_pagani_rules.argtypes = [i32, i32, dp, dp, dp, dp]
            L.orc_pagani_rules.restype = i32
            L.orc_pagani_error.argtypes = [dp]
            L.orc_pagani_error.restype = ctypes.c_double
            L.orc_gm_points.argtypes = [i32, dp, ctypes.POINTER(ctypes.c_int32)]
            L.orc_gm_points.restype = i32
            L.orc_pagani_evaluate.argtypes = [i32, i32, dp, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_int32), dp]
            L.orc_pagani_evaluate.restype = i32
            L.orc_pagani_integrate.argtypes = [i32, i32, dp, ctypes.c_double, i32, i64, i32, dp]
            L.orc_pagani_integrate.restype = i32
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def stratify(d: int, n: int):
    g, m, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().orc_stratify(d, n, ctypes.byref(g), ctypes.byref(m), ctypes.byref(p)), "stratify")
    return g.value, m.value, p.value


def uniform_grid(d: int) -> np.ndarray:
    B = np.empty((d, ND + 1))
    lib().orc_uniform_grid(d, _dp(B))
    return B


def integrand(fid: int, d: int, params, X) -> np.ndarray:
    """f at the rows of X (npts x d), FP64."""
    X = _f64(np.atleast_2d(X))
    par = _f64(params)
    out = np.empty(X.shape[0])
    lib().orc_integrand_many(fid, d, _dp(par), X.shape[0], _dp(X), _dp(out))
    return out


def vsample(fid, d, params, n, seed, it=0, job=0, mode=0, adjust=1, B=None, t0=0, t1=None,
            per_cube=False):
    """One V-Sample pass over sub-cubes [t0, t1).

    Returns dict with sumI, sumV (compensated pairs), C (d x ND, if adjust), and per-cube
    I_t, V_t arrays when per_cube is set. I = sumI / m, Var = sumV / m^2 over the full range.
    """
    g, m, p = stratify(d, n)
    if t1 is None:
        t1 = m
    par = _f64(params)
    B = uniform_grid(d) if B is None else _f64(B)
    sI = np.zeros(2)
    sV = np.zeros(2)
    C = np.zeros((d, ND)) if adjust else None
    Cc = np.zeros((d, ND)) if adjust else None
    cI = np.empty(t1 - t0) if per_cube else None
    cV = np.empty(t1 - t0) if per_cube else None
    st = lib().orc_vsample(fid, d, _dp(par), n, seed, it, job, mode, int(adjust), _dp(B), t0, t1,
                           _dp(sI), _dp(sV), _dp(C), _dp(Cc), _dp(cI), _dp(cV))
    _check(st, "vsample")
    out = dict(g=g, m=m, p=p, sumI=sI, sumV=sV, cubeI=cI, cubeV=cV)
    if adjust:
        out["C"] = C + Cc
    if t0 == 0 and t1 == m:
        out["I"] = float(sI[0] + sI[1]) / m
        out["Var"] = float(sV[0] + sV[1]) / (float(m) * float(m))
    return out


def sample_points(fid, d, params, n, seed, it=0, job=0, mode=0, B=None, t0=0, t1=1):
    g, m, p = stratify(d, n)
    par = _f64(params)
    B = uniform_grid(d) if B is None else _f64(B)
    rows = (t1 - t0) * p
    u = np.empty((rows, d)); x = np.empty((rows, d))
    k = np.empty((rows, d), dtype=np.int32)
    J = np.empty(rows); w = np.empty(rows)
    st = lib().orc_sample_points(fid, d, _dp(par), n, seed, it, job, mode, _dp(B), t0, t1,
                                 _dp(u), _dp(x), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 _dp(J), _dp(w))
    _check(st, "sample_points")
    return dict(g=g, m=m, p=p, u=u, x=x, k=k, J=J, w=w)


def rebin(B, C, alpha: float = 1.5) -> np.ndarray:
    B = _f64(B)
    C = _f64(C)
    d = B.shape[0]
    out = np.empty_like(B)
    lib().orc_rebin(d, _dp(B), _dp(C), alpha, _dp(out))
    return out


def damp(rho: float, alpha: float = 1.5) -> float:
    """Rebin's damped weight of a bin holding the fraction rho of the smoothed contributions."""
    return float(lib().orc_damp(float(rho), float(alpha)))


def integrate(fid, d, params, n, itmax, iter_adjust, seed, job=0, mode=0, B=None):
    """Full m-Cubes run; returns (estimate, sigma, chi2/dof, per-iteration I, per-iteration Var)."""
    par = _f64(params)
    est = np.zeros(3)
    iI = np.zeros(itmax)
    iV = np.zeros(itmax)
    Bp = None if B is None else _f64(B)
    st = lib().orc_integrate(fid, d, _dp(par), n, itmax, iter_adjust, seed, job, mode, _dp(Bp),
                             _dp(est), _dp(iI), _dp(iV))
    _check(st, "integrate")
    return float(est[0]), float(est[1]), float(est[2]), iI, iV


def adapted_grid(fid, d, params, n, iters, seed, job=0, mode=0) -> np.ndarray:
    """Grid after `iters` adjusting iterations from the uniform grid."""
    par = _f64(params)
    B = np.empty((d, ND + 1))
    _check(lib().orc_adapted_grid(fid, d, _dp(par), n, iters, seed, job, mode, _dp(B)), "adapted_grid")
    return B


# ------------------------------------------------------------------------------ PAGANI
def gm_rule(d: int):
    """The Genz-Malik degree-7/5 rule on [-1, 1]^d: points (n x d), class of each point (1..5),
    weights per class for degree 7 and degree 5."""
    L = lib()
    n = L.orc_gm_count(d)
    if n <= 0:
        raise ValueError(f"unsupported d = {d}")
    U = np.empty((n, d))
    cls = np.empty(n, dtype=np.int32)
    _check(L.orc_gm_points(d, _dp(U), cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "gm_points")
    w7 = np.empty(5)
    w5 = np.empty(5)
    L.orc_gm_weights(d, _dp(w7), _dp(w5))
    return U, cls, w7, w5


def gm_rules(d: int) -> np.ndarray:
    """Class weights (5 rules x 5 classes) of R7, R5, R3a, R3b, R1 on [-1, 1]^d."""
    W = np.empty((5, 5))
    lib().orc_gm_rules(d, _dp(W))
    return W


def pagani_rules(fid, d, params, lo, ln) -> np.ndarray:
    """The five rule values (R7, R5, R3a, R3b, R1) of one region."""
    out = np.empty(5)
    _check(lib().orc_pagani_rules(fid, d, _dp(_f64(params)), _dp(_f64(lo)), _dp(_f64(ln)), _dp(out)), "pagani_rules")
    return out


def pagani_error(rules) -> float:
    """The region error estimate from the five rule values (R7, R5, R3a, R3b, R1)."""
    R = np.ascontiguousarray(rules, dtype=np.float64)
    return float(lib().orc_pagani_error(_dp(R)))


def pagani_evaluate(fid, d, params, lo, length, want_fourth=False):
    """One region: (I, E, split axis[, fourth differences])."""
    par = _f64(params)
    lo = _f64(lo)
    length = _f64(length)
    I = ctypes.c_double()
    E = ctypes.c_double()
    ax = ctypes.c_int32()
    fourth = np.empty(d) if want_fourth else None
    _check(lib().orc_pagani_evaluate(fid, d, _dp(par), _dp(lo), _dp(length), ctypes.byref(I), ctypes.byref(E),
                                     ctypes.byref(ax), _dp(fourth)), "pagani_evaluate")
    if want_fourth:
        return I.value, E.value, ax.value, fourth
    return I.value, E.value, ax.value


def pagani_integrate(fid, d, params, rel_tol, max_iters=40, max_regions=1 << 20, init_split=2):
    """Adaptive run; dict(estimate, error, evaluated, iterations, status, active)."""
    par = _f64(params)
    out = np.zeros(6)
    _check(lib().orc_pagani_integrate(fid, d, _dp(par), float(rel_tol), int(max_iters), int(max_regions),
                                      int(init_split), _dp(out)), "pagani_integrate")
    return dict(estimate=out[0], error=out[1], evaluated=int(out[2]), iterations=int(out[3]), status=int(out[4]),
                active=int(out[5]))
