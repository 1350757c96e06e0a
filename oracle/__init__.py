"""m-Cubes CPU oracle -- test infrastructure only.

A plain FP64 C restatement of one m-Cubes iteration (paper Sec. 3.2, Algorithm 2), the VEGAS
grid refinement it relies on (Lepage 1978), the benchmark integrands (Sec. 5, Eq. 1-6 and the
addition integrand) and Philox4x32-10 (Salmon et al., SC'11), wrapped with ctypes.

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
_LIB = os.path.join(_HERE, "libmcubes_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
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
            L.orc_uniform_grid.argtypes = [i32, dp]
            L.orc_integrate.argtypes = [i32, i32, dp, i64, i32, i32, u64, u32, i32, dp, dp, dp, dp]
            L.orc_adapted_grid.argtypes = [i32, i32, dp, i64, i32, u64, u32, i32, dp]
            L.orc_sample_points.argtypes = [i32, i32, dp, i64, u64, i32, u32, i32, dp, i64, i64,
                                            dp, dp, ctypes.POINTER(ctypes.c_int32), dp, dp]
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
