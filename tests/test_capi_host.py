"""The C ABI without a GPU: the library loads, exports every function include/mcubes.h declares,
and its host-side logic (stratification, argument checks, status codes) behaves as documented.
None of these calls reaches a CUDA kernel."""
import ctypes
import importlib
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2302_05730_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2302_05730_gb300", "libmcubes.so")


@pytest.fixture(scope="module")
def capi():
    if not os.path.exists(LIB):
        from paper_2302_05730_gb300.build import build
        build()
    from paper_2302_05730_gb300 import capi as c
    return c


def test_library_exports_every_declared_function(capi):
    names = capi.header_functions()
    assert len(names) >= 12
    raw = ctypes.CDLL(LIB)
    for n in names:
        assert hasattr(raw, n), n


def test_stratify_matches_oracle(capi):
    rng = np.random.default_rng(0)
    for d in range(1, 17):
        for n in [2, 3, 100, 10 ** 4, 10 ** 6, 10 ** 8] + list(rng.integers(2, 10 ** 9, 5)):
            try:
                want = oracle.stratify(d, int(n))
            except ValueError:
                with pytest.raises(capi.McubesError):
                    capi.stratify(d, int(n))
                continue
            assert capi.stratify(d, int(n)) == want, (d, n)


def test_status_strings(capi):
    for s in range(9):
        assert capi.status_string(s)
    assert "unknown" in capi.status_string(99)


def _status(call):
    try:
        call()
    except Exception as e:  # noqa: BLE001
        return getattr(e, "status", None)
    return 0


def test_argument_checks_return_status_codes(capi):
    par = W.genz_params(W.GAUSSIAN, 3)
    assert _status(lambda: capi.integrate(W.GAUSSIAN, par, 0, 1000, 3, 1, 0)) == 2
    assert _status(lambda: capi.integrate(W.GAUSSIAN, np.ones(34), 17, 1000, 3, 1, 0)) == 2
    assert _status(lambda: capi.integrate(10, par, 3, 1000, 3, 1, 0)) == 3
    assert _status(lambda: capi.integrate(-1, par, 3, 1000, 3, 1, 0)) == 3
    assert _status(lambda: capi.integrate(W.GAUSSIAN, par, 3, 1, 3, 1, 0)) == 1       # ncall < 2
    assert _status(lambda: capi.integrate(W.GAUSSIAN, par, 3, 1000, 0, 0, 0)) == 1    # itmax < 1
    assert _status(lambda: capi.integrate(W.GAUSSIAN, par, 3, 1000, 3, 4, 0)) == 1    # iter_adjust > itmax
    assert _status(lambda: capi.integrate(W.GAUSSIAN, par, 3, 1000, 3, 1, 0, precision=2)) == 1
    bad = par.copy()
    bad[1] = np.nan
    assert _status(lambda: capi.integrate(W.GAUSSIAN, bad, 3, 1000, 3, 1, 0)) == 1
    # FP32-eval needs g <= 2^24
    assert _status(lambda: capi.vsample_once(W.GAUSSIAN, W.genz_params(W.GAUSSIAN, 1), 1, 2 ** 26, 0,
                                             precision=1)) == 1
    # grids must run 0 < ... < 1
    g = oracle.uniform_grid(3)
    g[1, 7] = g[1, 8]
    assert _status(lambda: capi.vsample_once(W.GAUSSIAN, par, 3, 1000, 0, grid_in=g)) == 1
    # device calls: workspace, aliasing and probe checks happen before any CUDA call
    assert _status(lambda: capi.iteration_dev(W.GAUSSIAN, par, 3, 1000, 0, 0, 0, 1, 0, 1 << 20, 2 << 20,
                                              3 << 20, None, 4 << 20, 16)) == 8
    assert _status(lambda: capi.iteration_dev(W.GAUSSIAN, par, 3, 1000, 0, 0, 0, 1, 0, 1 << 20, 2 << 20,
                                              3 << 20, None, (4 << 20) + 8, 1 << 20)) == 8
    assert _status(lambda: capi.iteration_dev(W.GAUSSIAN, par, 3, 1000, 0, 0, 0, 1, 0, 1 << 20, 1 << 20,
                                              3 << 20, None, 4 << 20, 1 << 20)) == 1
    assert _status(lambda: capi.vsample_dev(W.GAUSSIAN, par, 3, 1000, 0, 0, 0, 1, 0, 1 << 20, None,
                                            3 << 20)) == 1
    assert _status(lambda: capi.vsample_dev(W.GAUSSIAN, par, 3, 1000, 0, 0, 0, 0, 0, 1 << 20, None,
                                            3 << 20, d_probe=5 << 20, probe_shift=32)) == 1
    assert _status(lambda: capi.rebin_dev(3, 1 << 20, 2 << 20, 1 << 20)) == 1
    assert _status(lambda: capi.rebin_dev(0, 1 << 20, 2 << 20, 3 << 20)) == 2


def test_workspace_bytes(capi):
    assert capi.workspace_bytes(0) == 0 and capi.workspace_bytes(17) == 0
    for d in range(1, 17):
        b = capi.workspace_bytes(d)
        assert b % 256 == 0 and b >= d * 500 * 8 + 16


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2302_05730_gb300._capi as mod
    src = open(mod.__file__).read()
    fake = tmp_path / "_capi_probe.py"
    fake.write_text(src.replace('LIB_PATH = os.path.join(_HERE, "libmcubes.so")',
                                'LIB_PATH = os.path.join(_HERE, "missing-libmcubes.so")'))
    sys.path.insert(0, str(tmp_path))
    try:
        with pytest.raises(ImportError):
            importlib.import_module("_capi_probe")
    finally:
        sys.path.remove(str(tmp_path))


def test_combine_matches_inverse_variance_weighting(capi):
    rng = np.random.default_rng(4)
    I = rng.normal(2.0, 0.01, 9)
    V = rng.uniform(1e-6, 1e-4, 9)
    it = np.stack([I, V], axis=1)
    for skip in (0, 1, 4, 8):
        r = capi.combine(it, skip=skip)
        w = 1.0 / V[skip:]
        est = np.average(I[skip:], weights=w)
        assert abs(r["estimate"] - est) <= 1e-14 * abs(est)
        assert abs(r["error"] - np.sqrt(1.0 / w.sum())) <= 1e-14
        n = len(w)
        chi = np.sum(w * (I[skip:] - est) ** 2) / (n - 1) if n > 1 else 0.0
        assert abs(r["chi2_dof"] - chi) <= 1e-12 * max(chi, 1.0)
        assert r["iters_done"] == 9 - skip
    # zero-variance iterations dominate: their mean, error 0
    it2 = it.copy()
    it2[3, 1] = 0.0
    it2[5, 1] = 0.0
    r = capi.combine(it2)
    assert r["estimate"] == (it2[3, 0] + it2[5, 0]) / 2 and r["error"] == 0.0
    for bad in (dict(skip=9), dict(skip=-1)):
        with pytest.raises(capi.McubesError):
            capi.combine(it, **bad)
    it3 = it.copy()
    it3[2, 1] = np.nan
    with pytest.raises(capi.McubesError):
        capi.combine(it3)


def test_integrate_range_argument_checks(capi):
    par = W.genz_params(W.GAUSSIAN, 3)
    assert _status(lambda: capi.integrate_range(W.GAUSSIAN, par, 3, 1000, 6, 3, 2, 4, 0)) == 1   # no grid_in
    assert _status(lambda: capi.integrate_range(W.GAUSSIAN, par, 3, 1000, 6, 3, 4, 4, 0)) == 1   # empty range
    assert _status(lambda: capi.integrate_range(W.GAUSSIAN, par, 3, 1000, 6, 3, 5, 7, 0,
                                                grid_in=oracle.uniform_grid(3))) == 1          # past itmax


def test_flow_sample_work_bytes_and_argument_checks(capi):
    """The fused samplers' scratch holds the larger of two bf16 weight mirrors, then a 256-byte
    flag: the mma.sync layout per layer (W1 [H][24], W2 [H][H+8], W3 [N3][H+8] bf16, biases FP32,
    16-byte aligned) and the tcgen05 core-matrix layout (W1 [H][16], W2 [H][H], W3 [N3][H] bf16,
    b1, b2, b3 [N3] FP32), with N3 = |B| SW rounded up to 16, SW = 2K+1 rounded up to 8.
    Argument and workspace checks answer before any CUDA call."""
    al = lambda b, q=16: (b + q - 1) // q * q

    def layer_bytes(H, nB, K):
        SW = al(2 * K + 1, 8)
        return al(2 * H * 24) + al(2 * H * (H + 8)) + al(2 * al(nB * SW) * (H + 8)) + 2 * al(4 * H) + al(4 * nB * SW)

    def tc_layer_bytes(H, nB, K):
        N3 = al(nB * al(2 * K + 1, 8))
        return al(32 * H + 2 * H * H + 2 * N3 * H + 8 * H + 4 * N3)

    def scratch(H, K, nbs):
        return al(max(sum(layer_bytes(H, nb, K) for nb in nbs), sum(tc_layer_bytes(H, nb, K) for nb in nbs)), 256) + 256
    assert capi.flow_sample_work_bytes(capi.flow_shape(8, 4, 64, 16)) == scratch(64, 16, (4, 4, 4, 4))
    # d = 7: |B| = 4, 3, 3, 4 (upper half, lower half, odd axes, even axes)
    assert capi.flow_sample_work_bytes(capi.flow_shape(7, 4, 32, 8)) == scratch(32, 8, (4, 3, 3, 4))
    assert capi.flow_sample_work_bytes(capi.flow_shape(8, 17, 64, 16)) == 0    # more than 16 layers
    assert capi.flow_sample_work_bytes(capi.flow_shape(8, 4, 48, 16)) == 0     # unsupported width
    par = W.genz_params(W.GAUSSIAN, 8)
    sh = capi.flow_shape(8, 4, 64, 16)
    nb = capi.flow_sample_work_bytes(sh)
    call = lambda **kw: capi.flow_sample_dev(sh, kw.get("p", 1 << 20), W.GAUSSIAN, par, kw.get("ncall", 1 << 20), 0,
                                             0, 0, kw.get("i0", 0), kw.get("n", 100), 2 << 20, kw.get("ws", 3 << 20),
                                             kw.get("nb", nb))
    assert _status(lambda: call(n=-1)) == 1
    assert _status(lambda: call(ws=None)) == 8
    assert _status(lambda: call(ws=(3 << 20) + 64)) == 8
    assert _status(lambda: call(nb=nb - 16)) == 8
    assert _status(lambda: call(i0=781250 - 50)) == 1       # past the iteration's m p samples
    assert _status(lambda: call(p=None)) == 1


def test_pagani_rule_size_and_argument_checks(capi):
    for d in range(2, 17):
        assert capi.pagani_rule_points(d) == 1 + 4 * d + 2 * d * (d - 1) + 2 ** d
    assert capi.pagani_rule_points(1) == 0 and capi.pagani_rule_points(17) == 0
    par = W.genz_params(W.GAUSSIAN, 3)
    ev = lambda fid=W.GAUSSIAN, d=3, n=10, p=1 << 20, params=par: capi.pagani_evaluate_dev(
        fid, params, d, n, p, p, p, p, p)
    assert _status(lambda: ev(d=1, params=W.genz_params(W.GAUSSIAN, 1))) == 2
    assert _status(lambda: ev(d=17, params=np.ones(34))) == 2
    assert _status(lambda: ev(fid=10)) == 3
    assert _status(lambda: ev(n=-1)) == 1
    assert _status(lambda: ev(p=None)) == 1
    assert _status(lambda: capi.pagani_integrate(W.GAUSSIAN, par, 3, 0.0)) == 1
    assert _status(lambda: capi.pagani_integrate(W.GAUSSIAN, par, 3, 1e-3, max_iters=0)) == 1
    assert _status(lambda: capi.pagani_integrate(W.GAUSSIAN, par, 3, 1e-3, init_split=0)) == 1
    assert _status(lambda: capi.pagani_integrate(W.GAUSSIAN, par, 3, 1e-3, max_regions=7, init_split=2)) == 1
