"""Allocation failures through the library's fault hook (mcubes_fail_alloc).

Every allocation an entry point makes can fail. The call must then return ALLOC, having released
what it had allocated, and the next call, with nothing armed, must allocate afresh and give the
undisturbed result. The failure is made on the host (the allocation wrapper returns the
out-of-memory error): no GPU fault is involved.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2302_05730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ALLOC = 5


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi as c
    yield c
    c.fail_alloc(0)


def _expect_alloc(capi, fn):
    with pytest.raises(capi.McubesError) as e:
        fn()
    assert e.value.status == ALLOC, e.value


def _count_allocations(capi, fn):
    capi.fail_alloc(0)
    before = capi.fail_alloc(0)
    out = fn()
    return out, capi.fail_alloc(0) - before


@pytest.mark.parametrize("precision", [0, 1])
def test_integrate_survives_each_failed_allocation(capi, precision):
    d, fid = 4, W.GAUSSIAN
    par = W.genz_params(fid, d, seed=1)

    def run():
        return capi.integrate(fid, par, d, 20000, 4, 2, 9, precision=precision)

    capi.shutdown()   # a fresh workspace: the call allocates everything it needs
    ref, n = _count_allocations(capi, run)
    assert n >= 5, n   # two grids, C, the iteration sums, pinned staging
    for k in range(1, n + 1):
        capi.shutdown()
        capi.fail_alloc(k)
        _expect_alloc(capi, run)
        capi.fail_alloc(0)
        got = run()
        # the same draws and kernels; only the order of floating-point atomics may differ
        assert math.isclose(got["estimate"], ref["estimate"], rel_tol=1e-12 if precision == 0 else 1e-7), (k, got, ref)
        assert math.isclose(got["error"], ref["error"], rel_tol=1e-9 if precision == 0 else 1e-5), (k, got, ref)


def test_vsample_once_after_failed_workspace(capi):
    d, fid = 3, W.C0
    par = W.genz_params(fid, d, seed=2)

    def run():
        return capi.vsample_once(fid, par, d, 30000, 5, iteration=1, adjust=1)

    capi.shutdown()
    ref, n = _count_allocations(capi, run)
    for k in range(1, n + 1):
        capi.shutdown()
        capi.fail_alloc(k)
        _expect_alloc(capi, run)
        capi.fail_alloc(0)
        got = run()
        assert math.isclose(got["I"], ref["I"], rel_tol=1e-12), (k, got["I"], ref["I"])
        assert np.allclose(got["grid"], ref["grid"], rtol=0, atol=1e-13)


def test_batch_survives_each_failed_allocation(capi):
    jobs = [dict(fid=W.GAUSSIAN, d=3, ncall=20000, params=W.genz_params(W.GAUSSIAN, 3), seed=1),
            dict(fid=W.C0, d=5, ncall=50000, params=W.genz_params(W.C0, 5), seed=2)]

    def run():
        return capi.integrate_batch(jobs, 4, 2, precision=0)

    ref, n = _count_allocations(capi, run)
    assert n >= 2, n   # the plan's block and each class's tile list
    for k in range(1, n + 1):
        capi.fail_alloc(k)
        _expect_alloc(capi, run)
        capi.fail_alloc(0)
        got = run()
        for g, r in zip(got, ref):
            assert math.isclose(g["estimate"], r["estimate"], rel_tol=1e-12), (k, g, r)


def test_flow_and_pagani_fail_cleanly(capi):
    d = 4
    par = W.genz_params(W.GAUSSIAN, d, seed=3)

    def flow():
        return capi.flow_integrate(W.GAUSSIAN, par, d, layers=2, hidden=32, bins=8, loss="variance", vegas_iters=2,
                                   flow_iters=2, train_steps=20, batch=1 << 12, lr=1e-3, ncall=1 << 14,
                                   train_samples=1 << 14, seed=1)

    def pagani():
        return capi.pagani_integrate(W.GAUSSIAN, par, d, 1e-4, max_iters=20, max_regions=1 << 18)

    for fn in (flow, pagani):
        ref, n = _count_allocations(capi, fn)
        assert n >= 1
        capi.fail_alloc(1)
        _expect_alloc(capi, fn)
        capi.fail_alloc(0)
        got = fn()
        if fn is pagani:
            assert math.isclose(got["estimate"], ref["estimate"], rel_tol=1e-12) and got["iterations"] == ref["iterations"]
        else:
            assert math.isfinite(got["flow"]["estimate"]) and got["flow"]["error"] > 0


def test_environment_variable_arms_the_hook(tmp_path):
    """MCUBES_FAULT_ALLOC=n arms the hook at the library's first allocation (a fresh process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2302_05730_gb300 import capi, workloads as W\n"
        "par = W.genz_params(W.GAUSSIAN, 3)\n"
        "try:\n"
        "    capi.integrate(W.GAUSSIAN, par, 3, 20000, 3, 1, 1)\n"
        "    print('no failure')\n"
        "except capi.McubesError as e:\n"
        "    print('status', e.status)\n"
        "r = capi.integrate(W.GAUSSIAN, par, 3, 20000, 3, 1, 1)\n"
        "print('then', r['iters_done'])\n" % root)
    env = dict(os.environ, MCUBES_FAULT_ALLOC="2")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "status %d" % ALLOC in out.stdout and "then 3" in out.stdout, out.stdout


def test_run_log_lines(tmp_path):
    """MCUBES_LOG=<file>: one JSON line per iteration and one per call, matching the returned
    per-iteration results and estimate (a child process with the variable set)."""
    import json
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    log = tmp_path / "run.jsonl"
    out_json = tmp_path / "out.json"
    code = (
        "import sys, json; sys.path.insert(0, %r)\n"
        "from paper_2302_05730_gb300 import capi, workloads as W\n"
        "par = W.genz_params(W.C0, 4)\n"
        "r = capi.integrate(W.C0, par, 4, 40000, 5, 2, 3, precision=1, return_iters=True)\n"
        "q = capi.integrate_range(W.C0, par, 4, 40000, 5, 2, 0, 2, 3, precision=0)\n"
        "json.dump({'est': r['estimate'], 'err': r['error'], 'iters': r['iters'].tolist()}, open(%r, 'w'))\n"
        % (root, str(out_json)))
    env = dict(os.environ, MCUBES_LOG=str(log))
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    ref = json.loads(out_json.read_text())
    it_lines = [x for x in lines if x["event"] == "iteration" and x["call"] == "integrate"]
    runs = [x for x in lines if x["event"] == "run"]
    assert len(it_lines) == 5 and [x["it"] for x in it_lines] == list(range(5))
    assert [x["adjust"] for x in it_lines] == [True, True, False, False, False]
    for x, (I, V) in zip(it_lines, ref["iters"]):
        assert math.isclose(x["I"], I, rel_tol=1e-15) and math.isclose(x["sigma"], math.sqrt(V), rel_tol=1e-15)
    assert [r["call"] for r in runs] == ["integrate", "integrate_range"]
    assert math.isclose(runs[0]["estimate"], ref["est"], rel_tol=1e-15)
    assert math.isclose(it_lines[-1]["running_estimate"], ref["est"], rel_tol=1e-12)
    assert runs[0]["precision"] == "fp32_eval" and runs[1]["precision"] == "fp64" and runs[1]["iterations"] == 2
    assert runs[0]["ms"] > 0 and runs[0]["samples_per_s"] > 0
