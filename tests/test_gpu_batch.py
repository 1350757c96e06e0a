"""GPU parity of the batched form (mcubes_integrate_batch): every job of a mixed batch equals the
oracle's whole run of that job (Philox job word = the job's index), in both precisions and both
histogram modes. The autotuner returns valid launch shapes that do not change the results."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2302_05730_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi as c
    return c


def _mixed_jobs(n=22, seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n):
        fid = int(rng.integers(0, 8))
        d = int(rng.integers(1, 9))
        ncall = int(np.exp(rng.uniform(np.log(2e3), np.log(1.2e5))))
        par = W.constant_params(d, 1.5) if fid == W.CONSTANT else (
            W.paper_params(fid, d) if fid == W.ADDITION else W.genz_params(fid, d, seed=k))
        jobs.append(dict(fid=fid, d=d, ncall=ncall, params=par, seed=1000 + k))
    # edge cases: a single sub-cube with many samples, and the smallest problem
    jobs.append(dict(fid=W.GAUSSIAN, d=4, ncall=31, params=W.genz_params(W.GAUSSIAN, 4), seed=7))
    jobs.append(dict(fid=W.C0, d=2, ncall=2, params=W.genz_params(W.C0, 2), seed=8))
    return jobs


def _oracle_runs(jobs, itmax, adjust, mode):
    return [oracle.integrate(j["fid"], j["d"], j["params"], j["ncall"], itmax, adjust, j["seed"], job=k, mode=mode)
            for k, j in enumerate(jobs)]


@pytest.mark.parametrize("hist_mode,plain", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_batch_fp64_matches_oracle(capi, hist_mode, plain):
    """plain = 0: the Genz families' classes take the fast FP64 kernel (the others hist_mode's
    plain kernel); plain = 1: every class the plain kernel with hist_mode's histogram."""
    jobs = _mixed_jobs()
    itmax, adjust = 4, 2
    tune = None
    if hist_mode == 1 or plain:
        tune = capi.BatchTuning()
        tune.fp64_plain = plain
        for d in range(1, 17):
            tune.block_threads[d] = 128 if hist_mode == 1 else 256
            tune.cubes_per_thread[d] = 2 if hist_mode == 1 else 4
            tune.hist_mode[d] = hist_mode
    got = capi.integrate_batch(jobs, itmax, adjust, precision=0, tune=tune, return_iters=True)
    ref = _oracle_runs(jobs, itmax, adjust, 0)
    for k, (g, r) in enumerate(zip(got, ref)):
        est, sig, chi2, iI, iV = r
        assert g["status"] == 0
        scale = max(abs(est), sig, 1e-300)
        assert abs(g["estimate"] - est) <= 1e-10 * scale, (k, jobs[k]["fid"], g["estimate"], est)
        if jobs[k]["fid"] != W.CONSTANT:   # a constant's variance is pure rounding noise
            assert math.isclose(g["error"], sig, rel_tol=1e-8, abs_tol=1e-300), (k, g["error"], sig)
        assert np.allclose(g["iters"][:, 0], iI, rtol=1e-9, atol=1e-10 * max(np.abs(iI).max(), 1e-300)), k


def test_batch_fast_class_falls_back_whole(capi):
    """A (d, family) class takes the fast FP64 kernel only when every job of it can: one job with a
    zero a_i (oscillatory) or a negative a_i (C0) sends its whole class to the plain kernel, while
    the other classes keep the fast one. Every job still equals the oracle's run."""
    d = 3
    jobs = []
    for k, fid in enumerate([W.OSCILLATORY, W.OSCILLATORY, W.C0, W.C0, W.GAUSSIAN, W.PRODUCT_PEAK]):
        par = W.genz_params(fid, d, seed=40 + k)
        if k == 1:
            par[1] = 0.0
        if k == 3:
            par[0] = -par[0]
        jobs.append(dict(fid=fid, d=d, ncall=30000 + 977 * k, params=par, seed=60 + k))
    got = capi.integrate_batch(jobs, 3, 2, precision=0, return_iters=True)
    ref = _oracle_runs(jobs, 3, 2, 0)
    for k, (g, r) in enumerate(zip(got, ref)):
        est, sig, chi2, iI, iV = r
        assert g["status"] == 0
        assert abs(g["estimate"] - est) <= 1e-10 * max(abs(est), sig), (k, g["estimate"], est)
        assert math.isclose(g["error"], sig, rel_tol=1e-8), (k, g["error"], sig)


def test_batch_fp32_matches_oracle(capi):
    jobs = [j for j in _mixed_jobs(seed=1) if j["d"] >= 2 or j["ncall"] < 2 ** 24]
    itmax, adjust = 3, 2
    got = capi.integrate_batch(jobs, itmax, adjust, precision=1, return_iters=True)
    ref = _oracle_runs(jobs, itmax, adjust, 1)
    for k, (g, r) in enumerate(zip(got, ref)):
        est, sig, chi2, iI, iV = r
        assert g["status"] == 0
        # first iteration on the same uniform grid: per-iteration FP32-eval tolerance,
        # condition-scaled by the iteration's (1/m) sum |I_t|
        r0 = oracle.vsample(jobs[k]["fid"], jobs[k]["d"], jobs[k]["params"], jobs[k]["ncall"], jobs[k]["seed"],
                            it=0, job=k, mode=1, adjust=0, per_cube=True)
        cond = max(np.abs(r0["cubeI"]).mean(), 1e-300)
        assert abs(g["iters"][0, 0] - iI[0]) <= 1e-5 * cond, (k, g["iters"][0, 0], iI[0])
        # after the first refinement the two runs sample grids refined from single- vs
        # double-precision bin contributions; with the same draws the estimates stay within
        # one combined standard deviation
        assert abs(g["estimate"] - est) <= sig + 1e-5 * cond, (k, g["estimate"], est, sig)
    # the same batch with another launch shape: the global histogram sums in FP64 where the
    # block histogram sums in FP32 (in an order the atomics leave open), so the bin contributions
    # differ at single-precision rounding and the refined grids by far less than a bin. The two
    # runs then sample slightly different grids with the same draws: their estimates agree to a
    # small fraction of the statistical error (1e-3 sigma) and to 1e-5 of the estimate.
    tune = capi.BatchTuning()
    for d in range(1, 17):
        tune.block_threads[d] = 128
        tune.cubes_per_thread[d] = 8
        tune.hist_mode[d] = 1
    again = capi.integrate_batch(jobs, itmax, adjust, precision=1, tune=tune)
    for k, (g, h) in enumerate(zip(got, again)):
        assert abs(g["estimate"] - h["estimate"]) <= 1e-3 * g["error"] + 1e-5 * abs(g["estimate"]), k


def test_autotuner_shapes_and_results(capi):
    jobs = [dict(fid=W.GAUSSIAN, d=int(d), ncall=int(n), params=W.genz_params(W.GAUSSIAN, int(d), seed=i), seed=i)
            for i, (d, n) in enumerate([(2, 40000), (3, 90000), (3, 5000), (5, 200000), (8, 300000), (2, 100)])]
    t = capi.tune_batch(jobs, precision=1)
    shapes = t.as_dict()
    assert sorted(shapes) == [2, 3, 5, 8]
    for d, s in shapes.items():
        assert s["block_threads"] in (128, 256) and s["cubes_per_thread"] in (1, 2, 4, 8, 16)
        assert s["hist_mode"] in (0, 1)
    a = capi.integrate_batch(jobs, 4, 2, precision=0)
    b = capi.integrate_batch(jobs, 4, 2, precision=0, tune=t)
    for x, y in zip(a, b):
        assert math.isclose(x["estimate"], y["estimate"], rel_tol=1e-11)


def test_batch_reports_nonfinite_job(capi):
    jobs = [dict(fid=W.GAUSSIAN, d=2, ncall=1000, params=W.genz_params(W.GAUSSIAN, 2), seed=1),
            dict(fid=W.DISCONTINUOUS, d=1, ncall=1000, params=np.array([1000.0, 1.0]), seed=2),
            dict(fid=W.C0, d=3, ncall=1000, params=W.genz_params(W.C0, 3), seed=3)]
    out = capi.integrate_batch(jobs, 2, 1, precision=0, raise_on_error=False)
    assert [o["status"] for o in out] == [0, 6, 0]
    ref = oracle.integrate(W.C0, 3, jobs[2]["params"], 1000, 2, 1, 3, job=2, mode=0)
    assert math.isclose(out[2]["estimate"], ref[0], rel_tol=1e-10)
