"""The bounds-checked build (libmcubes_checked.so, `build(checked=True)`) as a sanitizer stand-in.

Its kernels check every computed bin, sub-cube, probe and batch-tile index against its bound and
count failures instead of accessing out of bounds. Tiny configurations (d = 1..3, m <= 64 sub-cubes,
every integrand, both precisions, adjusting and frozen, single jobs, a batch and the probe output)
run through it in a child process beside the oracle: results within the parity tolerances and no
failed check.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import oracle
from paper_2302_05730_gb300 import capi, workloads as W

assert capi.checked_violations() == (0, 0), "not a fresh checked library"

def params(fid, d):
    if fid == W.DOUBLE_GAUSSIAN:
        return W.double_gaussian_params(d, a=6.0, u=0.3)
    if fid == W.ROTATED_GAUSSIAN:
        return W.rotated_gaussian_params(d, seed=1, lam_min=1.0, lam_max=40.0)
    if fid == W.CONSTANT:
        return W.constant_params(d, 2.5)
    if fid == W.ADDITION:
        return W.paper_params(fid, d)
    return W.genz_params(fid, d, seed=d)

cases = 0
for d, n in [(1, 128), (2, 128), (3, 128), (2, 37), (3, 2)]:
    for fid in range(10):
        par = params(fid, d)
        for mode in (0, 1):
            for adjust in (1, 0):
                g = capi.vsample_once(fid, par, d, n, 11, iteration=1, adjust=adjust, precision=mode)
                r = oracle.vsample(fid, d, par, n, 11, it=1, mode=mode, adjust=adjust, per_cube=True)
                scale = float(np.abs(r["cubeI"]).sum()) / r["m"] + 1e-300
                tol = (1e-12 if mode == 0 else 1e-5) * scale
                assert abs(g["I"] - r["I"]) <= tol, (fid, d, n, mode, g["I"], r["I"])
                if adjust:
                    assert np.allclose(g["C"], r["C"], rtol=1e-12 if mode == 0 else 1e-4,
                                       atol=1e-6 * float(r["C"].mean()) + 1e-300), (fid, d, n, mode)
                cases += 1

# the probe output and explicit launch shapes
d, n, fid = 3, 128, W.GAUSSIAN
par = params(fid, d)
g_, m, p = capi.stratify(d, n)
dev = torch.device("cuda")
B = torch.from_numpy(oracle.uniform_grid(d)).to(dev)
for tune in (None, dict(block_threads=64), dict(blocks_per_sm=3)):
    probe = torch.zeros(((m >> 1) + 1, 2), dtype=torch.float64, device=dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    C = torch.zeros(d * 500, dtype=torch.float64, device=dev)
    capi.vsample_dev(fid, par, d, n, 3, 0, 0, 1, 1, B, C, sums, d_probe=probe, probe_shift=1, tune=tune)
    torch.cuda.synchronize()
    cases += 1

# a batch of tiny jobs, both precisions
jobs = [dict(fid=f, d=1 + f % 3, ncall=[2, 37, 128][f % 3], params=params(f, 1 + f % 3), seed=f) for f in range(10)]
for prec in (0, 1):
    capi.integrate_batch(jobs, 3, 2, precision=prec)
    cases += 1

v = capi.checked_violations()
print("cases", cases, "violations", v)
assert v == (0, 0), v
'''


def test_checked_build_runs_tiny_cases_without_violations():
    from paper_2302_05730_gb300.build import build
    lib = build(checked=True)
    env = dict(os.environ, MCUBES_LIB=lib)
    out = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=1800)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "violations (0, 0)" in out.stdout, out.stdout


def test_normal_build_reports_no_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi
    if os.environ.get("MCUBES_LIB"):
        pytest.skip("a non-default library is loaded")
    assert capi.checked_violations() is None
