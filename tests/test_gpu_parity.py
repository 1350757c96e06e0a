"""GPU parity: the CUDA V-Sample and Rebin kernels (through the C ABI) against the CPU oracle,
on the same seeded inputs.

Tolerances (FP64 path):
  - I: |dI| <= 1e-12 * (1/m) sum_t |I_t|. Condition-scaled, since the oscillatory family
    changes sign.
  - Var: |dV| <= 1e-12 V + floor. The floor is 8 eps (1/m^2) sum_t S2_t / (p (p-1)), the
    rounding floor of S2 - S1^2/p that Algorithm 2's sum-of-squares form carries.
  - C: 1e-12 relative per bin, plus 1e-14 of the axis' mean bin. The floor covers bins whose
    few weights sit near a zero of the oscillatory family, where libm cos and CUDA cos
    differ in relative terms.
  - Rebinned grid: 1e-13 absolute.
FP32-eval path (point and integrand in single precision; per-cube combination and sums FP64):
  - I and Var: 1e-5, with the same scaling.
  - C: 1e-4 relative per bin, plus 1e-6 of the axis' mean bin. C is accumulated in single
    precision per block. Bins whose weights underflow single precision, or sit near a zero
    of the oscillatory family, fall under the floor. Rebin only sees C_k / sum C.
  - Rebinned grid: the Rebin kernel is FP64 in both modes and is checked on the GPU's own C
    (1e-13). Bins whose contribution underflows single precision are exactly zero on the GPU.
    The VEGAS damping still gives a bin with rho = 1e-300 the weight (1/ln(1/rho))^1.5 ~ 5e-5,
    so the grid refined from the oracle's FP64 C can differ visibly in such tails.
  - Whole runs: the grids are refined from single-precision bin contributions, so the two
    runs sample slightly different grids. The estimates then agree to a fraction of their
    statistical error (0.2 sigma), not to 1e-5.
The bin index and the point x are decided in the same precision on both sides, so they
match exactly.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2302_05730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
ALL = list(range(10))


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi as c
    return c


def _params(fid, d, seed=0):
    if fid == W.DOUBLE_GAUSSIAN:
        return W.double_gaussian_params(d, a=6.0, u=0.3)
    if fid == W.ROTATED_GAUSSIAN:
        return W.rotated_gaussian_params(d, seed=seed, lam_min=1.0, lam_max=40.0)
    if fid == W.CONSTANT:
        return W.constant_params(d, 2.5)
    if fid == W.ADDITION:
        return W.paper_params(fid, d)
    return W.genz_params(fid, d, seed=seed)


def _random_grid(d, seed):
    rng = np.random.default_rng(seed)
    B = np.empty((d, 501))
    for i in range(d):
        w = 10.0 ** rng.uniform(-3.0, 0.0, 500)
        c = np.concatenate([[0.0], np.cumsum(w)])
        B[i] = c / c[-1]
        B[i, 0], B[i, -1] = 0.0, 1.0
    return B


# Per-sample relative error of the FP32-eval weight (single-precision point -> integrand ->
# Jacobian, SFU exp2): a few 2^-21. Its square bounds the FP32 variance floor.
F32_W = 2.0 ** -19


def _tols(ref, mode):
    """(absolute tolerance of I, relative tolerance of Var, absolute floor of Var)."""
    m, p = ref["m"], ref["p"]
    cI = np.abs(ref["cubeI"]).sum() / m
    s2 = ref["cubeV"] + ref["cubeI"] ** 2 / (p - 1)          # S2_t / (p (p-1))
    rel = 1e-12 if mode == 0 else 1e-5
    floor = (8 * EPS if mode == 0 else 4 * F32_W ** 2) * s2.sum() / m ** 2
    return rel * cI, rel, floor


def _osc_extra(fid, mode, d, par, n, seed, it, job, B):
    """The oscillatory family's per-bin phase-rounding bound (tests/phase_bounds.py), FP64 only."""
    if fid != W.OSCILLATORY or mode != 0:
        return None
    from phase_bounds import oscillatory_c_bound
    return oscillatory_c_bound(d, par, n, seed, it, job, oracle.uniform_grid(d) if B is None else B)


def _compare(gpu, ref, mode, B=None, check_grid=True, c_extra=None):
    tolI, rel, vfloor = _tols(ref, mode)
    assert abs(gpu["I"] - ref["I"]) <= tolI, ("I", gpu["I"], ref["I"], tolI)
    assert abs(gpu["Var"] - ref["Var"]) <= rel * ref["Var"] + vfloor, ("Var", gpu["Var"], ref["Var"])
    if "C" in gpu:
        crel, cfloor = (1e-12, 1e-14) if mode == 0 else (1e-4, 1e-6)
        tol = crel * ref["C"] + cfloor * ref["C"].mean(axis=1, keepdims=True)
        if c_extra is not None and mode == 0:
            tol = tol + c_extra
        err = np.abs(gpu["C"] - ref["C"])
        assert np.all(err <= tol), ("C", float(np.max(err / tol)), float(np.max(err / np.maximum(ref["C"], 1e-300))))
    if check_grid and "grid" in gpu and B is not None:
        # Rebin kernel (FP64 in both modes) against the oracle's Rebin of the same C
        same = oracle.rebin(B, gpu["C"])
        assert np.allclose(gpu["grid"], same, rtol=0, atol=1e-13), np.max(np.abs(gpu["grid"] - same))
        if mode == 0:
            want = oracle.rebin(B, ref["C"])
            assert np.allclose(gpu["grid"], want, rtol=0, atol=1e-12), np.max(np.abs(gpu["grid"] - want))


# ------------------------------------------------------------------------------ Philox
def test_philox_matches_curand_device_function_and_oracle(capi):
    rng = np.random.default_rng(1)
    n = 1 << 16
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0, 0, 0, 0xFFFFFFFF]]
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    for seed in [0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF]:
        own = torch.empty_like(d_ctr)
        ref = torch.empty_like(d_ctr)
        hoisted = torch.empty_like(d_ctr)
        hoisted_reg = torch.empty_like(d_ctr)
        capi.philox_dev(d_ctr, n, seed, 0, own)
        capi.philox_dev(d_ctr, n, seed, 1, ref)
        capi.philox_dev(d_ctr, n, seed, 2, hoisted)
        capi.philox_dev(d_ctr, n, seed, 3, hoisted_reg)
        torch.cuda.synchronize()
        a = own.cpu().numpy().view(np.uint32)
        b = ref.cpu().numpy().view(np.uint32)
        assert np.array_equal(a, b)
        # the hoisted forms the single-job and batched samplers draw with, bit for bit
        assert np.array_equal(hoisted.cpu().numpy().view(np.uint32), b)
        assert np.array_equal(hoisted_reg.cpu().numpy().view(np.uint32), b)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for j in list(range(4)) + list(rng.integers(0, n, 40)):
            assert oracle.philox(ctr[j], key) == [int(v) for v in a[j]]


# ------------------------------------------------------------------------------ one iteration
CASES = []
for fid in ALL:
    for d, n in [(1, 1000), (2, 5000), (3, 30000), (5, 20000), (8, 40000)]:
        CASES.append((fid, d, n))
CASES += [(W.DOUBLE_GAUSSIAN, 3, 30000), (W.DOUBLE_GAUSSIAN, 8, 40000), (W.ROTATED_GAUSSIAN, 2, 5000),
          (W.ROTATED_GAUSSIAN, 5, 20000), (W.ROTATED_GAUSSIAN, 8, 40000)]
CASES += [(W.GAUSSIAN, 12, 2 * 3 ** 12), (W.C0, 16, 2 ** 17 + 7), (W.PRODUCT_PEAK, 10, 2 * 3 ** 10 + 5),
          (W.DISCONTINUOUS, 6, 123457), (W.OSCILLATORY, 4, 31), (W.CORNER_PEAK, 2, 2),
          (W.ADDITION, 7, 2 * 5 ** 7 + 99)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid,d,n", CASES)
def test_vsample_parity(capi, fid, d, n, mode):
    par = _params(fid, d, seed=d)
    B = _random_grid(d, 100 + d)
    seed, it, job = 12345 + d, 3, 0
    gpu = capi.vsample_once(fid, par, d, n, seed, iteration=it, job=job, adjust=1, precision=mode, grid_in=B)
    ref = oracle.vsample(fid, d, par, n, seed, it=it, job=job, mode=mode, adjust=1, B=B, per_cube=True)
    _compare(gpu, ref, mode, B, c_extra=_osc_extra(fid, mode, d, par, n, seed, it, job, B))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid", ALL)
def test_vsample_parity_adapted_grid(capi, fid, mode):
    """On a grid adapted by the oracle itself (narrow bins near the peak)."""
    d, n = 4, 60000
    par = _params(fid, d, seed=7)
    B = oracle.adapted_grid(fid, d, par, 20000, 3, seed=1, mode=0)
    gpu = capi.vsample_once(fid, par, d, n, 99, iteration=5, adjust=1, precision=mode, grid_in=B)
    ref = oracle.vsample(fid, d, par, n, 99, it=5, mode=mode, adjust=1, B=B, per_cube=True)
    _compare(gpu, ref, mode, B, c_extra=_osc_extra(fid, mode, d, par, n, 99, 5, 0, B))


LAUNCH_SHAPES = [None, dict(block_threads=64), dict(block_threads=96, blocks_per_sm=3),
                 dict(block_threads=256, blocks_per_sm=2), dict(blocks_per_sm=1), dict(blocks_per_sm=5)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid,d,n", [(W.GAUSSIAN, 3, 30000), (W.OSCILLATORY, 8, 40000), (W.C0, 12, 2 * 3 ** 12 + 5)])
def test_launch_shapes_match_oracle(capi, fid, d, n, mode):
    """Every block size and grid shape gives the oracle's sums and bin contributions: the FP32
    fixed-point histogram (8 low-word copies at d = 8, 4 at d = 12; its per-block pilot scale with
    any block size), the FP64 histogram, the frozen instance, and sub-cube ranges cut for any
    thread count."""
    par = _params(fid, d, seed=d)
    B = _random_grid(d, 40 + d)
    seed, it = 777 + d, 2
    ref = {a: oracle.vsample(fid, d, par, n, seed, it=it, mode=mode, adjust=a, B=B, per_cube=True) for a in (0, 1)}
    dev = torch.device("cuda")
    g_in = torch.from_numpy(B).to(dev)
    for tune in LAUNCH_SHAPES:
        for adjust in (1, 0):
            sums = torch.zeros(2, dtype=torch.float64, device=dev)
            C = torch.zeros(d * 500, dtype=torch.float64, device=dev)
            capi.vsample_dev(fid, par, d, n, seed, it, 0, adjust, mode, g_in, C, sums, tune=tune)
            torch.cuda.synchronize()
            s = sums.cpu().numpy()
            m = ref[adjust]["m"]
            gpu = dict(I=s[0] / m, Var=s[1] / m ** 2)
            if adjust:
                gpu["C"] = C.cpu().numpy().reshape(d, 500)
            else:
                assert not C.any()
            _compare(gpu, ref[adjust], mode,
                     c_extra=_osc_extra(fid, mode, d, par, n, seed, it, 0, B) if adjust else None)


@pytest.mark.parametrize("fid,d,n,a,u", [
    (W.DISCONTINUOUS, 8, 200000, 9.0, 0.3),    # nonzero on 0.3^8 = 7e-5 of the cube: most pilots see only zeros
    (W.GAUSSIAN, 8, 400000, 25.0, 0.5),       # contributions over hundreds of octaves on the uniform grid
    (W.PRODUCT_PEAK, 6, 300000, 40.0, 0.35),
])
def test_fp32_histogram_extreme_spreads(capi, fid, d, n, a, u):
    """FP32 bin contributions whose sizes defeat any one fixed-point scale: sparse integrands
    (blocks whose pilot sees no positive contribution) and peaks on the uniform grid (most
    contributions far below or above the block's scale) against the oracle's C."""
    par = np.concatenate([np.full(d, a), np.full(d, u)])
    for it, B in [(0, None), (3, _random_grid(d, 17))]:
        gpu = capi.vsample_once(fid, par, d, n, 4242, iteration=it, adjust=1, precision=1, grid_in=B)
        ref = oracle.vsample(fid, d, par, n, 4242, it=it, mode=1, adjust=1, B=B, per_cube=True)
        _compare(gpu, ref, 1, B)


@pytest.mark.parametrize("mode", [0, 1])
def test_frozen_iteration_and_uniform_grid(capi, mode):
    d, n, fid = 5, 77777, W.GAUSSIAN
    par = _params(fid, d)
    gpu = capi.vsample_once(fid, par, d, n, 5, iteration=9, job=3, adjust=0, precision=mode)
    ref = oracle.vsample(fid, d, par, n, 5, it=9, job=3, mode=mode, adjust=0, per_cube=True)
    assert "C" not in gpu and "grid" not in gpu
    _compare(gpu, ref, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_constant_integrand_exact(capi, mode):
    for d in [1, 4, 9]:
        par = W.constant_params(d, 3.25)
        g, m, p = capi.stratify(d, 50000)
        r = capi.vsample_once(W.CONSTANT, par, d, 50000, 1, adjust=0, precision=mode)
        tolI = 1e-13 if mode == 0 else 1e-6
        assert abs(r["I"] - 3.25) <= tolI * 3.25
        floor = (8 * EPS if mode == 0 else 4 * F32_W ** 2) * 3.25 ** 2 / ((p - 1) * m)
        assert r["Var"] <= floor


# ------------------------------------------------------------------------------ whole runs
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid,d", [(W.GAUSSIAN, 3), (W.OSCILLATORY, 5), (W.PRODUCT_PEAK, 6), (W.C0, 8),
                                   (W.CORNER_PEAK, 5), (W.DISCONTINUOUS, 4)])
def test_integrate_parity(capi, fid, d, mode):
    """Several adjusting and frozen iterations: the map is continuous in the grid and the bins
    depend only on the draws, so rounding-level grid differences stay at rounding level."""
    par = _params(fid, d, seed=11)
    n = 100000
    g = capi.integrate(fid, par, d, n, 6, 3, seed=4, precision=mode, return_iters=True, return_grid=True)
    est, sig, chi2, iI, iV = oracle.integrate(fid, d, par, n, 6, 3, seed=4, mode=mode)
    if mode == 0:
        rel = 1e-10
        assert abs(g["estimate"] - est) <= rel * max(abs(est), sig), (g["estimate"], est)
        assert math.isclose(g["error"], sig, rel_tol=1e-8)
        assert np.allclose(g["iters"][:, 0], iI, rtol=1e-9, atol=1e-10 * np.abs(iI).max())
    else:
        assert abs(g["estimate"] - est) <= 0.2 * sig + 1e-5 * abs(est), (g["estimate"], est, sig)
        assert math.isclose(g["error"], sig, rel_tol=0.05)
        # the first iteration samples the same (uniform) grid: per-iteration tolerance,
        # condition-scaled by (1/m) sum |I_t| of that iteration
        r0 = oracle.vsample(fid, d, par, n, 4, it=0, mode=1, adjust=0, per_cube=True)
        assert abs(g["iters"][0, 0] - iI[0]) <= 1e-5 * np.abs(r0["cubeI"]).mean()
    assert g["samples_per_iter"] == np.prod(capi.stratify(d, n)[1:])


def test_config1_gaussian_full_run(capi):
    """The d = 3 Gaussian, a_i = 10, u_i = 1/2, 1e6 samples/iteration, 10 iterations (5 adjust),
    seed 0: the GPU run equals the oracle's and the closed form lies within its error."""
    d = 3
    par = W.gaussian_params(d, 10.0)
    g = capi.integrate(W.GAUSSIAN, par, d, 10 ** 6, 10, 5, 0, precision=0, return_iters=True)
    est, sig, chi2, iI, iV = oracle.integrate(W.GAUSSIAN, d, par, 10 ** 6, 10, 5, 0, mode=0)
    assert abs(g["estimate"] - est) <= 1e-10 * est
    assert np.allclose(g["iters"][:, 1], iV, rtol=1e-8)
    exact = (math.sqrt(math.pi) / 10 * math.erf(5.0)) ** 3
    assert abs(g["estimate"] - exact) < 4 * g["error"]


@pytest.mark.parametrize("precision", [0, 1])
def test_paper_f1_f6_d8_against_closed_forms(capi, precision):
    """The paper's own fixed-parameter f1..f6 at d = 8 (Sec. 5, Eq. 1-6), whole runs of 10
    iterations (5 adjusting) at 1e7 samples per iteration, seed 0, in both precisions: every
    estimate lies within 4.5 sigma of its closed form, and sigma is below 1e-3 of the integral for
    all but f1 (whose integral, 3.4e-5, is small against |f| ~ 1)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from closed_forms import exact
    d = 8
    for fid in W.GENZ6:
        par = W.paper_params(fid, d)
        r = capi.integrate(fid, par, d, 10 ** 7, 10, 5, 0, precision=precision)
        ex = exact(fid, par[:d], par[d:])
        assert abs(r["estimate"] - ex) < 4.5 * r["error"], (fid, precision, r, ex)
        if fid != W.OSCILLATORY:
            assert r["error"] < 1e-3 * abs(ex), (fid, precision, r, ex)


# ------------------------------------------------------------------------------ device API
def test_device_iteration_matches_host_call(capi):
    d, n, fid = 6, 300000, W.C0
    par = _params(fid, d)
    B = _random_grid(d, 3)
    dev = torch.device("cuda")
    g_in = torch.from_numpy(B).to(dev)
    g_out = torch.empty_like(g_in)
    res = torch.zeros(2, dtype=torch.float64, device=dev)
    ws = torch.empty(capi.workspace_bytes(d) // 8 + 64, dtype=torch.float64, device=dev)
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    for mode in (0, 1):
        capi.iteration_dev(fid, par, d, n, 8, 1, 0, 1, mode, g_in, g_out, res, None, aligned,
                           capi.workspace_bytes(d), stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        h = capi.vsample_once(fid, par, d, n, 8, iteration=1, adjust=1, precision=mode, grid_in=B)
        r = res.cpu().numpy()
        # same kernel and inputs; only the order of the floating-point atomics differs (the grid takes
        # it through C, to the FP64 grid tolerance of the oracle-parity checks)
        assert math.isclose(r[0], h["I"], rel_tol=1e-13 if mode == 0 else 1e-9)
        assert math.isclose(r[1], h["Var"], rel_tol=1e-11 if mode == 0 else 1e-7)
        assert np.allclose(g_out.cpu().numpy(), h["grid"], rtol=0, atol=1e-12 if mode == 0 else 1e-8)


F32_MIN = float(np.finfo(np.float32).tiny)


def _weight_error_bounds(fid, d, par, x, w, J, mode, dk=None):
    """Bound on the rounding error of each sample weight w = f J in the kernel's precision.
    The integrand's argument (the exponent, the oscillatory phase) is a sum of d rounded terms,
    so its absolute error grows with its size, and f's relative error with it; J is a product of
    d rounded bin widths. FP32-eval weights also underflow below FLT_MIN times the integrand's
    scale factor F (the peak value: 1, prod a_i^2 for the product peak, e^{sum a min(u, 1)} for
    the discontinuous family).
    FP64 Genz families (dk: the samples' bin widths, n x d): the kernel forms a (x - u) (or a x)
    as one fma of per-bin table entries a Delta_k and a (B_k - u) - a Delta_k, each rounded once,
    so each term carries up to 2 eps a (2 |x - u| + 3 Delta_k) (x for |x - u| in the uncentred
    families) of absolute error, which the argument's error adds up as below."""
    eps = 2.0 ** -24 if mode == 1 else 2.0 ** -53
    a, u = par[:d], par[d:]
    aw = np.abs(w)
    base = eps * (8 + 2 * d)
    fold = None
    if mode == 0 and dk is not None and fid in W.GENZ6:
        cen = np.abs(x - u) if fid in (W.GAUSSIAN, W.C0, W.PRODUCT_PEAK) else np.abs(x)
        dv = 2 * eps * np.abs(a) * (2 * cen + 3 * dk)          # per axis, absolute error of a (x - u) or a x
        if fid == W.GAUSSIAN:
            fold = aw * np.sum(2 * np.abs(a) * cen * dv + dv * dv, axis=1)
        elif fid == W.OSCILLATORY:
            fold = np.abs(J) * np.sum(dv, axis=1)
        elif fid == W.CORNER_PEAK:
            fold = aw * (d + 1) * np.sum(dv, axis=1) / (1.0 + x @ a)
        else:   # C0, product peak (2 |v| / (1 + v^2) <= 1), discontinuous
            fold = aw * np.sum(dv, axis=1)
    if fid == W.OSCILLATORY:
        t = np.abs(u[0] + x @ a / (2 * np.pi))
        delta = aw * base + np.abs(J) * (2 * np.pi * eps * (d + 4) * (t + 1.0) + 4 * eps)
    elif fid in (W.GAUSSIAN, W.C0, W.DISCONTINUOUS):
        if fid == W.GAUSSIAN:
            arg = np.sum((a * (x - u)) ** 2, axis=1)
        elif fid == W.C0:
            arg = np.sum(a * np.abs(x - u), axis=1)
        else:
            arg = np.abs(x @ a - np.sum(a * np.minimum(u, 1.0)))
        delta = aw * (base + eps * 1.5 * (d + 4) * arg)
    elif fid == W.PRODUCT_PEAK:
        delta = aw * (base + eps * 6 * d)
    elif fid == W.CORNER_PEAK:
        delta = aw * (base + eps * 4 * (d + 1))
    else:
        delta = aw * (base + eps * d)
    if mode == 1:
        # f / F below FLT_MIN, and w / F in the subnormal range (spacing 2^-149)
        delta = delta + 4 * F32_MIN * _f32_scale(fid, d, par) * np.abs(J) + 2.0 ** -148 * _f32_scale(fid, d, par)
    if fold is not None:
        delta = delta + fold
    return delta


def _f32_scale(fid, d, par):
    """The FP32-eval integrand's scale factor F (the peak value)."""
    a, u = par[:d], par[d:]
    return {W.PRODUCT_PEAK: float(np.prod(a ** 2)),
            W.DISCONTINUOUS: float(np.exp(np.sum(a * np.minimum(u, 1.0))))}.get(fid, 1.0)


def _check_probes(capi, fid, d, n, mode, B, shift, par, seed=3, it=0, job=0):
    """One full V-Sample pass (adjusting) on the device with sub-cube probes: every probed
    sub-cube's (I_t, V_t) against the oracle's computation of that sub-cube alone, within the
    rounding the kernel's precision allows for that sub-cube's own samples."""
    g, m, p = capi.stratify(d, n)
    dev = torch.device("cuda")
    probe = torch.full(((m >> shift) + 1, 2), -1.0, dtype=torch.float64, device=dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    C = torch.zeros(d * 500, dtype=torch.float64, device=dev)
    capi.vsample_dev(fid, par, d, n, seed, it, job, 1, mode, torch.from_numpy(B).to(dev), C, sums,
                     d_probe=probe, probe_shift=shift)
    torch.cuda.synchronize()
    pr = probe.cpu().numpy()
    s = sums.cpu().numpy()
    assert np.all(np.isfinite(s)) and s[1] >= 0.0
    for t in range(0, m, 1 << shift):
        ref = oracle.vsample(fid, d, par, n, seed, it=it, job=job, mode=mode, adjust=0, B=B, t0=t, t1=t + 1,
                             per_cube=True)
        sp = oracle.sample_points(fid, d, par, n, seed, it=it, job=job, mode=mode, B=B, t0=t, t1=t + 1)
        dk = np.take_along_axis(np.diff(B, axis=1)[None, :, :].repeat(sp["k"].shape[0], 0),
                                sp["k"][:, :, None].astype(np.int64), axis=2)[:, :, 0]
        delta = _weight_error_bounds(fid, d, par, sp["x"], sp["w"], sp["J"], mode, dk)
        rel = 1e-12 if mode == 0 else 1e-6
        I_ref, V_ref = ref["cubeI"][0], ref["cubeV"][0]
        tol_I = rel * abs(I_ref) + delta.sum() / p + 1e-300
        assert abs(pr[t >> shift, 0] - I_ref) <= tol_I, (t, pr[t >> shift], I_ref, tol_I)
        # V = sum (w_q - I)^2 / (p (p-1)): a weight error delta_q moves it by at most
        # 2 sum |w_q - I| delta_q / (p (p-1)) <= 2 max(delta) sqrt(V / (p-1)) (plus delta^2 terms)
        md = float(delta.max())
        vf = (8 * EPS if mode == 0 else 4 * F32_W ** 2) * (V_ref + I_ref ** 2 / (p - 1))
        if mode == 1:   # squared FP32 differences below FLT_MIN (in units of F^2) lose their digits
            vf += 4 * F32_MIN * _f32_scale(fid, d, par) ** 2
        tol_V = rel * V_ref + vf + 2 * md * math.sqrt(V_ref / (p - 1)) + 2 * md * md
        assert abs(pr[t >> shift, 1] - V_ref) <= tol_V, (t, pr[t >> shift], V_ref, tol_V)
    return m >> shift


def test_probe_outputs_match_oracle_cubes(capi):
    d, n, fid = 5, 10 ** 6, W.PRODUCT_PEAK
    for mode in (0, 1):
        _check_probes(capi, fid, d, n, mode, _random_grid(d, 5), 10, _params(fid, d))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid", list(W.GENZ6))
def test_headline_size_probes(capi, fid, mode):
    """The bench's workload at full size: d = 8, 1e8 samples per iteration (m = 9^8 = 43,046,721
    sub-cubes, p = 2), the default launch shape; every 65,536th sub-cube against the oracle."""
    d, n = 8, 10 ** 8
    assert _check_probes(capi, fid, d, n, mode, _random_grid(d, 77), 16, W.genz_params(fid, d, seed=0),
                         seed=11, it=4, job=0) >= 600


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fid", [W.PRODUCT_PEAK, W.C0])
def test_large_d10_probes(capi, fid, mode):
    """d = 10 at 1e9 samples per iteration (g = 7, m = 282,475,249 sub-cubes, p = 3): the cube
    index stays within its 32-bit counter word; every 2^18-th sub-cube against the oracle."""
    d, n = 10, 10 ** 9
    assert _check_probes(capi, fid, d, n, mode, _random_grid(d, 78), 18, W.genz_params(fid, d, seed=0),
                         seed=12, it=7, job=0) >= 1000


def test_batched_full_size_sampled_jobs(capi):
    """The 4096-job batch of the bench (d ~ U{2..8}, samples per iteration log-uniform in
    [1e4, 1e7], 8 iterations, 4 adjusting) in one call; the twelve smallest jobs' whole runs
    against the oracle's (Philox job word = the job's index)."""
    jobs = W.batch_jobs(4096, seed=0)
    got = capi.integrate_batch(jobs, 8, 4, precision=0, return_iters=True)
    assert all(g["status"] == 0 for g in got)
    order = sorted(range(len(jobs)), key=lambda k: jobs[k]["ncall"])[:12]
    for k in order:
        j = jobs[k]
        est, sig, chi2, iI, iV = oracle.integrate(j["fid"], j["d"], j["params"], j["ncall"], 8, 4, j.get("seed", 0),
                                                  job=k)
        g = got[k]
        assert abs(g["estimate"] - est) <= 1e-10 * max(abs(est), sig), (k, g["estimate"], est)
        assert math.isclose(g["error"], sig, rel_tol=1e-8), (k, g["error"], sig)


# ------------------------------------------------------------------------------ errors
def test_nonfinite_integrand_reported(capi):
    d = 1
    par = np.array([1000.0, 1.0])   # exp(1000 x) overflows for x > 0.71
    with pytest.raises(capi.McubesError) as e:
        capi.vsample_once(W.DISCONTINUOUS, par, d, 1000, 1, adjust=0, precision=0)
    assert e.value.status == 6
    with pytest.raises(capi.McubesError) as e:    # FP32-eval: its scale factor exp(1000) is rejected
        capi.vsample_once(W.DISCONTINUOUS, par, d, 1000, 1, adjust=0, precision=1)
    assert e.value.status == 1


def test_invalid_arguments(capi):
    par = np.ones(4)
    with pytest.raises(capi.McubesError):
        capi.vsample_once(10, par, 2, 100, 1)
    with pytest.raises(ValueError):      # the rotated Gaussian needs d^2 + d parameters
        capi.vsample_once(9, par, 2, 100, 1)
    with pytest.raises(capi.McubesError):
        capi.vsample_once(0, par, 2, 1, 1)
    with pytest.raises(capi.McubesError):
        capi.integrate(0, par, 2, 100, 3, 4, 1)
    bad = oracle.uniform_grid(2)
    bad[0, 10] = bad[0, 9]
    with pytest.raises(capi.McubesError):
        capi.vsample_once(0, par, 2, 100, 1, grid_in=bad)


@pytest.mark.parametrize("mode", [0, 1])
def test_checkpoint_resume_repeats_the_run(capi, mode):
    """[0, 3) then [3, 7) from the returned grid equals the uninterrupted 7-iteration run."""
    d, n, fid = 4, 200000, W.GAUSSIAN
    par = _params(fid, d, seed=2)
    full = capi.integrate(fid, par, d, n, 7, 4, 9, precision=mode, return_iters=True, return_grid=True)
    a = capi.integrate_range(fid, par, d, n, 7, 4, 0, 3, 9, precision=mode)
    b = capi.integrate_range(fid, par, d, n, 7, 4, 3, 7, 9, precision=mode, grid_in=a["grid"],
                             prev_estimate=a["iters"][-1, 0])
    iters = np.concatenate([a["iters"], b["iters"]])
    rel = 1e-12 if mode == 0 else 1e-6
    assert np.allclose(iters[:, 0], full["iters"][:, 0], rtol=rel, atol=0)
    assert np.allclose(b["grid"], full["grid"], rtol=0, atol=1e-12 if mode == 0 else 1e-7)
    r = capi.combine(iters)
    assert math.isclose(r["estimate"], full["estimate"], rel_tol=rel)
