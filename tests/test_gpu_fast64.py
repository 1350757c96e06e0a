"""The FP64 V-Sample kernel with integer bin extraction and folded per-bin tables (the default
for the six Genz families) against the oracle and against the plain FP64 kernel that evaluates
the definition step by step (tuning fp64_plain = 1), on the same draws.

Both kernels decide the bin from the same FP64 yn, so C per bin must agree to FP64 rounding; the
discontinuous family's cut is decided exactly as defined, which these cases probe at grid
boundaries, inside bin 0 and outside the cube. The exp and cos the fast kernel evaluates are its
own (table-driven); the cases below also reach their library fallbacks (|x| >= 708) and large
phases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2302_05730_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
ND = 500


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi as c
    return c


def _random_grid(d, seed):
    rng = np.random.default_rng(seed)
    B = np.empty((d, ND + 1))
    for i in range(d):
        w = 10.0 ** rng.uniform(-3.0, 0.0, ND)
        c = np.concatenate([[0.0], np.cumsum(w)])
        B[i] = c / c[-1]
        B[i, 0], B[i, -1] = 0.0, 1.0
    return B


def _run(capi, fid, par, d, n, seed, it, adjust, B, plain):
    dev = torch.device("cuda")
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    C = torch.zeros(d * ND, dtype=torch.float64, device=dev)
    capi.vsample_dev(fid, par, d, n, seed, it, 0, adjust, 0, torch.from_numpy(B).to(dev), C if adjust else None,
                     sums, tune={"fp64_plain": 1} if plain else None)
    torch.cuda.synchronize()
    _, m, _ = capi.stratify(d, n)
    s = sums.cpu().numpy()
    out = dict(I=s[0] / m, Var=s[1] / (float(m) * float(m)))
    if adjust:
        out["C"] = C.cpu().numpy().reshape(d, ND)
    return out


def _check(got, ref, what, c_extra=None):
    m, p = ref["m"], ref["p"]
    cI = np.abs(ref["cubeI"]).sum() / m
    s2 = (ref["cubeV"] + ref["cubeI"] ** 2 / (p - 1)).sum() / m ** 2
    assert abs(got["I"] - ref["I"]) <= 1e-12 * cI, (what, "I", got["I"], ref["I"])
    assert abs(got["Var"] - ref["Var"]) <= 1e-12 * ref["Var"] + 8 * EPS * s2, (what, "Var", got["Var"], ref["Var"])
    if "C" in got:
        tol = 1e-12 * ref["C"] + 1e-14 * ref["C"].mean(axis=1, keepdims=True)
        if c_extra is not None:
            tol = tol + c_extra
        err = np.abs(got["C"] - ref["C"])
        assert np.all(err <= tol), (what, "C", float(np.max(err / np.maximum(tol, 1e-300))))


def _both(capi, fid, par, d, n, B, seed=31, it=2, adjust=1):
    ref = oracle.vsample(fid, d, par, n, seed, it=it, mode=0, adjust=adjust, B=B, per_cube=True)
    fast = _run(capi, fid, par, d, n, seed, it, adjust, B, plain=False)
    plain = _run(capi, fid, par, d, n, seed, it, adjust, B, plain=True)
    extra = None
    if adjust and fid == W.OSCILLATORY:   # the phase's FP64 rounding (tests/phase_bounds.py)
        from phase_bounds import oscillatory_c_bound
        extra = oscillatory_c_bound(d, par, n, seed, it, 0, B)
    _check(fast, ref, "fast", extra)
    _check(plain, ref, "plain", extra)
    return fast, plain, ref


@pytest.mark.parametrize("fid", list(W.GENZ6))
@pytest.mark.parametrize("d,n", [(1, 3000), (3, 40000), (8, 60000), (12, 2 * 3 ** 12 + 11)])
def test_fast_and_plain_match_oracle(capi, fid, d, n):
    par = W.genz_params(fid, d, seed=d + 3)
    for adjust in (1, 0):
        _both(capi, fid, par, d, n, _random_grid(d, 10 + d), adjust=adjust)


@pytest.mark.parametrize("fid", list(W.GENZ6))
def test_paper_parameters_and_uniform_grid(capi, fid):
    """The paper's f1..f6 at d = 8 on the uniform grid, where the discontinuous family's cuts
    (3 + i) / 10 fall on bin boundaries k / 500 exactly."""
    d = 8
    _both(capi, fid, W.paper_params(fid, d), d, 200000, oracle.uniform_grid(d))


@pytest.mark.parametrize("u", [0.4, 0.0011, 1e-9, 0.0, -0.3, 1.0, 1.7, 0.5 + 1e-16])
def test_discontinuous_cut_edges(capi, u):
    """Cuts on a bin boundary, inside bin 0 (where the offset is yn itself), at and beyond the
    cube's faces: every sample's inside/outside decision shows in C per bin."""
    d = 3
    par = np.concatenate([np.array([3.0, 5.0, 7.0]), np.array([u, 0.6, 0.35])])
    for B in (oracle.uniform_grid(d), _random_grid(d, 5)):
        _both(capi, W.DISCONTINUOUS, par, d, 90000, B)


def test_exp_fallback_and_large_phases(capi):
    """Exponents beyond 708 in magnitude (the library exp takes over) and oscillatory phases of
    hundreds of radians (tens of turns; larger phases carry FP64 rounding of the phase itself,
    above the 1e-12 parity bar whichever order the sum is taken in)."""
    d = 4
    B = _random_grid(d, 8)
    g = np.concatenate([np.full(d, 60.0), np.full(d, 0.5)])     # exponents up to 4 * 3600 * 0.25
    _both(capi, W.GAUSSIAN, g, d, 80000, B)
    _both(capi, W.C0, np.concatenate([np.full(d, 700.0), np.full(d, 0.5)]), d, 80000, B)
    osc = np.concatenate([np.array([200.0, 150.0, 17.0, 90.0]), np.full(d, 0.3)])
    _both(capi, W.OSCILLATORY, osc, d, 80000, B)


def test_signs_and_fallbacks(capi):
    """Negative a (the folded Jacobian keeps its sign), and parameters the fast kernel declines
    (a zero a_i; a negative a for C0), which take the plain kernel: all against the oracle."""
    d = 3
    B = _random_grid(d, 9)
    _both(capi, W.GAUSSIAN, np.array([-7.0, 5.0, -9.0, 0.3, 0.6, 0.5]), d, 50000, B)
    _both(capi, W.OSCILLATORY, np.array([-7.0, 5.0, 11.0, 0.3, 0.0, 0.0]), d, 50000, B)
    _both(capi, W.PRODUCT_PEAK, np.array([-7.0, 5.0, 11.0, 0.3, 0.6, 0.5]), d, 50000, B)
    _both(capi, W.OSCILLATORY, np.array([0.0, 5.0, 11.0, 0.3, 0.0, 0.0]), d, 50000, B)
    _both(capi, W.C0, np.array([-7.0, 5.0, 11.0, 0.3, 0.6, 0.5]), d, 50000, B)


def test_fast_kernel_is_faster(capi):
    """The point of the fast kernel: fewer FP64-pipe operations a sample. At d = 8, 2e7 samples,
    it must beat the plain kernel on every family (CUDA events, after a warm-up)."""
    d, n = 8, 2 * 10 ** 7
    dev = torch.device("cuda")
    B = torch.from_numpy(_random_grid(d, 4)).to(dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()   # the events' stream (a NULL stream is the library's own)
    for fid in W.GENZ6:
        par = W.genz_params(fid, d, seed=0)
        ms = {}
        for plain in (0, 1):
            tune = {"fp64_plain": plain}
            capi.vsample_dev(fid, par, d, n, 1, 5, 0, 0, 0, B, None, sums, tune=tune, stream=st)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                capi.vsample_dev(fid, par, d, n, 1, 5, 0, 0, 0, B, None, sums, tune=tune, stream=st)
            b.record()
            b.synchronize()
            ms[plain] = a.elapsed_time(b) / 3
        assert ms[0] < ms[1], (fid, ms)
