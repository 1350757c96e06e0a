"""ctypes binding of libmcubes.so (include/mcubes.h). Argument marshalling only.

Every call forwards to the C ABI of the same name without the ``mcubes_`` prefix. Every step of
the integration runs in the library's CUDA kernels. There is no CPU fallback: if the library
has not been built, or cannot be loaded, importing this module raises.

Device buffers may be given as torch CUDA tensors (their data_ptr is passed) or as raw
integer addresses. Streams may be a torch.cuda.Stream, a raw cudaStream_t integer, or None.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MCUBES_LIB selects another build of the library (the bounds-checked libmcubes_checked.so)
LIB_PATH = os.environ.get("MCUBES_LIB") or os.path.join(_HERE, "libmcubes.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mcubes.h")

NBINS = 500
DMAX = 16
FP64, FP32_EVAL = 0, 1

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_DIM", 3: "UNKNOWN_INTEGRAND", 4: "CUDA",
          5: "ALLOC", 6: "NONFINITE", 7: "TIMEOUT", 8: "WORKSPACE"}


class McubesError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.mcubes_status_string(status).decode() if _lib is not None else STATUS.get(status, "?")
        extra = ""
        if status == 4 and _lib is not None:
            extra = f" (cudaError {_lib.mcubes_last_cuda_error()})"
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}{extra}")


class Result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("error", ctypes.c_double),
                ("chi2_dof", ctypes.c_double), ("iters_done", ctypes.c_int32),
                ("status", ctypes.c_int32), ("samples_per_iter", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("fp64_plain", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class PaganiResult(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("error", ctypes.c_double), ("regions_evaluated", ctypes.c_int64),
                ("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("active_regions", ctypes.c_int64)]


class FlowShape(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("layers", ctypes.c_int32), ("hidden", ctypes.c_int32),
                ("bins", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("integrand_id", ctypes.c_int32), ("d", ctypes.c_int32), ("ncall", ctypes.c_int64),
                ("params", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_uint64)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32 * (DMAX + 1)),
                ("cubes_per_thread", ctypes.c_int32 * (DMAX + 1)),
                ("hist_mode", ctypes.c_int32 * (DMAX + 1)),
                ("fp64_plain", ctypes.c_int32)]

    def as_dict(self):
        return {d: dict(block_threads=self.block_threads[d], cubes_per_thread=self.cubes_per_thread[d],
                        hist_mode=self.hist_mode[d]) for d in range(1, DMAX + 1) if self.block_threads[d]}


class FlowConfig(ctypes.Structure):
    _fields_ = [("shape", FlowShape), ("loss_kind", ctypes.c_int32), ("vegas_iters", ctypes.c_int32),
                ("flow_iters", ctypes.c_int32), ("train_steps", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("ncall", ctypes.c_int64), ("train_samples", ctypes.c_int64),
                ("seed", ctypes.c_uint64)]


class FlowReport(ctypes.Structure):
    _fields_ = [("vegas", Result), ("flow", Result), ("vegas_var_per_sample", ctypes.c_double),
                ("flow_var_per_sample", ctypes.c_double), ("train_loss_first", ctypes.c_double),
                ("train_loss_last", ctypes.c_double), ("seconds_vegas", ctypes.c_double),
                ("seconds_train", ctypes.c_double), ("seconds_flow", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmcubes.so is not built ({LIB_PATH}); run "
                          "`python -m paper_2302_05730_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, u32, u64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "mcubes_stratify": (i32, [i32, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "mcubes_integrate": (i32, [i32, dp, i32, i64, i32, i32, u64, ctypes.POINTER(Result)]),
        "mcubes_integrate_ex": (i32, [i32, dp, i32, i64, i32, i32, u64, i32, ctypes.POINTER(Tuning), vp,
                                      dp, dp, dp, ctypes.POINTER(Result)]),
        "mcubes_vsample_once": (i32, [i32, dp, i32, i64, u64, i32, u32, i32, i32, dp, dp, dp, dp, dp]),
        "mcubes_integrate_range": (i32, [i32, dp, i32, i64, i32, i32, i32, i32, u64, i32, dp, dbl, dp, dp, vp]),
        "mcubes_combine": (i32, [dp, i32, i32, ctypes.POINTER(Result)]),
        "mcubes_vsample_dev": (i32, [i32, dp, i32, i64, u64, i32, u32, i32, i32, vp, vp, vp, vp, vp, i32,
                                     ctypes.POINTER(Tuning), vp]),
        "mcubes_rebin_dev": (i32, [i32, vp, vp, vp, vp]),
        "mcubes_workspace_bytes": (ctypes.c_size_t, [i32]),
        "mcubes_iteration_dev": (i32, [i32, dp, i32, i64, u64, i32, u32, i32, i32, vp, vp, vp, vp, vp,
                                       ctypes.c_size_t, ctypes.POINTER(Tuning), vp]),
        "mcubes_iteration_dev_static": (i32, [i32, dp, i32, i64, u64, i32, u32, i32, i32, vp, vp, vp, vp,
                                              ctypes.POINTER(Tuning), vp]),
        "mcubes_static_scratch_bytes": (ctypes.c_size_t, []),
        "mcubes_integrate_batch": (i32, [i32, ctypes.POINTER(Job), i32, i32, i32, ctypes.POINTER(BatchTuning), vp,
                                         ctypes.POINTER(Result), dp]),
        "mcubes_tune_batch": (i32, [i32, ctypes.POINTER(Job), i32, ctypes.POINTER(BatchTuning)]),
        "mcubes_flow_param_count": (i64, [ctypes.POINTER(FlowShape)]),
        "mcubes_flow_work_bytes": (ctypes.c_size_t, [ctypes.POINTER(FlowShape), i64]),
        "mcubes_flow_forward_dev": (i32, [ctypes.POINTER(FlowShape), vp, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]),
        "mcubes_flow_inverse_dev": (i32, [ctypes.POINTER(FlowShape), vp, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]),
        "mcubes_flow_grad_dev": (i32, [ctypes.POINTER(FlowShape), vp, i64, vp, vp, i32, vp, vp, vp, ctypes.c_size_t,
                                       vp]),
        "mcubes_flow_adam_dev": (i32, [i64, vp, vp, vp, vp, i32, ctypes.c_float, vp]),
        "mcubes_flow_integrate": (i32, [i32, dp, i32, ctypes.POINTER(FlowConfig), vp, ctypes.POINTER(FlowReport)]),
        "mcubes_pagani_rule_points": (i32, [i32]),
        "mcubes_pagani_evaluate_dev": (i32, [i32, dp, i32, i64, vp, vp, vp, vp, vp, vp]),
        "mcubes_pagani_integrate": (i32, [i32, dp, i32, dbl, i32, i64, i32, ctypes.POINTER(PaganiResult)]),
        "mcubes_flow_sample_work_bytes": (ctypes.c_size_t, [ctypes.POINTER(FlowShape)]),
        "mcubes_flow_sample_dev": (i32, [ctypes.POINTER(FlowShape), vp, i32, dp, i64, u64, i32, u32, i64, i64, vp, vp,
                                         vp, dp, vp, ctypes.c_size_t, vp]),
        "mcubes_philox_dev": (i32, [vp, u64, u64, i32, vp, vp]),
        "mcubes_status_string": (ctypes.c_char_p, [i32]),
        "mcubes_last_cuda_error": (i32, []),
        "mcubes_shutdown": (None, []),
        "mcubes_checked_violations": (i64, [i32, ctypes.POINTER(i64)]),
        "mcubes_unit_rates": (i32, [dp, i32]),
        "mcubes_fail_alloc": (i64, [i64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


_lib = None
_lib = _load()


def header_functions() -> list[str]:
    """Names of the functions include/mcubes.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcubes_[a-z0-9_]+)\s*\(", text)))


def lib():
    return _lib


# ------------------------------------------------------------------------------ marshalling
def _dptr(x):
    """Address of a device buffer: torch tensor, int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return x.data_ptr()
    raise TypeError(type(x))


CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy


def _stream(s):
    """cudaStream_t for a torch stream / raw handle. None selects the library's own stream; a
    torch stream whose handle is 0 (the legacy default stream) maps to cudaStreamLegacy."""
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or CUDA_STREAM_LEGACY
    raise TypeError(type(s))


def _hd(a):
    """Contiguous float64 host array and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def param_len(fid: int, d: int) -> int:
    """FP64 parameters integrand fid takes at dimension d."""
    return d * d + d if int(fid) == 9 else 2 * d


def _par(fid, d, params):
    """Integrand parameters as contiguous float64, checked for length (the C side reads
    param_len(fid, d) values)."""
    a, p = _hd(params)
    if 0 <= int(fid) <= 9 and 1 <= int(d) <= DMAX and a.size < param_len(fid, d):
        raise ValueError(f"integrand {fid} at d={d} takes {param_len(fid, d)} parameters, got {a.size}")
    return a, p


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tune(tune):
    if tune is None:
        return None
    if isinstance(tune, Tuning):
        return ctypes.byref(tune)
    t = Tuning()
    t.block_threads = int(tune.get("block_threads", 0))
    t.blocks_per_sm = int(tune.get("blocks_per_sm", 0))
    t.fp64_plain = int(tune.get("fp64_plain", 0))
    return ctypes.byref(t)


def _check(st, where):
    if st != OK:
        raise McubesError(st, where)


# ------------------------------------------------------------------------------ calls
def stratify(d: int, ncall: int):
    g, m, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.mcubes_stratify(d, ncall, ctypes.byref(g), ctypes.byref(m), ctypes.byref(p)), "stratify")
    return g.value, m.value, p.value


def integrate(fid, params, d, ncall, itmax, iter_adjust, seed, precision=FP64, tune=None, stream=None,
              grid_in=None, return_iters=False, return_grid=False):
    """Whole m-Cubes integration. Returns dict(estimate, error, chi2_dof, iters_done,
    samples_per_iter[, iters (itmax x 2: I, Var)][, grid (d x 501)])."""
    par, pp = _par(fid, d, params)
    res = Result()
    iters = np.zeros((itmax, 2)) if return_iters else None
    grid = np.zeros((d, NBINS + 1)) if return_grid else None
    gin = None
    if grid_in is not None:
        gin, gp = _hd(grid_in)
    st = _lib.mcubes_integrate_ex(int(fid), pp, d, int(ncall), itmax, iter_adjust, int(seed) & (2 ** 64 - 1),
                                  precision, _tune(tune), _stream(stream), _hptr(iters),
                                  None if gin is None else gp, _hptr(grid), ctypes.byref(res))
    _check(st, "integrate")
    out = dict(estimate=res.estimate, error=res.error, chi2_dof=res.chi2_dof, iters_done=res.iters_done,
               samples_per_iter=res.samples_per_iter)
    if iters is not None:
        out["iters"] = iters
    if grid is not None:
        out["grid"] = grid
    return out


def integrate_range(fid, params, d, ncall, itmax, iter_adjust, it_begin, it_end, seed, precision=FP64,
                    grid_in=None, prev_estimate=0.0, stream=None):
    """Iterations [it_begin, it_end) of an itmax-iteration run (checkpoint / resume). Returns
    dict(iters (n x 2), grid (d x 501))."""
    par, pp = _par(fid, d, params)
    gin = gp = None
    if grid_in is not None:
        gin, gp = _hd(grid_in)
    n = it_end - it_begin
    iters = np.zeros((max(n, 1), 2))
    grid = np.zeros((d, NBINS + 1))
    st = _lib.mcubes_integrate_range(int(fid), pp, d, int(ncall), itmax, iter_adjust, it_begin, it_end,
                                     int(seed) & (2 ** 64 - 1), precision, gp, float(prev_estimate), _hptr(grid),
                                     _hptr(iters), _stream(stream))
    _check(st, "integrate_range")
    return dict(iters=iters[:n], grid=grid)


def combine(iters, skip=0):
    """Inverse-variance combination of per-iteration (I, Var) pairs from index skip on."""
    it = np.ascontiguousarray(iters, dtype=np.float64).reshape(-1, 2)
    res = Result()
    _check(_lib.mcubes_combine(_hptr(it), it.shape[0], int(skip), ctypes.byref(res)), "combine")
    return dict(estimate=res.estimate, error=res.error, chi2_dof=res.chi2_dof, iters_done=res.iters_done)


def vsample_once(fid, params, d, ncall, seed, iteration=0, job=0, adjust=1, precision=FP64,
                 grid_in=None, want_grid=True, want_C=True):
    """One V-Sample pass (+ Rebin when adjust) with host buffers. Returns dict(I, Var[, C][, grid])."""
    par, pp = _par(fid, d, params)
    gin = gp = None
    if grid_in is not None:
        gin, gp = _hd(grid_in)
    grid = np.zeros((d, NBINS + 1)) if (adjust and want_grid) else None
    C = np.zeros((d, NBINS)) if (adjust and want_C) else None
    I = ctypes.c_double()
    V = ctypes.c_double()
    st = _lib.mcubes_vsample_once(int(fid), pp, d, int(ncall), int(seed) & (2 ** 64 - 1), iteration, job,
                                  int(adjust), precision, gp, _hptr(grid), _hptr(C), ctypes.byref(I), ctypes.byref(V))
    _check(st, "vsample_once")
    out = dict(I=I.value, Var=V.value)
    if grid is not None:
        out["grid"] = grid
    if C is not None:
        out["C"] = C
    return out


def vsample_dev(fid, params, d, ncall, seed, iteration, job, adjust, precision, d_grid, d_C, d_sums,
                d_prev=None, d_probe=None, probe_shift=0, tune=None, stream=None):
    par, pp = _par(fid, d, params)
    st = _lib.mcubes_vsample_dev(int(fid), pp, d, int(ncall), int(seed) & (2 ** 64 - 1), iteration, job,
                                 int(adjust), precision, _dptr(d_grid), _dptr(d_C), _dptr(d_sums), _dptr(d_prev),
                                 _dptr(d_probe), probe_shift, _tune(tune), _stream(stream))
    _check(st, "vsample_dev")


def rebin_dev(d, d_grid_in, d_C, d_grid_out, stream=None):
    _check(_lib.mcubes_rebin_dev(d, _dptr(d_grid_in), _dptr(d_C), _dptr(d_grid_out), _stream(stream)), "rebin_dev")


def workspace_bytes(d: int) -> int:
    return int(_lib.mcubes_workspace_bytes(d))


def iteration_dev(fid, params, d, ncall, seed, iteration, job, adjust, precision, d_grid_in, d_grid_out,
                  d_result, d_prev=None, d_workspace=None, workspace_bytes=0, tune=None, stream=None):
    par, pp = _par(fid, d, params)
    st = _lib.mcubes_iteration_dev(int(fid), pp, d, int(ncall), int(seed) & (2 ** 64 - 1), iteration, job,
                                   int(adjust), precision, _dptr(d_grid_in), _dptr(d_grid_out), _dptr(d_result),
                                   _dptr(d_prev), _dptr(d_workspace), int(workspace_bytes), _tune(tune),
                                   _stream(stream))
    _check(st, "iteration_dev")


def iteration_dev_static(fid, params, d, ncall, seed, iteration, job, adjust, precision, d_grid_in,
                         d_grid_out, d_result, d_prev=None, tune=None, stream=None):
    """mcubes_iteration_dev with the library's fixed scratch array: the call allocates no device
    memory, for callers that cannot allocate at that point. Calls that overlap on the GPU share,
    and race on, that one array."""
    par, pp = _par(fid, d, params)
    st = _lib.mcubes_iteration_dev_static(int(fid), pp, d, int(ncall), int(seed) & (2 ** 64 - 1), iteration, job,
                                          int(adjust), precision, _dptr(d_grid_in), _dptr(d_grid_out),
                                          _dptr(d_result), _dptr(d_prev), _tune(tune), _stream(stream))
    _check(st, "iteration_dev_static")


def static_scratch_bytes() -> int:
    return int(_lib.mcubes_static_scratch_bytes())


def _jobs(jobs):
    """ctypes job array from dicts (fid, d, ncall, params, seed); keeps the parameter arrays alive."""
    keep = []
    arr = (Job * len(jobs))()
    for k, j in enumerate(jobs):
        par, _ = _par(j["fid"], j["d"], j["params"])
        keep.append(par)
        arr[k].integrand_id = int(j["fid"])
        arr[k].d = int(j["d"])
        arr[k].ncall = int(j["ncall"])
        arr[k].params = par.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[k].seed = int(j.get("seed", 0)) & (2 ** 64 - 1)
    return arr, keep


def integrate_batch(jobs, itmax, iter_adjust, precision=FP64, tune=None, stream=None, return_iters=False,
                    raise_on_error=True):
    """Many independent integrations in one graph launch. jobs: list of dicts with fid, d, ncall,
    params, seed. Returns a list of result dicts (and the itmax x 2 per-iteration arrays)."""
    arr, keep = _jobs(jobs)
    n = len(jobs)
    res = (Result * n)()
    iters = np.zeros((n, itmax, 2)) if return_iters else None
    st = _lib.mcubes_integrate_batch(n, arr, itmax, iter_adjust, precision,
                                     None if tune is None else ctypes.byref(tune), _stream(stream), res,
                                     _hptr(iters))
    if st != OK and (raise_on_error or st != 6):
        raise McubesError(st, "integrate_batch")
    out = [dict(estimate=r.estimate, error=r.error, chi2_dof=r.chi2_dof, iters_done=r.iters_done,
                samples_per_iter=r.samples_per_iter, status=r.status) for r in res]
    if iters is not None:
        for k in range(n):
            out[k]["iters"] = iters[k]
    return out


def tune_batch(jobs, precision=FP64) -> BatchTuning:
    """Autotune the batched kernel's launch shape per dimension on these jobs."""
    arr, keep = _jobs(jobs)
    t = BatchTuning()
    _check(_lib.mcubes_tune_batch(len(jobs), arr, precision, ctypes.byref(t)), "tune_batch")
    return t


def flow_shape(d, layers, hidden, bins) -> FlowShape:
    return FlowShape(int(d), int(layers), int(hidden), int(bins))


def flow_param_count(shape: FlowShape) -> int:
    return int(_lib.mcubes_flow_param_count(ctypes.byref(shape)))


def flow_work_bytes(shape: FlowShape, n: int) -> int:
    return int(_lib.mcubes_flow_work_bytes(ctypes.byref(shape), int(n)))


def flow_forward_dev(shape, d_params, n, d_x, d_z, d_logq, d_work, work_bytes, stream=None):
    _check(_lib.mcubes_flow_forward_dev(ctypes.byref(shape), _dptr(d_params), int(n), _dptr(d_x), _dptr(d_z),
                                        _dptr(d_logq), _dptr(d_work), int(work_bytes), _stream(stream)), "flow_forward")


def flow_inverse_dev(shape, d_params, n, d_z, d_x, d_logq, d_work, work_bytes, stream=None):
    _check(_lib.mcubes_flow_inverse_dev(ctypes.byref(shape), _dptr(d_params), int(n), _dptr(d_z), _dptr(d_x),
                                        _dptr(d_logq), _dptr(d_work), int(work_bytes), _stream(stream)), "flow_inverse")


def pagani_rule_points(d: int) -> int:
    return int(_lib.mcubes_pagani_rule_points(int(d)))


def pagani_evaluate_dev(fid, params, d, n, d_lo, d_len, d_I, d_E, d_axis, stream=None):
    """The PAGANI kernel on n device regions (lo, len: n x d FP64) -> I, E (FP64), axis (int32)."""
    par, pp = _par(fid, d, params)
    _check(_lib.mcubes_pagani_evaluate_dev(int(fid), pp, int(d), int(n), _dptr(d_lo), _dptr(d_len), _dptr(d_I),
                                           _dptr(d_E), _dptr(d_axis), _stream(stream)), "pagani_evaluate")


def pagani_integrate(fid, params, d, rel_tol, max_iters=40, max_regions=1 << 22, init_split=2):
    """Adaptive PAGANI run: dict(estimate, error, regions_evaluated, iterations, status, active_regions)."""
    par, pp = _par(fid, d, params)
    r = PaganiResult()
    _check(_lib.mcubes_pagani_integrate(int(fid), pp, int(d), float(rel_tol), int(max_iters), int(max_regions),
                                        int(init_split), ctypes.byref(r)), "pagani_integrate")
    return dict(estimate=r.estimate, error=r.error, regions_evaluated=r.regions_evaluated, iterations=r.iterations,
                status=r.status, active_regions=r.active_regions)


def flow_sample_work_bytes(shape: FlowShape) -> int:
    return int(_lib.mcubes_flow_sample_work_bytes(ctypes.byref(shape)))


def flow_sample_dev(shape, d_params, fid, params, ncall, seed, iteration, job, i0, n, d_w, d_work, work_bytes,
                    d_x=None, d_logq=None, stream=None) -> float:
    """Fused flow-proposal sampling of samples [i0, i0 + n) of one iteration; returns the
    integrand's FP32 scale F (d_w holds (f / F) / q)."""
    par, pp = _par(fid, shape.d, params)
    F = ctypes.c_double(0.0)
    _check(_lib.mcubes_flow_sample_dev(ctypes.byref(shape), _dptr(d_params), int(fid), pp, int(ncall),
                                       int(seed) & (2 ** 64 - 1), int(iteration), int(job) & 0xFFFFFFFF, int(i0),
                                       int(n), _dptr(d_x), _dptr(d_logq), _dptr(d_w), ctypes.byref(F),
                                       _dptr(d_work), int(work_bytes), _stream(stream)), "flow_sample")
    return F.value


def flow_grad_dev(shape, d_params, n, d_x, d_w, loss_kind, d_grad, d_loss, d_work, work_bytes, stream=None):
    _check(_lib.mcubes_flow_grad_dev(ctypes.byref(shape), _dptr(d_params), int(n), _dptr(d_x), _dptr(d_w),
                                     int(loss_kind), _dptr(d_grad), _dptr(d_loss), _dptr(d_work), int(work_bytes),
                                     _stream(stream)), "flow_grad")


def flow_adam_dev(n_params, d_params, d_grad, d_m, d_v, step, lr, stream=None):
    _check(_lib.mcubes_flow_adam_dev(int(n_params), _dptr(d_params), _dptr(d_grad), _dptr(d_m), _dptr(d_v),
                                     int(step), float(lr), _stream(stream)), "flow_adam")


def _res(r):
    return dict(estimate=r.estimate, error=r.error, chi2_dof=r.chi2_dof, iters_done=r.iters_done,
                samples_per_iter=r.samples_per_iter)


def flow_integrate(fid, params, d, layers=4, hidden=64, bins=16, loss="kl", vegas_iters=5, flow_iters=5,
                   train_steps=1000, batch=1 << 14, lr=5e-4, ncall=10 ** 6, train_samples=1 << 20, seed=0,
                   return_params=False):
    """m-Cubes with the learned proposal (VEGAS warm-up, training, flow-sampled iterations).
    Returns dict(vegas, flow (results), vegas_var_per_sample, flow_var_per_sample, train_loss_first,
    train_loss_last, seconds_*[, params])."""
    par, pp = _par(fid, d, params)
    cfg = FlowConfig(FlowShape(d, layers, hidden, bins), 0 if loss == "variance" else 1, vegas_iters, flow_iters,
                     train_steps, batch, lr, int(ncall), int(train_samples), int(seed) & (2 ** 64 - 1))
    rep = FlowReport()
    out_par = None
    if return_params:
        out_par = np.zeros(flow_param_count(cfg.shape), dtype=np.float32)
    st = _lib.mcubes_flow_integrate(int(fid), pp, d, ctypes.byref(cfg),
                                    None if out_par is None else out_par.ctypes.data, ctypes.byref(rep))
    _check(st, "flow_integrate")
    out = dict(vegas=_res(rep.vegas), flow=_res(rep.flow), vegas_var_per_sample=rep.vegas_var_per_sample,
               flow_var_per_sample=rep.flow_var_per_sample, train_loss_first=rep.train_loss_first,
               train_loss_last=rep.train_loss_last, seconds_vegas=rep.seconds_vegas,
               seconds_train=rep.seconds_train, seconds_flow=rep.seconds_flow)
    if out_par is not None:
        out["params"] = out_par
    return out


def philox_dev(d_ctr, n, seed, impl, d_out, stream=None):
    _check(_lib.mcubes_philox_dev(_dptr(d_ctr), int(n), int(seed) & (2 ** 64 - 1), impl, _dptr(d_out),
                                  _stream(stream)), "philox_dev")


def status_string(status: int) -> str:
    return _lib.mcubes_status_string(status).decode()


def last_cuda_error() -> int:
    return int(_lib.mcubes_last_cuda_error())


def shutdown() -> None:
    _lib.mcubes_shutdown()


def checked_violations(reset: bool = True):
    """(failed index checks since the last reset, first failure's site << 48 | index) of a
    bounds-checked build; None from a normal build."""
    first = ctypes.c_int64(0)
    n = int(_lib.mcubes_checked_violations(1 if reset else 0, ctypes.byref(first)))
    return None if n < 0 else (n, int(first.value))


UNIT_RATE_NAMES = ("ffma_lanes", "dfma_lanes", "exp2f_lanes", "philox_calls", "shared_gather8_lanes",
                   "shared_atomic_f32_lanes", "shared_atomic_u32x8_lanes", "shared_red_u64_lanes",
                   "shared_red_u64x4_lanes", "shared_red_u32x8_lanes", "l1_gather8_lanes",
                   "mixed_gather8_lanes")


def unit_rates() -> dict:
    """Per-SM, per-clock throughput of the V-Sample building blocks on the current device."""
    out = np.zeros(len(UNIT_RATE_NAMES))
    _check(_lib.mcubes_unit_rates(_hptr(out), len(out)), "unit_rates")
    return dict(zip(UNIT_RATE_NAMES, (float(v) for v in out)))


def fail_alloc(n: int) -> int:
    """Arm the allocation fault hook: the n-th allocation the library makes from now fails as if
    out of memory (0 disarms). Returns the number of allocations made so far."""
    return int(_lib.mcubes_fail_alloc(int(n)))
