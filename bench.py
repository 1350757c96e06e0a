"""Benchmark of the m-Cubes hot path (V-Sample + Rebin) on GB300.

Headline workload: the six Genz families at d = 8 with 1e8 samples per iteration (g = 9, m = 9^8
sub-cubes, p = 2), a_i ~ U[5, 15], u_i ~ U[0.2, 0.8] (seed 0), in plain FP64 (the paper's
precision). One step = one whole m-Cubes integration of every family from the uniform grid: 10
iterations, the first 5 adjusting (V-Sample with bin contributions, then Rebin), the rest frozen,
with every iteration's sums read back to the host and combined.

Output: every secondary leg first, one JSON line each ({"leg": name, ...}); the last line is the
compact headline (plain FP64 samples/s with its roofline, the end-to-end rate through the host
call, the oracle on the host cores, the clocks, and the FP32-eval variant's own rate and roofline).
The legs:
  estimates   each family's FP64 and FP32-eval estimate against its closed form
  pipes       unit-rate microbenchmarks and the FP32-eval V-Sample's pipe-level bounds
  config2     d = 5 and 6 at 1e8 samples per iteration, both precisions: samples/s, V-Sample
              launch times and true errors per family
  tta         time to a relative error of 1e-3 (sigma / |I| <= 1e-3, with the true error beside it)
              at 1e6, 1e7 and 1e8 samples per iteration, both precisions
  paper       the paper's own fixed-parameter f1..f6 at d = 8 (context for its per-family timings)
  config5     d = 10 product peak and C0 at 1e9 samples per iteration, 20 iterations, both
              precisions; and the learned proposal (6 layers, width 128) at d = 10
  batch       4096 independent Gaussian integrations in one graph launch
  train_step  one training step of the flow per shape and kernel path (tcgen05, mma.sync, per layer)
  learned     the learned proposal at d = 8 (double and rotated Gaussians)
  pagani      the paper's other workload (off unless --pagani)

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--headline-only]

Under torchrun (N > 1) every rank runs an independent replica (its own Philox job id): the method
has no exchange step, so there is no collective on the data path. `value` is the samples of all
ranks over the slowest rank's time.

`--impl reference` times the CPU oracle (plain C, FP64, threads over sub-cube ranges on every
host core) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D = 8
NCALL = 10 ** 8
ITMAX, ADJ = 10, 5   # one m-Cubes integration: 10 iterations, the first 5 adjust the grid
WORKLOAD = "genz6-d8-n1e8-fp64"
# the headline metric as named for this workload: samples/s is the value; the times to a relative
# error of 1e-3 (plain, FP32-eval, learned) are in the tta, config5 and learned legs
METRIC = "m-Cubes samples/s; time to 1e-3 rel err, plain vs learned/FP32 (1 GB300)"
# DRAM bytes (read + write) per vsample_fast64_kernel<8, fid, HK> launch at d = 8, 1e8 samples per
# iteration: the mean over one timed step's 30 adjusting and 30 frozen launches (six families), from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as it stands; None
# where the kernel changed after the capture.
VSAMPLE64_DRAM_BYTES_BY_KIND = {"adjusting": 370039, "frozen": 223061}
NB = 500
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# GB300 unit counts: 152 SMs; 4 SM sub-partitions x 32 lanes issue one instruction per clock;
# dense FP64 at 1.25 TFLOP/s nominal is 2 FP64 FMA lanes per SM per clock at the 2070 MHz maximum.
SMS = 152
LANES_PER_SM = 128
FP64_LANES_PER_SM = 2
FALLBACK_SM_MHZ = 2070.0


# ------------------------------------------------------------------------------ operation counts
# FP64 operations per sample of the FP64 V-Sample's formulation for the six Genz families (the
# kernel with integer c + u, an integer (c + u) R rounded as FP64 rounds it, integer bin extraction
# and folded per-bin tables): per axis the Jacobian's product (not for the families closed by exp:
# Gaussian, C0 and discontinuous, whose Jacobian joins the exponent through integer sums of the bins'
# exponents and fixed-point ln m_k) and the family's terms -- one fma of the folded table entries and
# its accumulation for the Gaussian and C0 (an fma, an add), three for the product peak (fma, fma,
# product), one fma into the sum for the families that only need sum a x (their constant parts
# summed as fixed-point integers, converted and added once a sample: 2; the Gaussian and C0 convert
# and add their ln m_k sum the same way); per sample the family's closing function at the FP64
# operations of its table-driven evaluation (exp 7, cos 11, a reciprocal 5, the corner peak's 1 + s
# and ninth power 5 + a reciprocal), w = f J where J is a product, and the two sub-cube sums; per
# sub-cube the mean, the variance (fma, clamp) and the two thread sums; on adjusting iterations the
# contribution (w F)^2 (2). The d bin additions of an adjusting sample are FP64 reductions the L2
# performs and compare-and-swap loops on the block's shared copy, not counted. Counted from the
# formulation, not from compiled code.
FP64_AXIS_TERMS = {0: 1, 1: 3, 2: 1, 3: 2, 4: 2, 5: 1}
FP64_FINISH = {0: 13, 1: 5, 2: 12, 3: 9, 4: 9, 5: 9}
FP64_JACOBIAN_IN_EXP = {0: False, 1: False, 2: False, 3: True, 4: True, 5: True}


def fp64_ops_per_sample(fid: int, d: int, adjust: bool, p: int = 2) -> float:
    jac = 0 if FP64_JACOBIAN_IN_EXP[fid] else 1
    return d * (jac + FP64_AXIS_TERMS[fid]) + FP64_FINISH[fid] + 2 + jac + 5.0 / p + (2 if adjust else 0)


def algorithmic_ops_per_sample(fid: int, d: int, adjust: bool, f32: bool) -> float:
    """Minimal per-sample instruction count of the V-Sample algorithm (FP32-eval path, thread
    lanes). Each entry is an operation the algorithm needs, not a count of compiled code."""
    philox = math.ceil(d / 4) * 10 * 4          # 10 rounds x (2 wide multiplies + 2 three-way xors)
    per_dim_map = 9 + (1 if adjust else 0)      # bits->u, +c, xR, cap, floor, delta, load, fma, xJ, [atomic]
    integrand_dim = {0: 1, 1: 4, 2: 1, 3: 3, 4: 3, 5: 3, 6: 1, 7: 0}[fid]
    finish = {0: 4, 1: 1, 2: 5, 3: 1, 4: 1, 5: 2, 6: 0, 7: 0}[fid]
    per_sample = 1 + 3 + (2 if adjust else 0) + math.ceil(d / 4)   # w = fJ, stats, hist value, J rescale
    return philox + d * (per_dim_map + integrand_dim) + finish + per_sample


def sm_peak_ops(sm_mhz: float) -> float:
    return SMS * LANES_PER_SM * sm_mhz * 1e6


def fp64_peak_ops(sm_mhz: float) -> float:
    return SMS * FP64_LANES_PER_SM * sm_mhz * 1e6


PHILOX_PRODUCTS_PER_CALL = 20      # two 32 x 32 -> 64-bit products a round, ten rounds
PHILOX_PRODUCTS_PER_DRAW = 17      # the sampler's hoisted form: rounds 2-9 and one product of round 1
PHILOX_PRODUCTS_PER_CUBE = 2       # ... plus round 0's and round 1's products of the sub-cube index


def pipe_bounds(rates: dict, fams, d: int, kinds: dict, sm_mhz: float, p: int = 2) -> dict:
    """Pipe-level roofline of the FP32-eval V-Sample kernels: per launch kind, the SM clocks a
    sample needs on each pipe at the measured unit rates (mcubes_unit_rates) -- Philox's 64-bit
    integer products (17 a draw plus 2 a sub-cube of p samples, at 20 a measured Philox call), the
    shared-memory pipe (table gathers, plus the histogram's u32 atomics when adjusting: both use
    it) and instruction issue of the algorithmic operations -- their maximum (the bound, every pipe
    overlapped), and the measured clocks a sample against it."""
    out = {}
    products = math.ceil(d / 4) * PHILOX_PRODUCTS_PER_DRAW + PHILOX_PRODUCTS_PER_CUBE / p
    for name, adj in (("adjusting", True), ("frozen", False)):
        ops = float(np.mean([algorithmic_ops_per_sample(f, d, adj, True) for f in fams]))
        t = {"philox": products / (PHILOX_PRODUCTS_PER_CALL * rates["philox_calls"]),
             "shared_memory": d / rates["shared_gather8_lanes"] +
             (d / rates["shared_atomic_u32x8_lanes"] if adj else 0.0),
             "issue": ops / LANES_PER_SM}
        bound = max(t.values())
        measured = SMS * sm_mhz * 1e6 / kinds[name]["samples_per_s"]
        out[name] = {"clk_per_sample_by_pipe": t, "bound_clk_per_sample": bound,
                     "binding_pipe": max(t, key=t.get), "measured_clk_per_sample": measured,
                     "frac_of_pipe_bound": bound / measured}
    return out


def launch_ms_by_family(kern_ev, fams, names) -> dict:
    """Mean CUDA-event time of one V-Sample launch per family and kind, over the timed steps."""
    out = {}
    for f in fams:
        row = {}
        for name, adj in (("adjusting", True), ("frozen", False)):
            ts = [e0.elapsed_time(e1) for (fid, a_, e0, e1) in kern_ev if fid == f and a_ == adj]
            row[name] = round(float(np.mean(ts)), 4) if ts else None
        out[names[f]] = row
    return out


def kind_roofline(kern_ev, samples: int, d: int, ops_fn, peak: float, p: int) -> dict:
    """Per launch kind (adjusting, frozen) and over all V-Sample launches of a timed region: the
    launches, their mean CUDA-event duration, samples/s, and algorithmic operations per second
    against `peak` (operations/s)."""
    out = {}
    tot_ops = tot_ms = 0.0
    for adj in (True, False):
        ev = [(fid, e0.elapsed_time(e1)) for (fid, a_, e0, e1) in kern_ev if a_ == adj]
        if not ev:
            continue
        ops = sum(ops_fn(fid, d, adj, p) * samples for fid, _ in ev)
        ms = sum(t for _, t in ev)
        tot_ops += ops
        tot_ms += ms
        out["adjusting" if adj else "frozen"] = {
            "launches": len(ev), "avg_launch_ms": ms / len(ev), "samples_per_s": samples * len(ev) / (ms * 1e-3),
            "achieved": ops / (ms * 1e-3) / 1e12, "frac": ops / (ms * 1e-3) / peak}
    n = len(kern_ev)
    return {"by_kind": out, "achieved": tot_ops / (tot_ms * 1e-3) / 1e12, "frac": tot_ops / (tot_ms * 1e-3) / peak,
            "avg_launch_ms": tot_ms / max(n, 1), "ops_per_launch": tot_ops / max(n, 1)}


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        """Samples `nvidia-smi` every 50 ms into `path` (default: a file in the system temp directory);
        stop() summarises the samples for the bench line."""
        self.gpu = gpu_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"mcubes_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (identity without torch.distributed)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_job(rank: int) -> int:
    """Philox job id (counter word 3) of a replica: every rank draws an independent stream."""
    return rank


def emit(leg: str, obj) -> None:
    """One secondary leg as its own JSON line (before the headline line)."""
    print(json.dumps({"leg": leg, **obj}), flush=True)


# ------------------------------------------------------------------------------ oracle timing
def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_vsample_ranges(fams, pars, grids, ncall, starts, cubes, threads, it=1, mode=0):
    """The oracle's V-Sample (adjusting, point layout of `mode`) over [t0, t0 + cubes) of each
    family, split into `threads` equal sub-ranges run side by side (the oracle holds no global state
    and ctypes releases the interpreter lock during the call). Returns the samples processed."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    g, m, p = oracle.stratify(D, ncall)
    jobs = []
    for fid in fams:
        t0 = starts[fid]
        step = -(-cubes // threads)
        for a in range(t0, t0 + cubes, step):
            jobs.append((fid, a, min(a + step, t0 + cubes)))

    def one(job):
        fid, a, b = job
        oracle.vsample(fid, D, pars[fid], ncall, 0, it=it, mode=mode, adjust=1, B=grids[fid], t0=a, t1=b)
        return (b - a) * p

    if threads == 1:
        return sum(one(j) for j in jobs)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return sum(ex.map(one, jobs))


# ------------------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    """The CPU oracle (FP64) on a bounded sample of the workload (sub-cube ranges of each family)."""
    if rank != 0:
        return
    import oracle
    from paper_2302_05730_gb300 import workloads as W

    g, m, p = oracle.stratify(D, NCALL)
    threads = host_threads()
    cubes = (1 << 15) * threads
    B = oracle.uniform_grid(D)
    grids = {fid: B for fid in W.GENZ6}
    pars = {fid: W.genz_params(fid, D, seed=0) for fid in W.GENZ6}

    def step(k):
        starts = {fid: (k * 7919 * cubes) % (m - cubes) for fid in W.GENZ6}
        return oracle_vsample_ranges(W.GENZ6, pars, grids, NCALL, starts, cubes, threads, it=k % 65536, mode=0)

    for k in range(args.warmup):
        step(k)
    t = time.perf_counter()
    n = 0
    for k in range(args.steps):
        n += step(args.warmup + k)
    el = time.perf_counter() - t
    v = n / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "d": D, "ncall": NCALL,
                       "families": [W.NAMES[f] for f in W.GENZ6], "sample_cubes_per_family_step": cubes},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"{cubes} sub-cubes ({cubes * p} samples) of each of the 6 families per step, "
                                       f"FP64, {threads} threads over equal sub-cube ranges"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ the timed step
class Harness:
    """Whole m-Cubes integrations of a set of families on the device, launch by launch through the
    C ABI's device calls (mcubes_vsample_dev, mcubes_rebin_dev) on one stream, with every
    iteration's sums read back to the host once per step and combined there (mcubes_combine)."""

    def __init__(self, capi, torch, dev, stream, d, ncall, fams, pars, itmax, adj, job, dist):
        self.capi, self.torch, self.dev, self.stream = capi, torch, dev, stream
        self.d, self.ncall, self.fams, self.pars = d, ncall, list(fams), pars
        self.itmax, self.adj, self.job, self.dist = itmax, adj, job, dist
        self.g, self.m, self.p = capi.stratify(d, ncall)
        self.samples = self.m * self.p
        self.uni = torch.from_numpy(np.tile(np.arange(NB + 1, dtype=np.float64) / NB, (d, 1))).to(dev)
        nf = len(self.fams)
        self.sums = torch.zeros((nf, itmax, 2), dtype=torch.float64, device=dev)
        self.sums_host = torch.zeros((nf, itmax, 2), dtype=torch.float64).pin_memory()
        self.counter = 0
        self.launches = 0

    def fresh_state(self):
        t = self.torch
        return {fid: dict(grid=[self.uni.clone(), t.empty_like(self.uni)], cur=0,
                          C=t.zeros(self.d * NB, dtype=t.float64, device=self.dev)) for fid in self.fams}

    def step(self, state, prec, kernel_events=None):
        """One whole integration of each family (all hot-path rows): uniform grid, itmax V-Sample
        passes (the first adj accumulate bin contributions and rebin), the sums of every iteration to
        the host in one copy; the host combination follows the step."""
        capi, t = self.capi, self.torch
        seed = self.counter
        self.counter += 1
        self.sums.zero_()
        for f, fid in enumerate(self.fams):
            s = state[fid]
            s["grid"][0].copy_(self.uni)
            s["cur"] = 0
            for it in range(self.itmax):
                adjust = it < self.adj
                if adjust:
                    s["C"].zero_()
                gin, gout = s["grid"][s["cur"]], s["grid"][1 - s["cur"]]
                if kernel_events is not None:
                    e0 = t.cuda.Event(enable_timing=True)
                    e1 = t.cuda.Event(enable_timing=True)
                    e0.record(self.stream)
                capi.vsample_dev(fid, self.pars[fid], self.d, self.ncall, seed, it, self.job, int(adjust), prec, gin,
                                 s["C"] if adjust else None, self.sums[f, it], stream=self.stream)
                if kernel_events is not None:
                    e1.record(self.stream)
                    kernel_events.append((fid, adjust, e0, e1))
                self.launches += 1
                if adjust and it + 1 < self.itmax:
                    capi.rebin_dev(self.d, gin, s["C"], gout, stream=self.stream)
                    self.launches += 1
                    s["cur"] = 1 - s["cur"]
        self.sums_host.copy_(self.sums, non_blocking=True)

    def combine_all(self):
        out = {}
        m = float(self.m)
        for f, fid in enumerate(self.fams):
            it = self.sums_host[f].numpy().copy()
            it[:, 0] /= m
            it[:, 1] /= m * m
            out[fid] = self.capi.combine(it)
        return out

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        self.torch.cuda.synchronize(self.dev)

    def timed(self, prec, steps, warmup, kern=None, flush=None):
        """`warmup` untimed steps, then `steps` steps each bracketed by CUDA events on the stream
        (L2 flushed before each, outside the events). Returns (total ms over ranks, state, last
        step's combined results)."""
        t = self.torch
        state = self.fresh_state()
        with t.cuda.stream(self.stream):
            for _ in range(warmup):
                self.step(state, prec)
        self.barrier()
        self.launches = 0
        step_ms = []
        res = None
        for _ in range(steps):
            if flush is not None:
                flush.add_(1.0)   # evict L2 between timed steps (outside the timed events)
            t.cuda.synchronize(self.dev)
            a = t.cuda.Event(enable_timing=True)
            b = t.cuda.Event(enable_timing=True)
            a.record(self.stream)
            with t.cuda.stream(self.stream):
                self.step(state, prec, kern)
            b.record(self.stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            res = self.combine_all()
        self.barrier()
        total_ms = max_over_ranks(sum(step_ms), self.dist, self.dev)
        for fid in self.fams:   # sanity: the last step's estimates are finite
            assert math.isfinite(res[fid]["estimate"]) and math.isfinite(res[fid]["error"]), (fid, res[fid])
        return total_ms, state, res


def closed_form_fn():
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from closed_forms import exact
    return exact


def vs_exact(exact, fid, par, d, r):
    ex = exact(fid, par[:d], par[d:])
    return {"exact": ex, "true_rel_err": abs(r["estimate"] / ex - 1.0),
            "z": (r["estimate"] - ex) / max(r["error"], 1e-300)}


# ------------------------------------------------------------------------------ time to 1e-3
def time_to_target(capi, fid, par, d, ncall, prec, kmax, adjust, exact=None, target=1e-3):
    """Time to a relative error of `target`, one definition for every entry: the wall time of the
    shortest whole run (in iterations, the first min(k, adjust) adjusting) whose combined estimate
    has sigma <= target |I|, measured by running it again through mcubes_integrate_ex; beside it the
    true relative error |I - I_exact| / |I_exact| and z = (I - I_exact) / sigma. A run of k
    iterations equals the first k iterations of a longer run with the same seed (the draws are
    indexed by iteration and the grid only depends on earlier iterations), so the k is read off one
    run of kmax iterations."""
    r = capi.integrate(fid, par, d, ncall, kmax, min(kmax, adjust), 0, precision=prec, return_iters=True)
    iters = r["iters"]
    k_hit = None
    for k in range(1, kmax + 1):
        c = capi.combine(iters[:k])
        if c["error"] <= target * abs(c["estimate"]):
            k_hit = k
            break
    out = {"kmax": kmax}
    if k_hit is None:
        c = capi.combine(iters)
        out.update(reached=False, iters=kmax, rel_sigma=c["error"] / max(abs(c["estimate"]), 1e-300))
        res = c
    else:
        t0 = time.perf_counter()
        res = capi.integrate(fid, par, d, ncall, k_hit, min(k_hit, adjust), 0, precision=prec)
        el = time.perf_counter() - t0
        out.update(reached=True, iters=k_hit, seconds=el, rel_sigma=res["error"] / max(abs(res["estimate"]), 1e-300))
    if exact is not None:
        ex = exact(fid, par[:d], par[d:])
        out.update(true_rel_err=abs(res["estimate"] / ex - 1.0), z=(res["estimate"] - ex) / max(res["error"], 1e-300))
    return out


def tta_leg(capi, W, d, pars, exact):
    out = {}
    budgets = {10 ** 6: 60, 10 ** 7: 30, 10 ** 8: 12}
    for prec, name in ((capi.FP64, "fp64"), (capi.FP32_EVAL, "fp32_eval")):
        for nb, kmax in budgets.items():
            out[f"{name}_n{nb:.0e}"] = {W.NAMES[f]: time_to_target(capi, f, pars[f], d, nb, prec, kmax, ADJ, exact)
                                       for f in W.GENZ6}
    return {"d": d, "definition": "shortest whole run with sigma <= 1e-3 |I| (first min(k, 5) iterations "
                                  "adjusting), timed through mcubes_integrate_ex; true error beside it",
            "by_budget": out}


# ------------------------------------------------------------------------------ learned proposal
def learned_leg(capi, W, train_steps: int, n_it: int = 1 << 20, seeds=(0, 1, 2)):
    """Learned proposal (4-layer coupling flow, width 64, 16 bins, variance loss on f^2 J weights;
    2^20 samples per iteration) on the double Gaussian exp(-100|x - p1|^2) + exp(-100|x - p2|^2),
    p1 = 0.25 1, p2 = 0.75 1, and on a rotated anisotropic Gaussian (random orthogonal Q,
    eigenvalues 1..400), d = 8. Per training seed: the variance per sample against the adapted grid
    at the same budget; each method's estimate against the closed form (z-score, true relative
    error); and the time to a relative error of 1e-3 (sigma <= 1e-3 |I|) for the learned proposal,
    the FP32-eval grid and the plain FP64 grid: warm-up plus the iterations the measured
    per-iteration variance needs, with the true error beside it, or null when the method's
    estimate disagrees with the closed form (|z| > 4), since then more iterations shrink its error
    bar but not its error. Training differs from seed to seed, so the leg reports every seed and
    the medians."""
    exact = {}
    gold = os.path.join(ROOT, "tests", "golden", "learned_exact_d8.json")
    if os.path.exists(gold):
        g = json.load(open(gold))
        exact = {"double_gaussian": g["double_gaussian"], "rotated_gaussian": g["rotated_gaussian_seed0"]}

    def assess(name, est, err):
        if name not in exact:
            return {}
        z = (est - exact[name]) / max(err, 1e-300)
        return {"z": z, "rel_err": abs(est / exact[name] - 1.0), "consistent": abs(z) <= 4.0}

    out = {}
    cases = [("double_gaussian", W.DOUBLE_GAUSSIAN, W.double_gaussian_params(8)),
             ("rotated_gaussian", W.ROTATED_GAUSSIAN, W.rotated_gaussian_params(8, seed=0))]
    g8, m8, p8 = capi.stratify(8, n_it)
    ok = lambda j: j.get("consistent", True)
    for name, fid, par in cases:
        I = abs(exact.get(name, 1.0))
        target = (1e-3 * I) ** 2
        for prec in (capi.FP64, capi.FP32_EVAL):   # one untimed call of each precision (launch attributes)
            capi.integrate(fid, par, 8, n_it, 2, 1, 0, precision=prec)
        t0 = time.perf_counter()
        pl = capi.integrate(fid, par, 8, n_it, 9, 5, 0, precision=capi.FP64, return_iters=True)
        t64 = (time.perf_counter() - t0) / 9
        c64 = capi.combine(pl["iters"], skip=5)
        k64 = int(math.ceil(float(np.mean(pl["iters"][5:, 1])) / target))
        t0 = time.perf_counter()
        p32 = capi.integrate(fid, par, 8, n_it, 9, 5, 0, precision=capi.FP32_EVAL, return_iters=True)
        t32 = (time.perf_counter() - t0) / 9
        c32 = capi.combine(p32["iters"], skip=5)
        k32 = int(math.ceil(float(np.mean(p32["iters"][5:, 1])) / target))
        j32 = assess(name, c32["estimate"], c32["error"])
        j64 = assess(name, c64["estimate"], c64["error"])
        per_seed = []
        for seed in seeds:
            r = capi.flow_integrate(fid, par, 8, layers=4, hidden=64, bins=16, loss="variance", vegas_iters=5,
                                    flow_iters=4, train_steps=train_steps, batch=1 << 14, lr=1e-3, ncall=n_it,
                                    train_samples=1 << 20, seed=seed)
            k_flow = int(math.ceil(r["flow_var_per_sample"] / (m8 * p8) / target))
            jf = assess(name, r["flow"]["estimate"], r["flow"]["error"])
            jg = assess(name, r["vegas"]["estimate"], r["vegas"]["error"])
            per_seed.append({
                "seed": seed, "flow": dict(r["flow"], **jf), "grid_same_budget": dict(r["vegas"], **jg),
                "variance_gain_per_sample": r["vegas_var_per_sample"] / r["flow_var_per_sample"],
                "train_seconds": r["seconds_train"],
                "flow_samples_per_s": 4 * m8 * p8 / max(r["seconds_flow"], 1e-9),
                "time_to_1e-3_s": (r["seconds_vegas"] * 5 / 9 + r["seconds_train"] + k_flow * r["seconds_flow"] / 4)
                if ok(jf) else None,
                "iters_to_1e-3": k_flow})
        gains = [x["variance_gain_per_sample"] for x in per_seed]
        ttas = [x["time_to_1e-3_s"] for x in per_seed if x["time_to_1e-3_s"] is not None]
        out[name] = {
            "exact": exact.get(name), "train_steps": train_steps, "seeds": per_seed,
            "variance_gain_per_sample": {"median": float(np.median(gains)), "min": min(gains), "max": max(gains)},
            "flow_consistent_seeds": sum(1 for x in per_seed if ok(x["flow"])),
            "fp32_grid": dict(c32, **j32), "fp64_grid": dict(c64, **j64),
            "time_to_1e-3_s": {
                "learned_median": float(np.median(ttas)) if ttas else None,
                "fp32_grid": (5 + k32) * t32 if ok(j32) else None,
                "fp64_grid": (5 + k64) * t64 if ok(j64) else None,
                "iters": {"fp32_grid": k32, "fp64_grid": k64}},
        }
    return out


# ------------------------------------------------------------------------------ training step
def train_step_leg(capi, torch, steps: int = 20):
    """One training step (loss and gradient of a 2^14-sample batch, mcubes_flow_grad_dev) per flow
    shape and per kernel path: the tcgen05 kernels (the default where the shape fits them), the
    fused mma.sync kernels and the per-layer chain (MCUBES_FLOW_TRAIN); CUDA events on the
    launching stream after three warm-up steps. A path that does not take a shape falls back, so a
    timing equal to the next path's means the path does not fit."""
    out = {}
    n = 1 << 14
    for (d, L, H, K) in [(8, 4, 64, 16), (8, 4, 128, 16), (10, 6, 128, 16)]:
        shape = capi.flow_shape(d, L, H, K)
        npar = capi.flow_param_count(shape)
        rng = np.random.default_rng(1)
        p = torch.from_numpy(rng.normal(0, 0.1, npar).astype(np.float32)).cuda()
        x = torch.from_numpy(rng.uniform(0, 1, (n, d)).astype(np.float32)).cuda()
        w = torch.from_numpy((rng.exponential(1.0, n) / n).astype(np.float32)).cuda()
        nb = capi.flow_work_bytes(shape, n)
        buf = torch.empty(nb // 4 + 128, dtype=torch.float32, device="cuda")
        ws = (buf.data_ptr() + 255) // 256 * 256
        g = torch.zeros(npar, dtype=torch.float32, device="cuda")
        lo = torch.zeros(1, dtype=torch.float32, device="cuda")
        st = torch.cuda.current_stream()
        res = {}
        for path in ("tc", "mma", "chain"):
            os.environ.pop("MCUBES_FLOW_TRAIN", None)
            if path != "tc":
                os.environ["MCUBES_FLOW_TRAIN"] = path
            for _ in range(3):
                capi.flow_grad_dev(shape, p, n, x, w, 0, g, lo, ws, nb, stream=st)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(steps):
                capi.flow_grad_dev(shape, p, n, x, w, 0, g, lo, ws, nb, stream=st)
            b.record(st)
            b.synchronize()
            res[path] = a.elapsed_time(b) / steps
        os.environ.pop("MCUBES_FLOW_TRAIN", None)
        out[f"d{d}_L{L}_H{H}_K{K}"] = res
    return {"batch": n, "ms_per_step": out}


# ------------------------------------------------------------------------------ config 5
def config5_leg(capi, W, exact, flow_steps: int, with_flow: bool = True):
    """d = 10 product peak and C0 (a_i ~ U[5, 15], u_i ~ U[0.2, 0.8], seed 0) at 1e9 samples per
    iteration (g = 7, m = 7^10, p = 3), 20 iterations with the first 10 adjusting, FP32-eval and
    FP64: samples/s of the whole run through mcubes_integrate_ex, the estimate against the closed
    form, and the time to 1e-3 (sigma <= 1e-3 |I|, the tta definition). Then the learned proposal
    at d = 10 (6 coupling layers, width 128, 16 bins) trained on 2^22-sample batches of m-Cubes'
    own samples, on the same two integrands: variance gain per sample over the adapted grid and its
    time to 1e-3 against plain FP64."""
    d, n, itmax, adj = 10, 10 ** 9, 20, 10
    g, m, p = capi.stratify(d, n)
    out = {"d": d, "ncall": n, "m": m, "p": p, "iters": itmax, "iter_adjust": adj}
    for fid in (W.PRODUCT_PEAK, W.C0):
        par = W.genz_params(fid, d, seed=0)
        fam = {}
        for prec, name in ((capi.FP32_EVAL, "fp32_eval"), (capi.FP64, "fp64")):
            capi.integrate(fid, par, d, n, 1, 1, 0, precision=prec)          # warm-up
            t0 = time.perf_counter()
            r = capi.integrate(fid, par, d, n, itmax, adj, 0, precision=prec, return_iters=True)
            el = time.perf_counter() - t0
            k_hit = None
            for k in range(1, itmax + 1):
                c = capi.combine(r["iters"][:k])
                if c["error"] <= 1e-3 * abs(c["estimate"]):
                    k_hit = k
                    break
            tt = None
            if k_hit is not None:
                t0 = time.perf_counter()
                capi.integrate(fid, par, d, n, k_hit, min(k_hit, adj), 0, precision=prec)
                tt = time.perf_counter() - t0
            fam[name] = dict({"samples_per_s": m * p * itmax / el, "seconds": el, "estimate": r["estimate"],
                              "error": r["error"], "iters_to_1e-3": k_hit, "time_to_1e-3_s": tt},
                             **vs_exact(exact, fid, par, d, r))
        if with_flow:
            try:
                t0 = time.perf_counter()
                fr = capi.flow_integrate(fid, par, d, layers=6, hidden=128, bins=16, loss="variance", vegas_iters=5,
                                         flow_iters=4, train_steps=flow_steps, batch=1 << 14, lr=1e-3,
                                         ncall=1 << 22, train_samples=1 << 22, seed=0)
                el = time.perf_counter() - t0
                n_it = fr["flow"].get("samples_per_iter") or (1 << 22)
                ex = exact(fid, par[:d], par[d:])
                k_flow = int(math.ceil(fr["flow_var_per_sample"] / n_it / (1e-3 * ex) ** 2))
                fam["learned_w128_l6"] = {
                    "variance_gain_per_sample": fr["vegas_var_per_sample"] / fr["flow_var_per_sample"],
                    "estimate": fr["flow"]["estimate"], "error": fr["flow"]["error"],
                    "true_rel_err": abs(fr["flow"]["estimate"] / ex - 1.0),
                    "z": (fr["flow"]["estimate"] - ex) / max(fr["flow"]["error"], 1e-300),
                    "train_seconds": fr["seconds_train"], "seconds_total": el,
                    "flow_samples_per_s": 4 * n_it / max(fr["seconds_flow"], 1e-9), "iters_to_1e-3": k_flow,
                    "time_to_1e-3_s": fr["seconds_vegas"] + fr["seconds_train"] + k_flow * fr["seconds_flow"] / 4}
            except Exception as e:   # reported, not hidden: the leg says what failed
                fam["learned_w128_l6"] = {"error": f"{type(e).__name__}: {e}"}
        out[W.NAMES[fid]] = fam
    return out


# ------------------------------------------------------------------------------ batch
def batch_leg(capi, W):
    """4096 independent Gaussian integrations, d ~ U{2..8}, a_i ~ U[5, 25], u_i ~ U[0.2, 0.8],
    samples/iteration log-uniform in [1e4, 1e7], 8 iterations (4 adjust), one graph launch per
    precision; plain FP64 one job at a time on a sample of the jobs. Jobs at 1e-3 use the tta
    definition (sigma <= 1e-3 |I|) on the whole run."""
    bjobs = W.batch_jobs(4096, seed=0)
    for jb in bjobs:
        jb["seed"] = 0
    per_job = [int(np.prod(capi.stratify(jb["d"], jb["ncall"])[1:])) for jb in bjobs]
    tot = sum(per_job)
    t0 = time.perf_counter()
    tune = capi.tune_batch(bjobs, precision=capi.FP32_EVAL)
    tune_s = time.perf_counter() - t0
    capi.integrate_batch(bjobs[:32], 2, 1, precision=capi.FP32_EVAL, tune=tune)
    out = {"jobs": len(bjobs), "samples_per_iter": tot, "iters": 8, "iter_adjust": 4, "autotune_s": tune_s,
           "autotuned": {str(k): v for k, v in tune.as_dict().items()}}
    exact = closed_form_fn()
    for prec, name in ((capi.FP32_EVAL, "fp32_eval"), (capi.FP64, "fp64")):
        t0 = time.perf_counter()
        res = capi.integrate_batch(bjobs, 8, 4, precision=prec, tune=tune, raise_on_error=False)
        el = time.perf_counter() - t0
        rel = np.array([r["error"] / abs(r["estimate"]) if r["estimate"] else np.inf for r in res])
        true = np.array([abs(r["estimate"] / exact(jb["fid"], jb["params"][:jb["d"]], jb["params"][jb["d"]:]) - 1.0)
                         for r, jb in zip(res, bjobs)])
        out[name] = {"seconds": el, "samples_per_s": 8 * tot / el, "jobs_sigma_1e-3": int(np.sum(rel <= 1e-3)),
                     "median_rel_sigma": float(np.median(rel)), "median_true_rel_err": float(np.median(true)),
                     "jobs_true_1e-3": int(np.sum(true <= 1e-3))}
    sample = list(range(0, len(bjobs), 16))
    t0 = time.perf_counter()
    for k in sample:
        jb = bjobs[k]
        capi.integrate(jb["fid"], jb["params"], jb["d"], jb["ncall"], 8, 4, 0, precision=capi.FP64)
    el = time.perf_counter() - t0
    frac = sum(per_job[k] for k in sample) / tot
    out["plain_fp64_sequential"] = {"seconds_sampled": el, "jobs_sampled": len(sample),
                                    "seconds_scaled": el / frac, "samples_per_s": 8 * tot * frac / el}
    return out


# ------------------------------------------------------------------------------ PAGANI
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64, NVIDIA's figure (no measured FP64 peak is recorded)


def pagani_leg(capi, W, torch, dev, pars, mcubes64):
    """The paper's other workload (Sec. 3.1): the PAGANI region-evaluation kernel on 2^18 random
    regions of [0,1]^8 for each Genz family (regions/s, integrand evaluations/s, and the FP64 rate
    a direct evaluation would need, 6 d + 2 FP64 operations a point, against the nominal FP64
    peak), and the adaptive driver to a relative error of 1e-3 per family with up to 2^24 regions
    (wall time, regions, status, its estimate's true relative error against the family's closed
    form, and its distance from the m-Cubes FP64 estimate of the same run)."""
    closed_form = closed_form_fn()
    d = 8
    n = 1 << 18
    rng = np.random.default_rng(0)
    lo = torch.from_numpy(rng.uniform(0.0, 0.5, (n, d))).to(dev)
    ln = torch.from_numpy(rng.uniform(0.05, 0.5, (n, d))).to(dev)
    dI = torch.empty(n, dtype=torch.float64, device=dev)
    dE = torch.empty_like(dI)
    dax = torch.empty(n, dtype=torch.int32, device=dev)
    npts = capi.pagani_rule_points(d)
    kern = {}
    for fid in W.GENZ6:
        capi.pagani_evaluate_dev(fid, pars[fid], d, n, lo, ln, dI, dE, dax)   # warm-up
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record()
        for _ in range(reps):
            capi.pagani_evaluate_dev(fid, pars[fid], d, n, lo, ln, dI, dE, dax)
        b.record()
        b.synchronize()
        sec = a.elapsed_time(b) * 1e-3 / reps
        ops = (6 * d + 2) * npts * n
        kern[W.NAMES[fid]] = {"regions_per_s": n / sec, "evaluations_per_s": n * npts / sec,
                              "fp64_equiv_tflops": ops / sec / 1e12,
                              "fp64_equiv_frac_of_nominal": ops / sec / 1e12 / FP64_NOMINAL_TFLOPS, "ms": sec * 1e3}
    adapt = {}
    for fid in W.GENZ6:
        t0 = time.perf_counter()
        r = capi.pagani_integrate(fid, pars[fid], d, 1e-3, max_iters=60, max_regions=1 << 24, init_split=2)
        el = time.perf_counter() - t0
        ref = mcubes64.get(fid)
        ex = closed_form(fid, pars[fid][:d], pars[fid][d:])
        adapt[W.NAMES[fid]] = dict(r, seconds=el, exact=ex, true_rel_err=abs(r["estimate"] / ex - 1.0),
                                   estimated_rel_err=r["error"] / max(abs(r["estimate"]), 1e-300),
                                   vs_mcubes_fp64_sigma=(abs(r["estimate"] - ref["estimate"]) /
                                                         math.hypot(r["error"], ref["error"]) if ref else None))
    return {"d": d, "rule_points": npts, "kernel": kern, "adaptive_1e-3": adapt, "adaptive_max_regions": 1 << 24,
            "kernel_config": f"{n} random regions, lo ~ U[0, 0.5], len ~ U[0.05, 0.5], a_i ~ U[5,15], u_i ~ U[0.2,0.8]"}


# ------------------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline-only", action="store_true",
                    help="only the timed FP64 and FP32-eval steps and the headline line (profiling runs)")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "fp32"],
                    help="with --headline-only: which timed region to run (profiling runs)")
    ap.add_argument("--ncall", type=float, default=NCALL, help="samples per iteration (profiling runs)")
    ap.add_argument("--fp32-steps", type=int, default=None, help="timed FP32-eval steps (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tta", action="store_true", help="skip the time-to-1e-3 leg")
    ap.add_argument("--no-config2", action="store_true", help="skip the d = 5, 6 leg")
    ap.add_argument("--no-config5", action="store_true", help="skip the d = 10, 1e9 leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (4096-job) leg")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's fixed-parameter f1..f6 leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal legs")
    ap.add_argument("--pagani", action="store_true", help="run the PAGANI leg")
    ap.add_argument("--pagani-only", action="store_true", help="only the PAGANI leg (profiling runs)")
    ap.add_argument("--learned-only", action="store_true", help="only the learned-proposal leg (profiling runs)")
    ap.add_argument("--config5-only", action="store_true", help="only the d = 10, 1e9 leg")
    ap.add_argument("--train-step-only", action="store_true", help="only the training-step leg (profiling runs)")
    ap.add_argument("--train-steps", type=int, default=2000, help="flow training steps in the learned legs")
    ap.add_argument("--unit-rates", action="store_true", help="only the unit-rate microbenchmarks")
    ap.add_argument("--clocks-csv", default=None,
                    help="where to keep the raw nvidia-smi clock samples ({rank} is replaced); default: temp dir")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2302_05730_gb300 import capi, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    if args.unit_rates:
        if rank == 0:
            print(json.dumps({"unit_rates_per_sm_clock": capi.unit_rates()}), flush=True)
        return
    if args.learned_only:
        if rank == 0:
            emit("train_step", train_step_leg(capi, torch))
            emit("learned", learned_leg(capi, W, args.train_steps))
        return
    if args.pagani_only:
        if rank == 0:
            pars0 = {fid: W.genz_params(fid, D, seed=0) for fid in W.GENZ6}
            emit("pagani", pagani_leg(capi, W, torch, dev, pars0, {}))
        return
    if args.train_step_only:
        if rank == 0:
            emit("train_step", train_step_leg(capi, torch, steps=args.steps))
        return
    if args.config5_only:
        if rank == 0:
            emit("config5", config5_leg(capi, W, closed_form_fn(), args.train_steps, not args.no_learned))
        return

    stream = torch.cuda.Stream(device=dev)
    job = replica_job(rank)
    ncall = int(args.ncall)
    fams = list(W.GENZ6)
    pars = {fid: W.genz_params(fid, D, seed=0) for fid in fams}
    H = Harness(capi, torch, dev, stream, D, ncall, fams, pars, ITMAX, ADJ, job, dist)
    samples, m, p = H.samples, H.m, H.p
    n_fam = len(fams)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    sm_mhz = FALLBACK_SM_MHZ
    peak_src = "fallback 2070 MHz"
    if os.path.exists(PEAKS_FILE):
        try:
            sm_mhz = float(json.load(open(PEAKS_FILE)).get("sm_max_mhz", FALLBACK_SM_MHZ))
            peak_src = "MEASURED_PEAKS.json sm_max_mhz"
        except (ValueError, OSError):
            pass

    # ---- timed regions: plain FP64 (headline), then FP32-eval, with the clocks sampled throughout
    clocks = ClockSampler(local, args.clocks_csv.replace("{rank}", str(local)) if args.clocks_csv else None)
    clocks.start()
    run64 = args.precision in ("both", "fp64")
    run32 = args.precision in ("both", "fp32")
    kern64, kern32 = [], []
    total64 = total32 = None
    res64 = res32 = None
    if run64:
        total64, _, res64 = H.timed(capi.FP64, args.steps, args.warmup, kern64, flush)
        n_launch = H.launches
    steps32 = args.fp32_steps or args.steps
    if run32:
        total32, state32, res32 = H.timed(capi.FP32_EVAL, steps32, args.warmup, kern32, flush)
        if not run64:
            n_launch = H.launches
    clk = clocks.stop()

    peak64 = fp64_peak_ops(sm_mhz)
    peak32 = sm_peak_ops(sm_mhz)
    roof64 = kind_roofline(kern64, samples, D, fp64_ops_per_sample, peak64, p) if run64 else None
    roof32 = kind_roofline(kern32, samples, D, lambda f, d, a, p_: algorithmic_ops_per_sample(f, d, a, True),
                           peak32, p) if run32 else None
    if run64:
        for kname, v in roof64["by_kind"].items():
            v["traffic"] = VSAMPLE64_DRAM_BYTES_BY_KIND[kname] if ncall == NCALL else None
    value64 = samples * n_fam * ITMAX * args.steps * world / (total64 * 1e-3) if run64 else None
    value32 = samples * n_fam * ITMAX * steps32 * world / (total32 * 1e-3) if run32 else None

    def fp32_obj():
        if not run32:
            return None
        return {"value": round(value32, 1), "unit": "samples/s", "steps": steps32,
                "ms_per_step": round(total32 / steps32, 4), "dtype": "f32 point/integrand, f64 sums/Rebin",
                "roofline": {"bound": "alu", "pipe": "fp32 issue", "unit": "T lane-ops/s", "peak": peak32 / 1e12,
                             "achieved": round(roof32["achieved"], 5), "frac": round(roof32["frac"], 4),
                             "by_kind": {k: {"avg_launch_ms": round(v["avg_launch_ms"], 4), "frac": round(v["frac"], 4)}
                                         for k, v in roof32["by_kind"].items()}}}

    def headline(extra):
        v = value64 if run64 else value32
        tot = total64 if run64 else total32
        st = args.steps if run64 else steps32
        line = {"metric": METRIC, "value": round(v, 1), "unit": "samples/s", "n_gpus": world, "steps": st,
                "warmup": args.warmup, "ms_per_step": round(tot / st, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if run64 else "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if run64 else "genz6-d8-n1e8-fp32eval", "d": D, "ncall": ncall,
                           "m": m, "p": p, "iters": ITMAX, "iter_adjust": ADJ, "families": n_fam,
                           "params": "a~U[5,15],u~U[0.2,0.8],seed 0",
                           "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
                "gpu_launches": n_launch}
        if run64:
            line["roofline"] = {
                "bound": "alu", "pipe": "fp64", "unit": "T fp64-ops/s", "peak": peak64 / 1e12,
                "achieved": round(roof64["achieved"], 5), "frac": round(roof64["frac"], 4),
                "traffic": None if ncall != NCALL or None in VSAMPLE64_DRAM_BYTES_BY_KIND.values() else
                float(np.mean(list(VSAMPLE64_DRAM_BYTES_BY_KIND.values()))),
                "kernel": "vsample_fast64_kernel<8,fid,HK>",
                "avg_launch_ms": round(roof64["avg_launch_ms"], 4),
                "by_kind": {k: {"avg_launch_ms": round(v["avg_launch_ms"], 4), "frac": round(v["frac"], 4),
                                "traffic": v["traffic"]} for k, v in roof64["by_kind"].items()},
                "peak_basis": f"152 SMs x 2 FP64 lanes x {sm_mhz:.0f} MHz ({peak_src})"}
        line.update(extra)
        line["fp32_eval"] = fp32_obj()
        line["clocks"] = clk
        return line

    if args.headline_only:
        if rank == 0:
            emit("launch_ms", {"fp64": launch_ms_by_family(kern64, fams, W.NAMES) if run64 else None,
                               "fp32_eval": launch_ms_by_family(kern32, fams, W.NAMES) if run32 else None})
            print(json.dumps(headline({})), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    exact = closed_form_fn()
    if rank == 0:
        emit("estimates", {
            "fp64": {W.NAMES[f]: dict({"estimate": res64[f]["estimate"], "error": res64[f]["error"],
                                       "chi2_dof": res64[f]["chi2_dof"]}, **vs_exact(exact, f, pars[f], D, res64[f]))
                     for f in fams} if run64 else None,
            "fp32_eval": {W.NAMES[f]: dict({"estimate": res32[f]["estimate"], "error": res32[f]["error"],
                                            "chi2_dof": res32[f]["chi2_dof"]},
                                           **vs_exact(exact, f, pars[f], D, res32[f])) for f in fams} if run32 else None,
            "fp64_roofline_by_kind": roof64["by_kind"] if run64 else None,
            "fp32_roofline_by_kind": roof32["by_kind"] if run32 else None,
            "fp64_launch_ms_by_family": launch_ms_by_family(kern64, fams, W.NAMES) if run64 else None,
            "fp32_launch_ms_by_family": launch_ms_by_family(kern32, fams, W.NAMES) if run32 else None})
        if run32:
            unit = capi.unit_rates()
            emit("pipes", dict(pipe_bounds(unit, fams, D, roof32["by_kind"], sm_mhz, p), unit_rates_per_sm_clock=unit,
                               basis="mcubes_unit_rates microbenchmarks on this device; bound = the slowest pipe, "
                                     "all overlapped (FP32-eval V-Sample)"))

    # ---- end to end through the public host call (mcubes_integrate_ex, FP64: parameters in, per-iteration
    # results and the combined estimate out; the call uploads the previous-estimate slot and reads back
    # every iteration's sums)
    prec_e2e = capi.FP64 if run64 else capi.FP32_EVAL
    for fid in fams:   # warm-up
        capi.integrate(fid, pars[fid], D, ncall, ITMAX, ADJ, 0, precision=prec_e2e)
    H.barrier()
    e2e_steps = 2
    t = time.perf_counter()
    for k in range(e2e_steps):
        for fid in fams:
            capi.integrate(fid, pars[fid], D, ncall, ITMAX, ADJ, 1 + k, precision=prec_e2e, return_iters=True)
    e2e_s = max_over_ranks(time.perf_counter() - t, dist, dev)
    e2e = {"value": round(samples * n_fam * ITMAX * e2e_steps * world / e2e_s, 1), "unit": "samples/s",
           "h2d_bytes_per_step": n_fam * 16, "d2h_bytes_per_step": n_fam * 2 * (ITMAX + 1) * 8,
           "call": "mcubes_integrate_ex per family, host results"}

    # ---- secondary legs (rank 0)
    if rank == 0 and not args.no_config2:
        sweep = {}
        for d in (5, 6):
            pd = {fid: W.genz_params(fid, d, seed=0) for fid in fams}
            Hd = Harness(capi, torch, dev, stream, d, ncall, fams, pd, ITMAX, ADJ, job, None)
            entry = {"ncall": ncall, "m": Hd.m, "p": Hd.p}
            for prec, name, st in ((capi.FP64, "fp64", 2), (capi.FP32_EVAL, "fp32_eval", 3)):
                ev = []
                tot, _, res = Hd.timed(prec, st, 1, ev, flush)
                fam = {}
                for fid in fams:
                    ka = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and a_]
                    kf = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and not a_]
                    fam[W.NAMES[fid]] = dict({"vsample_ms_adjusting": statistics.mean(ka),
                                              "vsample_ms_frozen": statistics.mean(kf),
                                              "estimate": res[fid]["estimate"], "error": res[fid]["error"]},
                                             **vs_exact(exact, fid, pd[fid], d, res[fid]))
                entry[name] = {"samples_per_s": Hd.samples * n_fam * ITMAX * st / (tot * 1e-3), "families": fam}
            sweep[f"d{d}"] = entry
        emit("config2", sweep)

    if rank == 0 and not args.no_tta:
        emit("tta", tta_leg(capi, W, D, pars, exact))

    if rank == 0 and not args.no_paper:
        pp = {fid: W.paper_params(fid, D) for fid in fams}
        Hp = Harness(capi, torch, dev, stream, D, ncall, fams, pp, ITMAX, ADJ, job, None)
        out = {}
        for name, prec, steps in (("fp32_eval", capi.FP32_EVAL, 3), ("fp64", capi.FP64, 2)):
            ev = []
            tot, _, res = Hp.timed(prec, steps, 1, ev, flush)
            fam = {}
            for fid in fams:
                ka = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and a_]
                kf = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and not a_]
                fam[W.NAMES[fid]] = dict({"vsample_ms_adjusting": statistics.mean(ka),
                                          "vsample_ms_frozen": statistics.mean(kf),
                                          "estimate": res[fid]["estimate"], "error": res[fid]["error"]},
                                         **vs_exact(exact, fid, pp[fid], D, res[fid]))
            out[name] = {"samples_per_s": Hp.samples * n_fam * ITMAX * steps / (tot * 1e-3), "families": fam}
        emit("paper", out)

    if rank == 0 and not args.no_config5:
        emit("config5", config5_leg(capi, W, exact, args.train_steps, not args.no_learned))

    if rank == 0 and not args.no_batch:
        emit("batch", batch_leg(capi, W))

    if rank == 0 and not args.no_learned:
        emit("train_step", train_step_leg(capi, torch))
        emit("learned", learned_leg(capi, W, args.train_steps))

    if rank == 0 and args.pagani:
        emit("pagani", pagani_leg(capi, W, torch, dev, pars, res64 or {}))

    # ---- CPU baseline: the oracle (FP64) on a bounded sample of the same workload (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        grids = {fid: np.tile(np.arange(NB + 1, dtype=np.float64) / NB, (D, 1)) for fid in fams}
        starts = {fid: 0 for fid in fams}
        c1 = min(1 << 18, m)
        t0 = time.perf_counter()
        n1 = oracle_vsample_ranges(fams, pars, grids, ncall, starts, c1, 1, mode=0)
        el1 = time.perf_counter() - t0
        cn = min((1 << 18) * threads, m)
        t0 = time.perf_counter()
        nn = oracle_vsample_ranges(fams, pars, grids, ncall, starts, cn, threads, mode=0)
        el = time.perf_counter() - t0
        cpu = {"value": round(nn / el, 1), "unit": "samples/s", "cores": threads, "kind": "oracle",
               "sample": f"first {cn} sub-cubes of each of 6 families, FP64, adjusting, {threads} threads ({el:.1f} s)",
               "single_thread": round(n1 / el1, 1)}

    if rank == 0:
        line = headline({"e2e": e2e, "cpu_baseline": cpu})
        s = json.dumps(line)
        if len(s) > 2048:   # keep the headline line compact: drop the descriptive strings first
            for obj, key in ((line.get("cpu_baseline") or {}, "sample"), (line["e2e"], "call"),
                             (line["config"], "params"), (line.get("roofline") or {}, "peak_basis")):
                obj.pop(key, None)
            s = json.dumps(line)
        print(s, flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
