"""Benchmark of the m-Cubes hot path (V-Sample + Rebin) on GB300.

Workload: the six Genz families at d = 8 with 1e8 samples per iteration (g = 9, m = 9^8 sub-cubes,
p = 2), a_i ~ U[5, 15], u_i ~ U[0.2, 0.8] (seed 0). One step = one whole m-Cubes integration of
every family from the uniform grid: 10 iterations, the first 5 adjusting (V-Sample with bin
contributions, then Rebin), the rest frozen, with every iteration's sums read back to the host
and combined. The headline arm is FP32-eval (point and integrand in single precision, FP64 sums
and Rebin); the plain FP64 arm runs the same steps. The same line reports the end-to-end rate
through the host call, the roofline (FP32 issue, and pipe by pipe from measured unit rates), the
oracle on the host cores, times to a relative error of 1e-3, the same integration of the
paper's own fixed-parameter f1..f6 (per-family launch times and errors), the batched path, the
learned proposal and PAGANI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
# the headline metric as named for this workload: samples/s is the value; the times to a relative
# error of 1e-3 (plain, FP32-eval, learned) are in the line's time_to_1e-3 and learned blocks
METRIC = "m-Cubes samples/s; time to 1e-3 rel err, plain vs learned/FP32 (1 GB300)"
# DRAM bytes (read + write) per vsample_kernel<8, oscillatory, FP32-eval> launch at d = 8, 1e8 samples
# per iteration, from one ncu capture of this kernel as it stands: the mean over the 5 adjusting and
# 5 frozen launches of one integration, and each kind's own mean.
VSAMPLE_DRAM_BYTES = 102553
VSAMPLE_DRAM_BYTES_BY_KIND = {"adjusting": 137625, "frozen": 67481}
NB = 500
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# GB300 unit counts: 152 SMs, 4 SM sub-partitions x 32 lanes issue one instruction per clock.
SMS = 152
LANES_PER_SM = 128
FALLBACK_SM_MHZ = 2070.0


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


PHILOX_PRODUCTS_PER_CALL = 20      # two 32 x 32 -> 64-bit products a round, ten rounds
PHILOX_PRODUCTS_PER_DRAW = 17      # the sampler's hoisted form: rounds 2-9 and one product of round 1
PHILOX_PRODUCTS_PER_CUBE = 2       # ... plus round 0's and round 1's products of the sub-cube index


def pipe_bounds(rates: dict, fams, d: int, kinds: dict, sm_mhz: float, p: int = 2) -> dict:
    """Pipe-level roofline of the V-Sample kernels: per launch kind, the SM clocks a sample needs on
    each pipe at the measured unit rates (mcubes_unit_rates) -- Philox's 64-bit integer products
    (17 a draw plus 2 a sub-cube of p samples, at 20 a measured Philox call), the shared-memory
    pipe (table gathers, plus the histogram's u32 atomics when adjusting: both use it) and
    instruction issue of the algorithmic operations -- their maximum (the bound, every pipe
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


# ------------------------------------------------------------------------------ oracle timing
def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_vsample_ranges(fams, pars, grids, ncall, starts, cubes, threads, it=1):
    """The oracle's V-Sample over [t0, t0 + cubes) of each family, split into `threads` equal
    sub-ranges run side by side (the oracle holds no global state and ctypes releases the
    interpreter lock during the call). Returns the samples processed."""
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
        oracle.vsample(fid, D, pars[fid], ncall, 0, it=it, mode=1, adjust=1, B=grids[fid], t0=a, t1=b)
        return (b - a) * p

    if threads == 1:
        return sum(one(j) for j in jobs)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return sum(ex.map(one, jobs))


# ------------------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    """The CPU oracle on a bounded sample of the workload (sub-cube ranges of each family)."""
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
        return oracle_vsample_ranges(W.GENZ6, pars, grids, NCALL, starts, cubes, threads, it=k % 65536)

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
            "config": {"workload": "genz6-d8-n1e8-fp32eval", "d": D, "ncall": NCALL,
                       "families": [W.NAMES[f] for f in W.GENZ6], "sample_cubes_per_family_step": cubes},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"{cubes} sub-cubes ({cubes * p} samples) of each of the 6 families per step, "
                                       f"FP32-eval point layout, {threads} threads over equal sub-cube ranges"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ learned proposal
def learned_leg(capi, W, train_steps: int, n_it: int = 1 << 20, seeds=(0, 1, 2)):
    """Learned proposal (4-layer coupling flow, width 64, 16 bins, variance loss on f^2 J weights;
    2^20 samples per iteration) on the double Gaussian exp(-100|x - p1|^2) + exp(-100|x - p2|^2),
    p1 = 0.25 1, p2 = 0.75 1, and on a rotated anisotropic Gaussian (random orthogonal Q,
    eigenvalues 1..400), d = 8. Per training seed: the variance per sample against the adapted grid
    at the same budget; each method's estimate against the closed form (z-score, true relative
    error); and the time to a relative error of 1e-3 for the learned proposal, the FP32-eval grid
    and the plain FP64 grid: warm-up plus the iterations the measured per-iteration variance needs,
    or null when the method's estimate disagrees with the closed form (|z| > 4), since then more
    iterations shrink its error bar but not its error. Training differs from seed to seed, so the
    leg reports every seed and the medians."""
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
        # plain m-Cubes on the same integrand: per-iteration time and variance after adaptation (after
        # one untimed call of each precision, which sets up the kernels' launch attributes)
        for prec in (capi.FP64, capi.FP32_EVAL):
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


# ------------------------------------------------------------------------------ PAGANI
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64, NVIDIA's figure (no measured FP64 peak is recorded)


def pagani_leg(capi, W, torch, dev, pars, mcubes64):
    """The paper's other workload (Sec. 3.1): the PAGANI region-evaluation kernel on 2^18 random
    regions of [0,1]^8 for each Genz family (regions/s, integrand evaluations/s, and the FP64 rate
    a direct evaluation would need, 6 d + 2 FP64 operations a point -- the map to the region, the
    family's per-axis arithmetic, the class sum, the exp -- against the nominal FP64 peak; the
    kernel itself tabulates the separable families per axis and does less), and the
    adaptive driver to a relative error of 1e-3 per family with up to 2^24 regions (wall time,
    regions, status, its estimate's true relative error against the family's closed form, and its
    distance from the m-Cubes FP64 estimate of the same run)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from closed_forms import exact as closed_form
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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tta", action="store_true", help="skip the time-to-1e-3 leg")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the FP32-eval device-resident leg (profiling runs)")
    ap.add_argument("--ncall", type=float, default=NCALL, help="samples per iteration (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (4096-job) leg")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's fixed-parameter f1..f6 leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal leg")
    ap.add_argument("--no-pagani", action="store_true", help="skip the PAGANI leg")
    ap.add_argument("--pagani-only", action="store_true", help="only the PAGANI leg (profiling runs)")
    ap.add_argument("--learned-only", action="store_true", help="only the learned-proposal leg (profiling runs)")
    ap.add_argument("--train-steps", type=int, default=2000, help="flow training steps in the learned leg")
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
            print(json.dumps({"learned": learned_leg(capi, W, args.train_steps)}), flush=True)
        return
    if args.pagani_only:
        if rank == 0:
            pars0 = {fid: W.genz_params(fid, D, seed=0) for fid in W.GENZ6}
            print(json.dumps({"pagani": pagani_leg(capi, W, torch, dev, pars0, {})}), flush=True)
        return

    stream = torch.cuda.Stream(device=dev)
    job = replica_job(rank)
    ncall = int(args.ncall)
    g, m, p = capi.stratify(D, ncall)
    samples = m * p
    fams = list(W.GENZ6)
    pars = {fid: W.genz_params(fid, D, seed=0) for fid in fams}
    uni = torch.from_numpy(np.tile(np.arange(NB + 1, dtype=np.float64) / NB, (D, 1))).to(dev)

    ITMAX, ADJ = 10, 5   # one m-Cubes integration: 10 iterations, the first 5 adjust the grid
    n_fam = len(fams)
    sums_all = torch.zeros((n_fam, ITMAX, 2), dtype=torch.float64, device=dev)
    sums_host = torch.zeros((n_fam, ITMAX, 2), dtype=torch.float64).pin_memory()

    def fresh_state():
        st = {}
        for fid in fams:
            st[fid] = dict(grid=[uni.clone(), torch.empty_like(uni)], cur=0,
                           C=torch.zeros(D * NB, dtype=torch.float64, device=dev))
        return st

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    run_counter = [0]
    launches = [0]

    def step(state, prec, kernel_events=None):
        """One whole integration of each family (all hot-path rows): uniform grid, ITMAX
        V-Sample passes (the first ADJ accumulate bin contributions and rebin), the sums of every
        iteration to the host in one copy; the host combination follows the step."""
        seed = run_counter[0]
        run_counter[0] += 1
        sums_all.zero_()
        for f, fid in enumerate(fams):
            s = state[fid]
            s["grid"][0].copy_(uni)
            s["cur"] = 0
            for it in range(ITMAX):
                adjust = it < ADJ
                if adjust:
                    s["C"].zero_()
                gin, gout = s["grid"][s["cur"]], s["grid"][1 - s["cur"]]
                if kernel_events is not None:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                capi.vsample_dev(fid, pars[fid], D, ncall, seed, it, job, int(adjust), prec, gin,
                                 s["C"] if adjust else None, sums_all[f, it], stream=stream)
                if kernel_events is not None:
                    e1.record(stream)
                    kernel_events.append((fid, adjust, e0, e1))
                launches[0] += 1
                if adjust and it + 1 < ITMAX:
                    capi.rebin_dev(D, gin, s["C"], gout, stream=stream)
                    launches[0] += 1
                    s["cur"] = 1 - s["cur"]
        sums_host.copy_(sums_all, non_blocking=True)

    def combine_all():
        """The combination (mcubes_combine) of every family's iterations after a step."""
        out = {}
        for f, fid in enumerate(fams):
            it = sums_host[f].numpy().copy()
            it[:, 0] /= m
            it[:, 1] /= float(m) * float(m)
            out[fid] = capi.combine(it)
        return out

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(prec, steps, warmup, kern=None):
        state = fresh_state()
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step(state, prec)
        barrier()
        launches[0] = 0
        step_ms = []
        res = None
        for _ in range(steps):
            flush.add_(1.0)   # evict L2 between timed steps (outside the timed events)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                step(state, prec, kern)
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            res = combine_all()
        barrier()
        total_ms = max_over_ranks(sum(step_ms), dist, dev)
        for fid in fams:   # sanity: the last step's estimates are finite
            assert math.isfinite(res[fid]["estimate"]) and math.isfinite(res[fid]["error"]), (fid, res[fid])
        return total_ms, state, res

    # ---- headline: FP32-eval
    clocks = ClockSampler(local, args.clocks_csv.replace("{rank}", str(local)) if args.clocks_csv else None)
    clocks.start()
    kern_ev = []
    total_ms, state32, res32 = timed(capi.FP32_EVAL, args.steps, args.warmup, kern_ev)
    clk = clocks.stop()
    n_launch = launches[0]
    ms_step = total_ms / args.steps
    value = samples * n_fam * ITMAX * args.steps * world / (total_ms * 1e-3)

    # dominant kernel: the V-Sample launches inside the timed region (adjusting and frozen)
    sm_mhz = FALLBACK_SM_MHZ
    peak_src = "fallback (2070 MHz max SM clock)"
    if os.path.exists(PEAKS_FILE):
        try:
            sm_mhz = float(json.load(open(PEAKS_FILE)).get("sm_max_mhz", FALLBACK_SM_MHZ))
            peak_src = "MEASURED_PEAKS.json sm_max_mhz"
        except (ValueError, OSError):
            pass
    peak = sm_peak_ops(sm_mhz) / 1e12
    kinds = {}
    for adj in (True, False):
        ev = [(fid, e0.elapsed_time(e1)) for (fid, a_, e0, e1) in kern_ev if a_ == adj]
        ops_k = sum(algorithmic_ops_per_sample(fid, D, adj, True) * samples for fid, _ in ev)
        ms_k = sum(t for _, t in ev)
        name = "adjusting" if adj else "frozen"
        kinds[name] = {
            "launches": len(ev), "avg_launch_ms": ms_k / len(ev), "samples_per_s": samples * len(ev) / (ms_k * 1e-3),
            "achieved": ops_k / (ms_k * 1e-3) / 1e12, "frac": ops_k / (ms_k * 1e-3) / 1e12 / peak,
            "traffic": VSAMPLE_DRAM_BYTES_BY_KIND[name] if ncall == NCALL else None}
    all_ms = sum(e0.elapsed_time(e1) for (_, _, e0, e1) in kern_ev)
    ops = sum(algorithmic_ops_per_sample(fid, D, a_, True) * samples for (fid, a_, _, _) in kern_ev)
    avg_kms = all_ms / len(kern_ev)
    achieved = ops / (all_ms * 1e-3) / 1e12
    ops_per_launch = ops / len(kern_ev)

    if args.headline_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "samples/s",
                              "ms_per_step": ms_step, "ncall": ncall, "avg_launch_ms": avg_kms,
                              "by_kind": kinds, "gpu_launches": n_launch, "clocks": clk}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- each estimate against the family's closed form (the last timed step of each precision)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from closed_forms import exact as closed_form

    def vs_exact(fid, r):
        ex = closed_form(fid, pars[fid][:D], pars[fid][D:])
        return {"exact": ex, "true_rel_err": abs(r["estimate"] / ex - 1.0),
                "z": (r["estimate"] - ex) / max(r["error"], 1e-300)}

    # ---- pipe-level roofline of the same launches, from the device's measured unit rates (after the
    # timed region)
    unit = capi.unit_rates()
    pipes = dict(pipe_bounds(unit, fams, D, kinds, sm_mhz, p), unit_rates_per_sm_clock=unit,
                 basis="mcubes_unit_rates microbenchmarks on this device; bound = the slowest pipe, all overlapped")

    # ---- plain FP64 arm (same steps)
    f64_steps = 3
    total64, _, res64 = timed(capi.FP64, f64_steps, 3)
    value64 = samples * n_fam * ITMAX * f64_steps * world / (total64 * 1e-3)

    # ---- end to end through the public host call (mcubes_integrate_ex: parameters in, per-iteration
    # results and the combined estimate out; the call uploads the previous-estimate slot and reads back
    # every iteration's sums)
    for fid in fams:   # warm-up
        capi.integrate(fid, pars[fid], D, ncall, ITMAX, ADJ, 0, precision=capi.FP32_EVAL)
    barrier()
    e2e_steps = 3
    t = time.perf_counter()
    e2e_res = {}
    for k in range(e2e_steps):
        for fid in fams:
            e2e_res[fid] = capi.integrate(fid, pars[fid], D, ncall, ITMAX, ADJ, 1 + k, precision=capi.FP32_EVAL,
                                          return_iters=True)
    e2e_s = max_over_ranks(time.perf_counter() - t, dist, dev)
    e2e_value = samples * n_fam * ITMAX * e2e_steps * world / e2e_s
    h2d = n_fam * 16                       # the previous-estimate slot
    d2h = n_fam * 2 * (ITMAX + 1) * 8      # every iteration's (sum I_t, sum V_t)

    # ---- the paper's own fixed-parameter f1..f6 at d = 8 (Sec. 5, Eq. 1-6) through the same integration:
    # mean V-Sample launch times per family beside the estimates' errors against the closed forms. This
    # is context for the paper's per-family kernel timings (Sec. 5), which state no sample count.
    def paper_leg():
        saved = dict(pars)
        pars.update({fid: W.paper_params(fid, D) for fid in fams})
        out = {}
        try:
            for name, prec, steps in (("fp32_eval", capi.FP32_EVAL, 3), ("fp64", capi.FP64, 2)):
                ev = []
                tot, _, res = timed(prec, steps, 2, ev)
                fam = {}
                for fid in fams:
                    ka = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and a_]
                    kf = [e0.elapsed_time(e1) for (f, a_, e0, e1) in ev if f == fid and not a_]
                    fam[W.NAMES[fid]] = dict({"vsample_ms_adjusting": statistics.mean(ka),
                                              "vsample_ms_frozen": statistics.mean(kf),
                                              "estimate": res[fid]["estimate"], "error": res[fid]["error"]},
                                             **vs_exact(fid, res[fid]))
                out[name] = {"samples_per_s": samples * n_fam * ITMAX * steps * world / (tot * 1e-3), "families": fam}
        finally:
            pars.clear()
            pars.update(saved)
        return out

    paper = None if args.no_paper else paper_leg()

    # ---- time to 1e-3 relative error (full mcubes_integrate runs, host buffers)
    tta = None
    if not args.no_tta and rank == 0:
        tta = {}
        for prec, name in ((capi.FP64, "fp64"), (capi.FP32_EVAL, "fp32_eval")):
            per = {}
            for fid in fams:
                k_hit = None
                for k in range(1, 11):
                    t0 = time.perf_counter()
                    r = capi.integrate(fid, pars[fid], D, ncall, k, min(k, 5), 0, precision=prec)
                    el = time.perf_counter() - t0
                    if r["error"] <= 1e-3 * abs(r["estimate"]):
                        k_hit = (k, el)
                        break
                per[W.NAMES[fid]] = {"iters": k_hit[0], "seconds": k_hit[1]} if k_hit else None
            tta[name] = per

    # ---- batched form: 4096 independent Gaussian integrations, d ~ U{2..8}, a_i ~ U[5, 25],
    # u_i ~ U[0.2, 0.8], samples/iteration log-uniform in [1e4, 1e7], 8 iterations (4 adjust),
    # one graph launch per precision; plain FP64 one job at a time on a sample of the jobs
    batch = None
    if not args.no_batch and rank == 0:
        bjobs = W.batch_jobs(4096, seed=0)
        for k, jb in enumerate(bjobs):
            jb["seed"] = 0
        per_job = [int(np.prod(capi.stratify(jb["d"], jb["ncall"])[1:])) for jb in bjobs]
        tot = sum(per_job)
        t0 = time.perf_counter()
        tune = capi.tune_batch(bjobs, precision=capi.FP32_EVAL)
        tune_s = time.perf_counter() - t0
        capi.integrate_batch(bjobs[:32], 2, 1, precision=capi.FP32_EVAL, tune=tune)
        batch = {"jobs": len(bjobs), "samples_per_iter": tot, "iters": 8, "iter_adjust": 4, "autotune_s": tune_s,
                 "autotuned": {str(k): v for k, v in tune.as_dict().items()}}
        for prec, name in ((capi.FP32_EVAL, "fp32_eval"), (capi.FP64, "fp64")):
            t0 = time.perf_counter()
            res = capi.integrate_batch(bjobs, 8, 4, precision=prec, tune=tune, raise_on_error=False)
            el = time.perf_counter() - t0
            rel = np.array([r["error"] / abs(r["estimate"]) if r["estimate"] else np.inf for r in res])
            batch[name] = {"seconds": el, "samples_per_s": 8 * tot / el,
                           "jobs_at_1e-3": int(np.sum(rel <= 1e-3)), "median_rel_err": float(np.median(rel))}
        # plain FP64 m-Cubes, one job at a time, on every 16th job; scaled to the whole batch
        sample = list(range(0, len(bjobs), 16))
        t0 = time.perf_counter()
        for k in sample:
            jb = bjobs[k]
            capi.integrate(jb["fid"], jb["params"], jb["d"], jb["ncall"], 8, 4, 0, precision=capi.FP64)
        el = time.perf_counter() - t0
        frac = sum(per_job[k] for k in sample) / tot
        batch["plain_fp64_sequential"] = {"seconds_sampled": el, "jobs_sampled": len(sample),
                                          "seconds_scaled": el / frac, "samples_per_s": 8 * tot * frac / el}

    learned = None
    if not args.no_learned and rank == 0:
        learned = learned_leg(capi, W, args.train_steps)

    pagani = None
    if not args.no_pagani and rank == 0:
        pagani = pagani_leg(capi, W, torch, dev, pars, res64)

    # ---- CPU baseline: the oracle on a bounded sample of the same workload (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        grids = {fid: state32[fid]["grid"][state32[fid]["cur"]].cpu().numpy() for fid in fams}   # adapted
        starts = {fid: 0 for fid in fams}
        c1 = min(1 << 20, m)
        t0 = time.perf_counter()
        n1 = oracle_vsample_ranges(fams, pars, grids, ncall, starts, c1, 1)
        el1 = time.perf_counter() - t0
        cn = min((1 << 19) * threads, m)
        t0 = time.perf_counter()
        nn = oracle_vsample_ranges(fams, pars, grids, ncall, starts, cn, threads)
        el = time.perf_counter() - t0
        cpu = {"value": nn / el, "unit": "samples/s", "cores": threads, "kind": "oracle",
               "sample": f"first {cn} sub-cubes ({cn * p} samples) of each of the 6 families on the adapted "
                         f"grids, FP32-eval point layout, {threads} threads over equal sub-cube ranges ({el:.1f} s)",
               "single_thread": {"value": n1 / el1, "sample": f"first {c1} sub-cubes of each family ({el1:.1f} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "genz6-d8-n1e8-fp32eval", "d": D, "ncall": ncall, "g": g, "m": m, "p": p,
                       "families": [W.NAMES[f] for f in fams], "params": "a_i~U[5,15], u_i~U[0.2,0.8], seed 0",
                       "step": f"one whole m-Cubes integration of each family: {ITMAX} iterations, the first {ADJ} "
                               "adjusting (V-Sample with bin contributions + Rebin), the rest frozen; sums to the "
                               "host and the combination", "precision": "FP32-eval, FP64 sums/Rebin",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "estimates": {W.NAMES[f]: dict({"estimate": res32[f]["estimate"], "error": res32[f]["error"],
                                            "chi2_dof": res32[f]["chi2_dof"]}, **vs_exact(f, res32[f])) for f in fams},
            "fp64": {"value": value64, "unit": "samples/s", "steps": f64_steps,
                     "estimates": {W.NAMES[f]: dict({"estimate": res64[f]["estimate"], "error": res64[f]["error"]},
                                                   **vs_exact(f, res64[f])) for f in fams}},
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": f"mcubes_integrate_ex per family ({ITMAX} iterations, {ADJ} adjusting), host results"},
            "gpu_launches": n_launch,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s",
                         "frac": achieved / peak,
                         "traffic": VSAMPLE_DRAM_BYTES if ncall == NCALL else None,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the 10 "
                                           "launches of one full-size integration "
                                           "(profiles/vsample_fp32_d8_genz6_n1e8_launches.md)",
                         "kernel": "vsample_kernel<8, fid, FP32, HK> (adjusting launches: HK = 2, fixed-point "
                                   "histogram, 152 x 1024; frozen launches: HK = 0, 608 x 256)",
                         "ops_per_launch": ops_per_launch, "avg_launch_ms": avg_kms, "by_kind": kinds,
                         "peak_basis": f"152 SMs x 128 lanes x {sm_mhz:.0f} MHz ({peak_src})",
                         "pipes": pipes},
            "cpu_baseline": cpu,
            "time_to_1e-3": tta,
            "paper_f1_f6_d8": paper,
            "batch": batch,
            "learned": learned,
            "pagani": pagani,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
