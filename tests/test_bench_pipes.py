"""The bench's pipe-level roofline arithmetic (pipe_bounds) on made-up unit rates: each pipe's
clocks a sample (Philox counted in 64-bit products: 17 a draw, 2 a sub-cube, 20 a call), the
binding pipe, and the measured clocks a sample against the bound."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_pipe_bounds_arithmetic():
    rates = {"philox_calls": 2.0, "shared_gather8_lanes": 4.0, "shared_atomic_u32x8_lanes": 8.0}
    fams = [0, 3]
    d = 8
    sm_mhz = 2000.0
    # launch rates that make the measured clocks a sample 4 (adjusting) and 3 (frozen)
    sps = lambda clk: bench.SMS * sm_mhz * 1e6 / clk
    kinds = {"adjusting": {"samples_per_s": sps(4.0)}, "frozen": {"samples_per_s": sps(3.0)}}
    out = bench.pipe_bounds(rates, fams, d, kinds, sm_mhz)
    adj, frz = out["adjusting"], out["frozen"]
    # 2 draws of 17 products and 2 products a sub-cube of 2 samples: 35 products, 40 a clock
    assert math.isclose(adj["clk_per_sample_by_pipe"]["philox"], 35.0 / 40.0)
    # a sub-cube's products spread over more samples
    wide = bench.pipe_bounds(rates, fams, d, kinds, sm_mhz, p=8)
    assert math.isclose(wide["frozen"]["clk_per_sample_by_pipe"]["philox"], 34.25 / 40.0)
    assert math.isclose(adj["clk_per_sample_by_pipe"]["shared_memory"], 3.0)    # 8/4 gathers + 8/8 atomics
    assert math.isclose(frz["clk_per_sample_by_pipe"]["shared_memory"], 2.0)    # gathers only
    ops = sum(bench.algorithmic_ops_per_sample(f, d, True, True) for f in fams) / len(fams)
    assert math.isclose(adj["clk_per_sample_by_pipe"]["issue"], ops / bench.LANES_PER_SM)
    assert adj["binding_pipe"] == "shared_memory" and math.isclose(adj["bound_clk_per_sample"], 3.0)
    assert math.isclose(adj["measured_clk_per_sample"], 4.0) and math.isclose(adj["frac_of_pipe_bound"], 0.75)
    assert math.isclose(frz["frac_of_pipe_bound"], 2.0 / 3.0)
