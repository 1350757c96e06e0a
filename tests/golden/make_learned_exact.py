"""Closed-form integrals of the learned-proposal workload (d = 8), written to
learned_exact_d8.json:
  - double Gaussian exp(-100|x - p1|^2) + exp(-100|x - p2|^2), p1 = 0.25 1, p2 = 0.75 1:
    twice the product of one-dimensional Gaussian integrals (erf);
  - rotated Gaussian exp(-(x - c)^T M (x - c)) with the seed-0 parameters of
    workloads.rotated_gaussian_params(8): pi^{d/2} / sqrt(det M) times the probability that
    X ~ N(c, (2M)^-1) falls in the unit cube, from scipy's multivariate normal CDF by
    inclusion-exclusion over the 2^8 corners (about a minute and a half).
Run from the repository root: python tests/golden/make_learned_exact.py"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from closed_forms import rotated_gaussian_exact   # noqa: E402
from paper_2302_05730_gb300 import workloads as W   # noqa: E402


def main():
    d = 8
    a, u = 10.0, 0.25
    one = math.sqrt(math.pi) / (2 * a) * (math.erf(a * (1 - u)) + math.erf(a * u))
    par = W.rotated_gaussian_params(d, seed=0)
    out = {"d": d,
           "double_gaussian": 2.0 * one ** d,
           "rotated_gaussian_seed0": rotated_gaussian_exact(par[:d * d].reshape(d, d), par[d * d:])}
    with open(os.path.join(HERE, "learned_exact_d8.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
