"""The library's three forms of Philox4x32-10 (the plain generator, the hoisted form of the
single-job V-Sample kernels and the register form of the batched kernel), compiled for the host
from the library's own header and checked word for word against the oracle's Philox on the CPU.

The forms differ only in where the work sits: round 0 and part of round 1 are precomputed per
launch (the products of counter word 2) and per sub-cube (the products of counter word 0), and
the round keys are stored or formed as needed. Counter word 2 is split into the launch constant
(its top 29 bits) and the draw word j (its low 3 bits)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_05730_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "common.cuh"
using namespace mcubes;
int main()
{
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        const Words4 a = philox4x32_10(c0, c1, c2, c3, k0, k1);
        PhiloxPre pp;
        philox_prepare(pp, k0, k1, c2 & ~7u, c3);
        const Words4 b = philox_draw(c1, (int)(c2 & 7u), philox_cube(c0, pp), pp);
        uint32_t aj, bkj;
        philox_draw_consts(k0, c2 & ~7u, (int)(c2 & 7u), aj, bkj);
        const Words4 c = philox_draw_k(c1, aj, bkj, philox_cube_k(c0, c3 ^ k1), k0, k1);
        std::printf("%u %u %u %u %u %u %u %u %u %u %u %u\n", a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w,
                    c.x, c.y, c.z, c.w);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def forms_exe(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("philox_forms")
    src = d / "forms.cpp"
    src.write_text(PROGRAM)
    exe = d / "forms"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe)


def _run(exe, rows):
    inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    return [[int(v) for v in line.split()] for line in out if line.strip()]


def test_three_forms_match_the_oracle(forms_exe):
    rng = np.random.default_rng(11)
    rows = rng.integers(0, 2 ** 32, size=(400, 6), dtype=np.uint64).tolist()
    # edge counters and keys, and the sampler's own layout (t, q, it << 16 | j, job)
    rows += [[0, 0, 0, 0, 0, 0], [2 ** 32 - 1] * 6, [1, 2, 3, 4, 5, 6], [0, 0, 7, 0, 2 ** 32 - 1, 0],
             [43046720, 1, (9 << 16) | 1, 0, 0x12345678, 0x9ABCDEF0], [5, 0, (65535 << 16) | 3, 2 ** 30, 1, 2]]
    got = _run(forms_exe, rows)
    assert len(got) == len(rows)
    for r, g in zip(rows, got):
        want = oracle.philox(r[:4], r[4:])
        assert g[0:4] == want, (r, g[0:4], want)      # plain generator
        assert g[4:8] == want, (r, g[4:8], want)      # hoisted, launch constants stored
        assert g[8:12] == want, (r, g[8:12], want)    # hoisted, register form


def test_a_wrong_split_is_caught(forms_exe):
    """The split of counter word 2 matters: the same counters with word 2 offset by one give
    different words, so the comparison above is not vacuous."""
    rows = [[3, 1, 16, 9, 7, 8]]
    got = _run(forms_exe, rows)[0]
    assert got[4:8] != oracle.philox([3, 1, 17, 9], [7, 8])
