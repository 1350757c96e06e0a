"""The fast FP64 V-Sample kernel's bit-level steps (`csrc/fp64_bits.cuh`), compiled for the host
from the library's own header and checked on the CPU (paper Sec. 3.2, Algorithm 2: the map's bin
and offset, and the closing exp and cos of the Genz families, Eq. 1-6):

- yn = fl(fl(c + u) R) from the integers c 2^52 + bits, bit for bit against numpy's FP64 addition and
  multiplication (strata counts 1-2048, ties of both roundings included);
- the bin k = floor(yn) and the offset G = 1 + (yn - k) from yn's bits (exact for yn >= 1; within
  2^-52 below 1);
- small integers as FP64 values, and the FP32-found reduction integer;
- 2^E exp(x) and cos(2 pi t) from the tables the kernel fills, against 120-digit arithmetic: within
  3 units of 2^-53 (relative; exp) and 2 units of 2^-53 (absolute; cos), across the library
  fallbacks (|x| >= 708, where the library's exp is scaled after rounding, as the definition forms f
  before the Jacobian; subnormal and overflowing results; |t| >= 2^12).
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_05730_gb300", "csrc")
U53 = 2.0 ** -53

PROGRAM = r"""
#include <cstdio>
#include "fp64_bits.cuh"
using namespace mcubes;
static double d(unsigned long long b) { return bits::from_dbits(b); }
static unsigned long long b(double x) { return bits::dbits(x); }
int main()
{
    static double T[kExpTab];
    static double2 CS[kCosTab];
    unsigned long long v, w;
    for (int j = 0; j < kExpTab; ++j) { if (std::scanf("%llu", &v) != 1) return 1; T[j] = d(v); }
    for (int j = 0; j < kCosTab; ++j) {
        if (std::scanf("%llu %llu", &v, &w) != 2) return 1;
        CS[j].x = d(v);
        CS[j].y = d(w);
    }
    char op[2];
    while (std::scanf("%1s", op) == 1) {
        if (op[0] == 'Y') {            // c bits g: yn = fl(fl(c + u) R), R = 500 / g
            unsigned c, g;
            unsigned long long u;
            if (std::scanf("%u %llu %u", &c, &u, &g) != 3) return 1;
            const unsigned long long Rb = b(500.0 / (double)g);
            const unsigned long long Rm = (Rb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
            const int eR = (int)(Rb >> 52) - 1023;
            const unsigned long long N = ((unsigned long long)c << 52) | u;
            std::printf("%llu\n", cu_times_r_bits((uint32_t)(N >> 32), (uint32_t)N, Rm, eR));
        } else if (op[0] == 'S') {     // yn bits: bin and offset
            if (std::scanf("%llu", &v) != 1) return 1;
            unsigned long long gb;
            const int k = split_bin(v, gb);
            std::printf("%d %llu\n", k, gb);
        } else if (op[0] == 'I') {     // k: FP64 value and the FP32 reduction integer of k + 0.3
            int k;
            if (std::scanf("%d", &k) != 1) return 1;
            std::printf("%llu %d\n", b(small_int_to_double(k)), f32_round_int((float)k + 0.3f));
        } else if (op[0] == 'E') {     // x bits, E: 2^E exp(x)
            int E;
            if (std::scanf("%llu %d", &v, &E) != 2) return 1;
            std::printf("%llu\n", b(exp_tab(d(v), E, T)));
        } else if (op[0] == 'J') {     // d, s bits, then d bin factors P_k: the exp families' folded weight
            int dd;
            if (std::scanf("%d %llu", &dd, &v) != 2) return 1;
            const double s = d(v);
            int sE = 0;                 // the exponent fields of the P_k
            long long sl = 0;           // ln m_k, |P_k| = 2^E_k m_k, in 2^-52 units (the block's table)
            for (int i = 0; i < dd; ++i) {
                if (std::scanf("%llu", &w) != 1) return 1;
                const double pk = d(w), ap = std::fabs(pk);
                const int field = (bits::hi(pk) >> 20) & 0x7FF;
                const double lm = ap > 0.0 ? std::log(std::ldexp(ap, -(field - 1023))) : -64.0;
                sE += field;
                sl += std::llrint(std::ldexp(lm, 52));
            }
            std::printf("%llu\n", b(exp_tab(bits::fma_rn((double)sl, 0x1p-52, -s), sE - dd * 1023, T)));
        } else if (op[0] == 'C') {     // t bits: cos(2 pi t)
            if (std::scanf("%llu", &v) != 1) return 1;
            std::printf("%llu\n", b(cos_turns(d(v), CS)));
        } else {
            return 1;
        }
    }
    return 0;
}
"""


def _bits(x):
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])


def _from_bits(b):
    return float(np.array([b], dtype=np.uint64).view(np.float64)[0])


@pytest.fixture(scope="module")
def mp():
    return pytest.importorskip("mpmath")


@pytest.fixture(scope="module")
def bits_exe(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "vector_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("fp64_bits")
    src = d / "bits.cpp"
    src.write_text(PROGRAM)
    exe = d / "bits"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", "-I", CSRC, "-I", cuda_inc, str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe)


@pytest.fixture(scope="module")
def tables(mp):
    """The kernel's per-block tables, correctly rounded: 2^(j/256), and cos, sin of 2 pi j / 256."""
    with mp.workprec(200):
        ex = [_bits(float(mp.mpf(2) ** (mp.mpf(j) / 256))) for j in range(256)]
        cs = [(_bits(float(mp.cos(2 * mp.pi * j / 256))), _bits(float(mp.sin(2 * mp.pi * j / 256))))
              for j in range(256)]
    return "\n".join(str(x) for x in ex) + "\n" + "\n".join(f"{c} {s}" for c, s in cs) + "\n"


def _run(exe, tables, lines):
    r = subprocess.run([exe], input=tables + "\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout.split("\n")
    return out[:len(lines)]


def test_yn_bit_identical_to_fp64(bits_exe, tables):
    rng = np.random.default_rng(5)
    cases = []
    for g in (1, 2, 3, 7, 9, 10, 33, 34, 100, 500, 501, 1000, 2047, 2048):
        cases += [(c, b, g) for c in sorted({0, 1, g - 1}) for b in (0, 1, (1 << 52) - 1, 1 << 51)]
        cs = rng.integers(0, g, 1500)
        bs = rng.integers(0, 1 << 52, 1500, dtype=np.int64)
        cases += [(int(c), int(b), g) for c, b in zip(cs, bs)]
        # c + u exactly halfway between two doubles (low bits 100...0 under the rounding point)
        cases += [(int(c), (int(b) & ~0xFFF) | 0x800, g) for c, b in zip(cs[:400], bs[:400])]
    out = _run(bits_exe, tables, [f"Y {c} {b} {g}" for c, b, g in cases])
    bad = 0
    for (c, b, g), got in zip(cases, out):
        want = (np.float64(c) + np.float64(b) * np.float64(2.0 ** -52)) * (np.float64(500.0) / np.float64(g))
        bad += int(got) != _bits(want)
    assert bad == 0, f"{bad} of {len(cases)} differ from the FP64 operations"


def test_split_bin(bits_exe, tables):
    rng = np.random.default_rng(6)
    ys = list(rng.uniform(0.0, 500.0, 3000)) + list(rng.uniform(0.0, 1.0, 1000)) + list(10.0 ** rng.uniform(-300, 0, 500))
    ys += [0.0, 5e-324, 1.0, np.nextafter(1.0, 0.0), 2.0, np.nextafter(2.0, 0.0), 499.5, np.nextafter(500.0, 0.0)]
    ys += [float(k) for k in range(1, 500, 37)] + [np.nextafter(float(k), 0.0) for k in range(1, 500, 37)]
    out = _run(bits_exe, tables, [f"S {_bits(y)}" for y in ys])
    for y, line in zip(ys, out):
        k, gb = (int(v) for v in line.split())
        G = _from_bits(gb)
        assert k == math.floor(y), (y, k)
        if y >= 1.0:
            assert G == 1.0 + (y - k), (y, G)          # exact: y - k and 1 + (y - k) are representable
        else:
            assert 1.0 <= G < 2.0 and 0.0 <= (1.0 + y) - G < 2.0 ** -52 * 1.0000001, (y, G)


def test_small_integers(bits_exe, tables):
    ks = list(range(-(1 << 20), (1 << 20) + 1, 4099)) + [0, 1, -1, 2, 3, 255, 256, -256, 1 << 20, -(1 << 20)]
    out = _run(bits_exe, tables, [f"I {k}" for k in ks])
    for k, line in zip(ks, out):
        v, r = (int(x) for x in line.split())
        assert _from_bits(v) == float(k), k
        assert r == k, (k, r)                        # the FP32 round of k + 0.3 is k


def test_exp_tab_against_high_precision(bits_exe, tables, mp):
    rng = np.random.default_rng(7)
    xs = list(rng.uniform(-707.9, 707.9, 1500)) + list(rng.uniform(-6.0, 6.0, 1500))
    xs += [0.0, -0.0, 1e-300, -1e-200, 707.9, -707.9, 0.5 * math.log(2) / 256, 745.5, -745.0, -800.0, 709.5]
    es = [0, -48, 37, -1000, 900]
    lines, cases = [], []
    for x in xs:
        for E in es:
            lines.append(f"E {_bits(x)} {E}")
            cases.append((x, E))
    out = _run(bits_exe, tables, lines)
    tiny, huge = 2.0 ** -1022, np.finfo(np.float64).max
    worst = 0.0
    with mp.workprec(400):
        for (x, E), line in zip(cases, out):
            got = _from_bits(int(line))
            if abs(x) >= 708.0:
                # the library's exp first (rounded to FP64: overflow to inf, underflow to a subnormal or 0),
                # then the scaling, as the definition forms f before it meets the Jacobian
                f = float(mp.exp(mp.mpf(x)))
                try:
                    want = math.ldexp(f, E) if math.isfinite(f) else math.inf
                except OverflowError:
                    want = math.inf
                if want == math.inf or want == 0.0:
                    assert got == want, (x, E, got, want)
                else:
                    assert abs(got - want) <= 4 * U53 * abs(want) + 2.0 ** -1073, (x, E, got, want)
                continue
            want = mp.exp(mp.mpf(x)) * mp.mpf(2) ** E
            if want > huge * (1 + U53):
                assert got == math.inf, (x, E, got)
            elif want >= tiny:
                err = float(abs(mp.mpf(got) - want) / want)
                worst = max(worst, err)
                assert err <= 3 * U53, (x, E, got, float(want), err / U53)
            else:                                   # subnormal or zero: within two subnormal units
                assert abs(mp.mpf(got) - want) <= 2 * mp.mpf(2) ** -1074 + 3 * U53 * want, (x, E, got, float(want))
    assert worst > 0.0


def test_jacobian_in_exponent(bits_exe, tables, mp):
    """The Gaussian's and C0's weight exp(-s) prod |P_k| as the kernel forms it: the bins' exponent
    fields summed as integers, ln m_k summed in 2^-52 fixed point, one exp_tab call. Its error is that of
    exp at the argument x = sum ln m_k - s (|x| units of 2^-53) plus the d table entries' roundings."""
    rng = np.random.default_rng(9)
    lines, cases = [], []
    for _ in range(3000):
        d = int(rng.integers(1, 17))
        P = rng.choice([-1.0, 1.0], d) * 10.0 ** rng.uniform(-6, 1.5, d)
        s = float(rng.uniform(0.0, 40.0))
        lines.append(f"J {d} {_bits(s)} " + " ".join(str(_bits(float(p))) for p in P))
        cases.append((s, P))
    # subnormal and zero-width factors: the weight is prod |P_k| exp(-s), or zero
    for P in ([1e-310, 0.3, 2.0], [0.0, 0.5, 0.7], [5e-324, 1e300, 1e10]):
        lines.append(f"J 3 {_bits(0.5)} " + " ".join(str(_bits(p)) for p in P))
        cases.append((0.5, np.array(P)))
    out = _run(bits_exe, tables, lines)
    worst = 0.0
    with mp.workprec(400):
        for (s, P), line in zip(cases, out):
            got = _from_bits(int(line))
            want = mp.exp(-mp.mpf(s)) * mp.fprod([abs(mp.mpf(float(p))) for p in P])
            if want == 0:
                assert got == 0.0
                continue
            if want < 2.0 ** -1022:
                assert abs(mp.mpf(got) - want) <= 2 * mp.mpf(2) ** -1074 + 1e-12 * want, (s, P, got)
                continue
            # the argument exp_tab receives: ln m_k with E_k = (exponent field) - 1023, as the kernel takes it
            # (a subnormal factor's m_k lies below 1)
            x = abs(float(sum(mp.log(abs(mp.mpf(float(p))) / mp.mpf(2) ** (((_bits(float(p)) >> 52) & 0x7FF) - 1023))
                              for p in P)) - s)
            err = float(abs(mp.mpf(got) - want) / want) / U53
            worst = max(worst, err)
            assert err <= x + len(P) + 4, (s, list(P), got, float(want), err)
    assert worst > 1.0


def test_cos_turns_against_high_precision(bits_exe, tables, mp):
    rng = np.random.default_rng(8)
    ts = list(rng.uniform(-4000.0, 4000.0, 1500)) + list(rng.uniform(-25.0, 25.0, 1500))
    ts += [0.0, 1 / 512, -1 / 512, 0.25, 0.5, 1.0, 1 / 256 * 0.5, 4095.9, 4096.0, 5000.3, -7777.25, 1e9 + 0.1, 2.0 ** 39 + 0.3]
    out = _run(bits_exe, tables, [f"C {_bits(t)}" for t in ts])
    with mp.workprec(400):
        for t, line in zip(ts, out):
            got = _from_bits(int(line))
            want = mp.cos(2 * mp.pi * mp.mpf(t))
            assert float(abs(mp.mpf(got) - want)) <= 2 * U53, (t, got, float(want))
