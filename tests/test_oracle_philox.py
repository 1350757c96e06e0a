"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11) against something other than
itself: the CUDA toolkit's cuRAND host generator (run as a library, on the CPU) and the
statistics every uniform generator must have."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cuda_home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for path in (os.path.join(cuda_home, "lib64", "libcurand.so"), ctypes.util.find_library("curand")):
        if not path:
            continue
        try:
            return ctypes.CDLL(path)
        except OSError:
            pass
    return None


@pytest.fixture(scope="module")
def curand_host():
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    st = lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10)
    if st != 0:
        pytest.skip(f"curandCreateGeneratorHost returned {st}")

    def draw(seed, offset, n=4):
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint * max(n, 4))()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(max(n, 4))) == 0
        return [int(v) for v in buf][:n]

    yield draw
    lib.curandDestroyGenerator(gen)


# The host generator lays its stream out as 2^16 interleaved Philox streams: output block b
# (4 words) is Philox4x32-10 of counter (b >> 16 as a 64-bit number in words 0-1,
# b mod 2^16 in word 2, 0) under key (seed mod 2^32, seed >> 32). Observed by running it.
# Offsets are 64-bit word counts, so blocks stay below 2^62.
def _host_counter(block):
    pos, lane = block >> 16, block & 0xFFFF
    return [pos & 0xFFFFFFFF, pos >> 32, lane, 0]


SEEDS = [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0x00000000DEADBEEF, 0xCAFEF00D00000000]
BLOCKS = [0, 1, 7, 0xFFFF, 0x10000, 0x12345, (5 << 16) | 77, (0xFFFFFFFF << 16) | 3,
          (0x1_0000_0001 << 16) | 0xABCD, (0x3FFF_FFFF_FFFF << 16) | 0xFFFF]


@pytest.mark.parametrize("seed", SEEDS)
def test_philox_matches_curand_host_generator(curand_host, seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for blk in BLOCKS:
        want = curand_host(seed, 4 * blk)
        got = oracle.philox(_host_counter(blk), key)
        assert got == want, (hex(seed), hex(blk))


def _uniforms(layout_fp32, n_cubes=4096, d=8):
    """The oracle's uniforms for the first n_cubes sub-cubes (n = 2 * 3^d: g = 3, p = 2)."""
    pts = oracle.sample_points(oracle.ADDITION, d, np.zeros(2 * d), 2 * 3 ** d, seed=99,
                               mode=1 if layout_fp32 else 0, t0=0, t1=n_cubes)
    return pts["u"]


@pytest.mark.parametrize("fp32", [False, True])
def test_uniform_statistics(fp32):
    u = _uniforms(fp32)
    assert u.min() >= 0.0 and u.max() < 1.0
    n = u.size
    # mean 1/2, variance 1/12, within 5 standard errors
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    # no correlation between axes or between the two samples of a cube
    c = np.corrcoef(u.T)
    off = c[~np.eye(c.shape[0], dtype=bool)]
    assert np.abs(off).max() < 6 / np.sqrt(u.shape[0])
    lag = np.corrcoef(u[0::2].ravel(), u[1::2].ravel())[0, 1]
    assert abs(lag) < 6 / np.sqrt(u.size / 2)
    # resolution of the layout: 2^-23 (FP32) or 2^-52 (FP64)
    step = 2.0 ** -23 if fp32 else 2.0 ** -52
    assert np.all(np.mod(u / step, 1.0) == 0.0)
    if not fp32:
        assert np.any(np.mod(u / 2.0 ** -40, 1.0) != 0.0)  # really uses the low bits


def test_counter_fields_change_the_stream():
    base = oracle.philox([5, 6, 7, 8], [9, 10])
    for w in range(4):
        ctr = [5, 6, 7, 8]
        ctr[w] ^= 1
        assert oracle.philox(ctr, [9, 10]) != base
    assert oracle.philox([5, 6, 7, 8], [9, 11]) != base
    assert oracle.philox([5, 6, 7, 8], [8, 10]) != base
