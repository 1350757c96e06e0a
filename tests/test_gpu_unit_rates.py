"""The unit-rate microbenchmarks (mcubes_unit_rates): every rate positive and below the SM's
issue limit (128 lanes a clock), and the orderings the V-Sample design rests on: u32 shared
atomics into 8 lane-interleaved copies beat FP32 shared atomics into one copy, and FP64 runs far
below FP32."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_unit_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05730_gb300 import capi
    r = capi.unit_rates()
    assert set(r) == set(capi.UNIT_RATE_NAMES)
    for k, v in r.items():
        assert 0.0 < v <= 130.0, (k, v)
    assert r["ffma_lanes"] > 60.0
    assert r["dfma_lanes"] < r["ffma_lanes"] / 8
    assert r["shared_atomic_u32x8_lanes"] > r["shared_atomic_f32_lanes"]
    assert r["philox_calls"] > 0.2
