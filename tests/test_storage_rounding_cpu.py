"""Pins of the 16-bit rounding the tensor-core trajectory tests apply to G_off
before running the oracle: values fixed by the IEEE FP16 and BF16 formats."""
import numpy as np
import pytest

from storage_rounding import round_to_storage


def test_bf16_round_to_nearest_even():
    u = 2.0 ** -7  # BF16 spacing in [1, 2): 8 significant bits
    x = np.array([1.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2.0 ** -20, -(1 + 3 * u / 2), 0.0])
    # ties go to the even neighbour (1 and 1 + 2u), just above a tie rounds up
    want = np.array([1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 0.0])
    np.testing.assert_array_equal(round_to_storage(x, "bf16"), want)
    # a small normal value keeps 8 significant bits (relative error <= 2^-9)
    assert abs(round_to_storage(3.0e-30, "bf16") - 3.0e-30) <= 3.0e-30 * 2.0 ** -9


def test_fp16_round_to_nearest_even_and_subnormals():
    u = 2.0 ** -10  # FP16 spacing in [1, 2)
    x = np.array([1 + u / 2, 1 + 3 * u / 2, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 65504.0, 65520.0])
    with np.errstate(over="ignore"):
        got = round_to_storage(x, "fp16")
    assert got[0] == 1.0 and got[1] == 1 + 2 * u
    assert got[2] == 2.0 ** -24            # smallest subnormal
    assert got[3] == 0.0                   # half of it: tie to even (zero)
    assert got[4] == 2.0 ** -24            # 0.75 of it rounds up
    assert got[5] == 65504.0 and np.isinf(got[6])


@pytest.mark.parametrize("precision,bits", [("fp16", 11), ("bf16", 8)])
def test_relative_error_bound_on_random_values(precision, bits):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000) * 0.05
    x = x[np.abs(x) > 1e-4]  # normal range of both types
    r = round_to_storage(x, precision)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -bits)
    assert np.all(round_to_storage(r, precision) == r)  # idempotent
