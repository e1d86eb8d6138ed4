"""Pins of the oracle's weight generator and parameter layout."""
import os

import numpy as np
import pytest

import synth
from oracle import weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_reference_outputs():
    ref = [int(x) for x in open(GOLDEN) if x.strip() and not x.startswith("#")]
    got = [int(v) for v in weights.stream(1234567, 5)]
    assert got == ref


def test_uniform_unit_variance():
    w = weights.tensor_uniform(42, 3, 1_000_000)
    assert w.min() >= -np.sqrt(3) and w.max() < np.sqrt(3)
    assert abs(w.mean()) < 5e-3
    assert abs(w.var() - 1.0) < 5e-3


def test_tensor_streams_independent_and_reproducible():
    a = weights.tensor_uniform(42, 0, 1000)
    b = weights.tensor_uniform(42, 1, 1000)
    c = weights.tensor_uniform(43, 0, 1000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1 and abs(np.corrcoef(a, c)[0, 1]) < 0.1
    np.testing.assert_array_equal(a, weights.tensor_uniform(42, 0, 1000))
    # element k of a tensor does not depend on how many elements are drawn
    np.testing.assert_array_equal(a[:10], weights.tensor_uniform(42, 0, 10))


@pytest.mark.parametrize("name,paper", [("fm64", 44.4e3), ("fm256", 690e3), ("fm512", 2.6e6)])
def test_parameter_count_near_table1(name, paper):
    """Loose structural pin: Table 1 of the paper prints 44.4K / 690K / 2.6M parameters.

    The count of this reading (89 one-hot species rows in the first two-body layer,
    8 radial functions, (lmax+1)*C environment weights, per-channel path weights) lands
    within 6% of each printed figure."""
    n = weights.count_params(synth.preset(name))
    assert abs(n - paper) / paper < 0.06, n
