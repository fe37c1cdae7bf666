"""The small configuration of the benchmark description on the GPU:
Strassen with two levels, n = 256, U[-1, 1] (ten seeded trials), against the
oracle elementwise and under the first-order bound of Theorem 4.1; and
n = 16 with integer entries in [-4, 4], exact."""
import numpy as np
import pytest

from gpu_common import assert_within, dev_values, oracle_reference, require_gpu, to_dev
from oracle import fmm as OF
from oracle import rules as OR
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu

NAMES = ["strassen", "strassen"]


@pytest.fixture(scope="module")
def api():
    return require_gpu()


@pytest.mark.parametrize("leaf", ["bf16x3", "bf16", "fp16"])
def test_strassen_two_levels_n256_trials(api, leaf):
    plan = api.Plan(NAMES, leaf)
    s = OR.strassen()
    eps = {"bf16x3": 3 * 2.0**-16, "bf16": 2.0**-8, "fp16": 2.0**-11}[leaf]
    for trial in range(10):
        n = 256
        A = inputs.uniform((n, n), -1, 1, seed=1507 + trial)
        B = inputs.uniform((n, n), -1, 1, seed=1507 + 100 + trial)
        Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
        A64, B64 = dev_values(Ad), dev_values(Bd)
        got = dev_values(api.multiply(plan, Ad, Bd))
        api.sync_status()
        C, G = oracle_reference(A64, B64, NAMES)
        assert_within(got, C, G, NAMES, n, leaf, f"trial {trial}")
        # Theorem 4.1 (first order): (K/4 + 2Q)(K/4) E^2 ||A|| ||B|| eps
        bound = OF.bound_uniform([s, s], n, np.abs(A64).max(), np.abs(B64).max(), eps)
        assert np.abs(got - A64 @ B64).max() <= bound


def test_strassen_two_levels_n16_integers_exact(api):
    for trial in range(10):
        A = inputs.integers((16, 16), -4, 4, seed=1507 + trial)
        B = inputs.integers((16, 16), -4, 4, seed=1507 + 50 + trial)
        # Strassen sums at most two blocks per level: |S|, |T| <= 16, integers
        # of at most 4 significant bits, exact in every leaf format (E4M3
        # after its power-of-two block scale too); products and sums < 2^24
        for dt, leaf in (("f32", "bf16x3"), ("bf16", "bf16"), ("f16", "fp16"), ("f32", "e4m3b128")):
            got = api.multiply(api.Plan(NAMES, leaf), to_dev(A, dt), to_dev(B, dt))
            api.sync_status()
            assert np.array_equal(dev_values(got), A @ B), (trial, dt, leaf)
