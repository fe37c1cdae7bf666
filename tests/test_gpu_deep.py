"""Deep plans (more C blocks than the stored-products pass keeps on chip):
the products are stored and the output pass gathers per C block."""
import numpy as np
import pytest

from gpu_common import assert_within, dev_values, oracle_reference, require_gpu, to_dev
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return require_gpu()


@pytest.mark.parametrize("names", [["strassen"] * 4, ["winograd", "strassen", "strassen", "classical121"],
                                   ["strassen"] * 5, ["fast323", "fast323"]], ids=lambda n: "-".join(n))
@pytest.mark.parametrize("schedule", ["pass_products", "pass_epilogue"])
def test_deep_plan_within_tolerance(api, names, schedule):
    M, K, N = 333, 290, 301
    A = inputs.uniform((M, K), -1, 1, seed=21)
    B = inputs.uniform((K, N), -1, 1, seed=22)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    got = dev_values(api.multiply(api.Plan(names, "bf16x3", schedule), Ad, Bd))
    api.sync_status()
    C, G = oracle_reference(A64, B64, names)
    assert_within(got, C, G, names, K, "bf16x3", f"{names} {schedule}")


@pytest.mark.parametrize("L", [4, 5, 6])
def test_deep_strassen_integer_exact(api, L):
    # six levels of Strassen on a 200 x 200 problem: 117649 leaves of 4 x 4
    # blocks, 4096 C blocks
    n = 200
    A = inputs.integers((n, n), -2, 2, seed=L)
    B = inputs.integers((n, n), -2, 2, seed=L + 10)
    for schedule in ("pass_products", "pass"):
        got = api.multiply(api.Plan(["strassen"] * L, "bf16x3", schedule), to_dev(A, "f32"), to_dev(B, "f32"))
        api.sync_status()
        assert np.array_equal(dev_values(got), A @ B), (L, schedule)


def test_deep_scaled_between(api):
    names = ["strassen"] * 4
    M = K = N = 320
    A, B = inputs.diag_scaled_pair(M, K, N, seed=5, span=10.0)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    eA, d, eB = api.scale(Ad, Bd, "OI")
    got = dev_values(api.multiply(api.Plan(names, "bf16x3", "pass_products"), Ad, Bd, eA, d, eB))
    api.sync_status()
    from oracle import scaling as OS
    st = OS.pow2_repeated(A64, B64, "OI")
    C, G = oracle_reference(A64, B64, names, st.eA, st.d, st.eB)
    assert_within(got, C, G, names, K, "bf16x3", "deep scaled")
