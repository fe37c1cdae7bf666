"""Scaling between recursive steps (each first-level pair (S_r, T_r)
inside-scaled as its own product) against the oracle."""
import numpy as np
import pytest
import torch

from gpu_common import U_LEAF, assert_within, dev_values, max_terms, oracle_tree, require_gpu, to_dev
from oracle import fmm as OF
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu

PLANS2 = [["strassen", "strassen"], ["winograd", "winograd"], ["strassen", "classical121"],
          ["winograd", "strassen"], ["strassen", "fast323"]]


@pytest.fixture(scope="module")
def api():
    return require_gpu()


@pytest.mark.parametrize("names", PLANS2, ids=lambda n: "-".join(n))
@pytest.mark.parametrize("leaf", ["bf16x3", "bf16", "fp16"])
@pytest.mark.parametrize("steps", ["", "OI"])
def test_between_within_tolerance(api, names, leaf, steps):
    M, K, N = 520, 384, 456
    A, B = inputs.diag_scaled_pair(M, K, N, seed=71, span=4.0 if leaf == "fp16" else 12.0)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan(names, leaf, "pass", between=True)
    if steps:
        eA, d, eB = api.scale(Ad, Bd, steps)
        got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
        st = OS.pow2_repeated(A64, B64, steps)
        Ap, Bp = OS.pow2_apply(A64, B64, st.eA, st.d, st.eB)
        G = OS.pow2_unscale(OF.growth(Ap, Bp, oracle_tree(names), between=True), st.eA, st.eB)
    else:
        got = dev_values(api.multiply(plan, Ad, Bd))
        G = OF.growth(A64, B64, oracle_tree(names), between=True)
    api.sync_status()
    C = A64 @ B64  # the scaling cancels exactly: the exact fast product is the exact product
    assert_within(got, C, G, names, K, leaf, f"between {names} {leaf} {steps}")


def test_between_rescues_fp16_range(api):
    # Columns of A spread by 2^18 against rows of B by 2^-18: the first-level
    # sums S_r, T_r leave the fp16 range unless each pair is rescaled.  With
    # the between-steps scaling every leaf operand is a small multiple of a
    # power of two, exact in fp16, so the result is the classical product
    # exactly; without it, the leaf operands overflow.
    names = ["strassen", "strassen"]
    M = K = N = 256
    rng = np.random.default_rng(3)
    # the exponent depends on the column's index inside its first-level
    # block, so each first-level sum adds entries of one magnitude
    s = np.where((np.arange(K) % (K // 2)) % 3 == 0, 18, 0)
    A = rng.integers(-4, 5, size=(M, K)).astype(np.float64) * np.exp2(s)[None, :]
    B = rng.integers(-4, 5, size=(K, N)).astype(np.float64) * np.exp2(-s)[:, None]
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    with_b = dev_values(api.multiply(api.Plan(names, "fp16", "pass", between=True), Ad, Bd))
    without = dev_values(api.multiply(api.Plan(names, "fp16", "pass"), Ad, Bd))
    api.sync_status()
    assert np.array_equal(with_b, A @ B)
    assert not np.array_equal(without, A @ B)


def test_between_is_a_noop_below_two_levels_and_refused_where_unsupported(api):
    from paper_1507_00687_gb300 import _native as N
    A = to_dev(inputs.uniform((192, 160), -1, 1, seed=1), "f32")
    B = to_dev(inputs.uniform((160, 128), -1, 1, seed=2), "f32")
    one = dev_values(api.multiply(api.Plan(["winograd"], "bf16x3", "pass", between=True), A, B))
    ref = dev_values(api.multiply(api.Plan(["winograd"], "bf16x3", "pass"), A, B))
    assert np.array_equal(one, ref)
    with pytest.raises(N.FmmError) as e:
        api.multiply(api.Plan(["strassen", "strassen"], "bf16x3", "load_stage", between=True), A, B)
    assert e.value.code == 10
    with pytest.raises(N.FmmError) as e:
        api.Batch([(api.Plan(["strassen", "strassen"], "bf16x3", between=True), A, B,
                    torch.empty((192, 128), device="cuda"))], "")
    assert e.value.code == 10
