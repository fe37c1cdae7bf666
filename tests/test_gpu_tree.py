"""Non-uniform plans (Sec. 3.4) and rotated <3,2,3> rules (App. B) on the
GPU against the oracle's recursion trees, through the C ABI."""
import numpy as np
import pytest

import tree_cases as TC
from gpu_common import U_LEAF, dev_values, require_gpu, to_dev
from oracle import fmm as OF
from oracle import rules as OR
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu

TREES = {"dalberto": TC.dalberto(), "fast323_nonuniform": TC.fast323_nonuniform(), "mixed_rank": TC.mixed_rank(),
         "fast323_then_rot1": ["F", ["F_r1"] * 15], "rot2_then_S": ["F_r2", ["S"] * 15]}
SCHEDULES = ["load_stage", "pass_epilogue", "pass_products"]


@pytest.fixture(scope="module")
def api():
    return require_gpu()


def _tol(G, orc, K, leaf):
    _, pk, _ = OF.dims(orc)
    kl = -(-K // pk)
    return (U_LEAF[leaf] + (kl + 2 * TC.max_terms(orc) + 8) * 2.0**-23) * G


def _check(got, C, G, orc, K, leaf, what):
    tol = _tol(G, orc, K, leaf)
    bad = np.abs(got - C) > tol
    assert not bad.any(), f"{what}: {bad.sum()} entries outside tolerance"


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("tree", list(TREES))
def test_tree_integer_inputs_bit_exact(api, schedule, tree):
    lib, orc = TC.two_level(*TREES[tree])
    pm, pk, pn = OF.dims(orc)
    # ragged sizes: several tiles per leaf block plus padding on every side
    M, K, N = 37 * pm + 5, 29 * pk + 3, 41 * pn + 7
    A = inputs.integers((M, K), -4, 4, seed=M)
    B = inputs.integers((K, N), -4, 4, seed=N)
    for dt, leaf in (("f32", "bf16x3"), ("bf16", "bf16"), ("f16", "fp16")):
        plan = api.Plan.tree(lib, leaf, schedule)
        got = api.multiply(plan, to_dev(A, dt), to_dev(B, dt))
        api.sync_status()
        assert np.array_equal(dev_values(got), A @ B), (tree, dt, leaf)
    # the oracle's tree gives the same exact result
    assert np.array_equal(OF.fmm(A, B, orc), A @ B)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("tree", list(TREES))
@pytest.mark.parametrize("leaf", ["bf16x3", "bf16"])
def test_tree_within_tolerance(api, schedule, tree, leaf):
    lib, orc = TC.two_level(*TREES[tree])
    M, K, N = 610, 530, 470
    A = inputs.uniform((M, K), -1, 1, seed=81)
    B = inputs.uniform((K, N), -1, 1, seed=82)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    got = dev_values(api.multiply(api.Plan.tree(lib, leaf, schedule), Ad, Bd))
    api.sync_status()
    _check(got, OF.fmm(A64, B64, orc), OF.growth(A64, B64, orc), orc, K, leaf, f"{tree} {leaf}")


def test_tree_one_rule_per_level_matches_uniform_plan_bitwise(api):
    # The tree with one rule per level flattens to the same leaves in the
    # same order as the uniform plan, so every kernel sees the same work.
    lib, _ = TC.two_level("Wg", ["S"] * 7)
    A = to_dev(inputs.uniform((300, 260), -1, 1, seed=3), "f32")
    B = to_dev(inputs.uniform((260, 330), -1, 1, seed=4), "f32")
    for schedule in SCHEDULES:
        t = api.multiply(api.Plan.tree(lib, "bf16x3", schedule), A, B)
        u = api.multiply(api.Plan(["winograd", "strassen"], "bf16x3", schedule), A, B)
        api.sync_status()
        assert np.array_equal(dev_values(t), dev_values(u)), schedule


@pytest.mark.parametrize("tree", ["dalberto", "fast323_nonuniform"])
@pytest.mark.parametrize("steps", ["", "OI"])
def test_tree_scaled_and_between(api, tree, steps):
    # outside-inside scaling (Alg. 3) and scaling between the recursive
    # steps compose with a non-uniform tree as with a uniform plan
    lib, orc = TC.two_level(*TREES[tree])
    M, K, N = 420, 380, 400
    A, B = inputs.diag_scaled_pair(M, K, N, seed=91, span=12.0)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    for between in (False, True):
        plan = api.Plan.tree(lib, "bf16x3", "pass", between=between)
        if steps:
            eA, d, eB = api.scale(Ad, Bd, steps)
            got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
            st = OS.pow2_repeated(A64, B64, steps)
            Ap, Bp = OS.pow2_apply(A64, B64, st.eA, st.d, st.eB)
            G = OS.pow2_unscale(OF.growth(Ap, Bp, orc, between=between), st.eA, st.eB)
        else:
            got = dev_values(api.multiply(plan, Ad, Bd))
            G = OF.growth(A64, B64, orc, between=between)
        api.sync_status()
        _check(got, A64 @ B64, G, orc, K, "bf16x3", f"{tree} between={between} {steps}")


def _grad_tree(orc, fn):
    if orc is None:
        return None
    return OF.Node(fn(orc.rule), [_grad_tree(c, fn) for c in orc.children])


@pytest.mark.parametrize("tree", ["dalberto", "mixed_rank", "fast323_then_rot1"])
def test_tree_backward(api, tree):
    lib, orc = TC.two_level(*TREES[tree])
    M, K, N = 330, 290, 350
    A = inputs.uniform((M, K), -1, 1, seed=61)
    B = inputs.uniform((K, N), -1, 1, seed=62)
    G0 = inputs.uniform((M, N), -1, 1, seed=63)
    Ad, Bd, dC = to_dev(A, "bf16"), to_dev(B, "bf16"), to_dev(G0, "f32")
    A64, B64, dC64 = dev_values(Ad), dev_values(Bd), dev_values(dC)
    dA, dB = api.multiply_backward(api.Plan.tree(lib, "bf16x3"), dC, Ad, Bd)
    api.sync_status()
    ra, rb = _grad_tree(orc, OR.rule_for_dA), _grad_tree(orc, OR.rule_for_dB)
    _check(dev_values(dA), dC64 @ B64.T, OF.growth(dC64, B64.T, ra), ra, N, "bf16x3", "dA")
    _check(dev_values(dB), A64.T @ dC64, OF.growth(A64.T, dC64, rb), rb, M, "bf16x3", "dB")


def test_tree_e4m3_leaves_integer_exact(api):
    lib, orc = TC.two_level(*TREES["dalberto"])
    M, K, N = 300, 520, 260
    A = inputs.integers((M, K), -3, 3, seed=5)
    B = inputs.integers((K, N), -3, 3, seed=6)
    got = api.multiply(api.Plan.tree(lib, "e4m3b128", "pass"), to_dev(A, "f32"), to_dev(B, "f32"))
    api.sync_status()
    assert np.array_equal(dev_values(got), A @ B)


def test_rotated_rules_one_level(api):
    # each rotation of <3,2,3;15> is a rule of its own shape; on the GPU it
    # must agree with the oracle's rotation
    for lab in ("F_r1", "F_r2"):
        pr, orr = TC.package_rule(lab), TC.oracle_rule(lab)
        orc = OF.uniform([orr])
        M, K, N = 401, 377, 389
        A = inputs.uniform((M, K), -1, 1, seed=11)
        B = inputs.uniform((K, N), -1, 1, seed=12)
        Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
        A64, B64 = dev_values(Ad), dev_values(Bd)
        for schedule in SCHEDULES:
            got = dev_values(api.multiply(api.Plan([pr], "bf16x3", schedule), Ad, Bd))
            api.sync_status()
            _check(got, OF.fmm(A64, B64, orc), OF.growth(A64, B64, orc), orc, K, "bf16x3", f"{lab} {schedule}")
