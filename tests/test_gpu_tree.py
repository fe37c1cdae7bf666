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
SCHEDULES = ["load_stage", "pass_epilogue", "pass_products", "pass_accumulate"]
# schedules whose results are the same from run to run
DETERMINISTIC = ["load_stage", "pass_epilogue", "pass_products"]


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
    for schedule in DETERMINISTIC:
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


# ---------------------------------------------------------------- Castrapel-Gustafson variants (Sec. 3.4)

def _cg_max_terms(name, levels):
    r = OR.principal(OR.winograd() if name == "winograd" else OR.strassen())
    return int(max(r.alpha.max(), r.beta.max(), r.gamma.max())) ** levels


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_block_max_exact(api, dt):
    # fmm_block_max against the oracle's block max-abs on ragged grids
    from oracle import variants as CG
    for (M, K), (nrb, ncb) in (((300, 260), (4, 4)), ((37, 513), (8, 2)), ((5, 7), (8, 8)), ((1000, 64), (2, 16))):
        X = inputs.uniform((M, K), -3, 3, seed=M * K)
        X[M // 3, K // 5] = 40.0
        Xd = to_dev(X, dt)
        got = api.block_max(Xd, nrb, ncb).cpu().numpy().astype(np.float64)
        assert np.array_equal(got, CG.block_max(dev_values(Xd), nrb, ncb)), (M, K, nrb, ncb)


@pytest.mark.parametrize("name", ["strassen", "winograd"])
@pytest.mark.parametrize("selection", ["random", "round_robin", "matrix"])
@pytest.mark.parametrize("leaf", ["bf16x3", "bf16"])
def test_variant_plans_against_oracle(api, name, selection, leaf):
    # Two-level Castrapel-Gustafson plans: the library's choice per node is
    # the oracle's (for the matrix-dependent one, from the block maxima the
    # GPU found on the scaled-row/column inputs), and the product is within
    # tolerance of the oracle's product over the same tree; integer inputs
    # give the classical product exactly.
    from oracle import variants as CG
    levels = 2
    M, K, N = 610, 530, 470
    A, B = inputs.diag_scaled_pair(M, K, N, seed=91)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan.variants(name, levels, selection, seed=2024, A=Ad, B=Bd, leaf=leaf)
    base = OR.winograd() if name == "winograd" else OR.strassen()
    if selection == "random":
        want = CG.select_random(7, levels, 2024)
    elif selection == "round_robin":
        want = CG.select_round_robin(7, levels)
    else:
        g = 1 << levels
        want = CG.select_matrix(base, levels, CG.block_max(A64, g, g), CG.block_max(B64, g, g))
    assert plan.chosen == want
    orc = CG.tree(base, levels, want)
    got = dev_values(api.multiply(plan, Ad, Bd))
    api.sync_status()
    _, pk, _ = OF.dims(orc)
    kl = -(-K // pk)
    tol = (U_LEAF[leaf] + (kl + 2 * _cg_max_terms(name, levels) + 8) * 2.0**-23) * OF.growth(A64, B64, orc)
    bad = np.abs(got - OF.fmm(A64, B64, orc)) > tol
    assert not bad.any(), f"{name} {selection} {leaf}: {bad.sum()} entries outside tolerance"
    Ai = inputs.integers((M, K), -4, 4, seed=1)
    Bi = inputs.integers((K, N), -4, 4, seed=2)
    exact = dev_values(api.multiply(plan, to_dev(Ai, "f32" if leaf == "bf16x3" else "bf16"),
                                    to_dev(Bi, "f32" if leaf == "bf16x3" else "bf16")))
    api.sync_status()
    assert np.array_equal(exact, Ai @ Bi)
