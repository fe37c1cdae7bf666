"""Host-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host plan compiler (Brent check, flattening,
principal quantities, bound) agrees with the oracle.  No GPU calls."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import fmm as OF
from oracle import rules as OR
from paper_1507_00687_gb300 import build as B
from paper_1507_00687_gb300 import rules as PR

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    B.build()
    from paper_1507_00687_gb300 import _native
    return _native


def header_symbols():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|fmm_status)\s*(fmm_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_header_symbol(native):
    syms = header_symbols()
    assert len(syms) >= 14
    assert sorted(native.EXPORTS) == syms
    L = native.lib()
    for s in syms:
        assert hasattr(L, s)
    assert b"sm_103a" in L.fmm_version()


def _plan(native, rules, leaf="bf16"):
    from paper_1507_00687_gb300 import api
    return api.Plan(rules, leaf)


def _oracle_rule(name):
    return {"strassen": OR.strassen, "winograd": OR.winograd, "fast323": OR.fast323,
            "classical121": lambda: OR.classical(1, 2, 1), "classical211": lambda: OR.classical(2, 1, 1),
            "classical222": lambda: OR.classical(2, 2, 2)}[name]()


@pytest.mark.parametrize("names", [["strassen"], ["winograd"], ["fast323"], ["strassen", "strassen"],
                                   ["winograd", "classical121", "winograd"], ["strassen", "fast323"],
                                   ["classical222"], []])
def test_plan_info_matches_oracle(native, names):
    p = _plan(native, names)
    info = p.info()
    orules = [_oracle_rule(n) for n in names]
    assert info["q_sum"] == sum(OR.principal(r).Q for r in orules)
    assert info["e_prod"] == float(np.prod([OR.principal(r).E for r in orules])) if orules else 1.0
    assert info["leaves"] == int(np.prod([r.R for r in orules])) if orules else 1
    pm, pk, pn = OF.dims(OF.uniform(orules))
    assert (info["pm"], info["pk"], info["pn"]) == (pm, pk, pn)
    # flattened nnz = product over levels of each rule's per-operand nnz sums
    if orules:
        want = 1
        nU = np.prod([(r.U != 0).sum() for r in orules])
        nV = np.prod([(r.V != 0).sum() for r in orules])
        nW = np.prod([(r.W != 0).sum() for r in orules])
        assert info["nnz"] == nU + nV + nW
    K = 4096
    b = p.bound(K, 1.0, 1.0, 2.0**-24)
    assert b == pytest.approx(OF.bound_uniform(orules, K, 1.0, 1.0, 2.0**-24))


def test_plan_rejects_non_matmul(native):
    from paper_1507_00687_gb300 import api
    s = PR.strassen()
    bad = PR.BaseRule("bad", 2, 2, 2, s.U, s.V, s.W, PR.COL, PR.COL, PR.ROW)  # the stated ordering
    with pytest.raises(native.FmmError) as e:
        api.Plan([bad])
    assert e.value.code == 2
    W = s.W.copy()
    W[0, 0] = -1
    with pytest.raises(native.FmmError):
        api.Plan([PR.BaseRule("bad2", 2, 2, 2, s.U, s.V, W, s.order_a, s.order_b, s.order_c)])


def test_plan_rejects_bad_args(native):
    L = native.lib()
    h = C.c_void_p()
    assert L.fmm_plan(None, 1, None, 0) == 1
    assert L.fmm_plan(C.byref(h), -1, None, 0) == 1
    assert L.fmm_plan(C.byref(h), 0, None, 7) == 1
    assert L.fmm_plan_info(None, None, None, None, None, None, None, None) == 1
    # unsupported flattening: Winograd^4 needs 256 terms per operand (the
    # limit is 64, which Winograd^3 reaches)
    from paper_1507_00687_gb300 import api
    assert api.Plan(["winograd"] * 3).info()["leaves"] == 343
    with pytest.raises(native.FmmError) as e:
        api.Plan(["winograd"] * 4)
    assert e.value.code == 10


def test_status_strings(native):
    L = native.lib()
    for code in range(11):
        assert len(L.fmm_status_string(code)) > 0


def test_package_rules_match_oracle_tables():
    # The package and the oracle hold separate copies of the printed tables.
    for name, orule in (("strassen", OR.strassen()), ("winograd", OR.winograd()), ("fast323", OR.fast323())):
        pr = PR.get(name)
        assert np.array_equal(pr.U, orule.U) and np.array_equal(pr.V, orule.V) and np.array_equal(pr.W, orule.W)
        assert (pr.order_a, pr.order_b, pr.order_c) == tuple(0 if o == "row" else 1 for o in
                                                             (orule.order_a, orule.order_b, orule.order_c))


# ---------------------------------------------------------------- non-uniform plans (Sec. 3.4)

def _tree_plan(desc, leaf="bf16"):
    import tree_cases as TC
    from paper_1507_00687_gb300 import api
    lib, orc = TC.two_level(*desc)
    return api.Plan.tree(lib, leaf), orc


def test_tree_plan_dalberto_growth_factor(native):
    # The Sec. 3.4 example: the variant at three level-2 nodes lowers the
    # largest two-level growth factor of Strassen; the library's max xi_k
    # must equal the oracle's (pinned to the printed value in the oracle
    # tests), and max delta_k likewise.
    import tree_cases as TC
    plan, orc = _tree_plan(TC.dalberto())
    info = plan.info()
    assert info["leaves"] == 49
    assert info["e_prod"] == float(OF.xi_vector(orc).max())
    assert info["q_sum"] == float(OF.delta_vector(orc).max())
    uni = _plan(native, ["strassen", "strassen"]).info()
    assert info["e_prod"] < uni["e_prod"]
    assert (info["pm"], info["pk"], info["pn"]) == (4, 4, 4)
    b = plan.bound(4096, 1.0, 1.0, 2.0**-24)
    assert b == pytest.approx(OF.bound_tree(orc, 4096, 1.0, 1.0, 2.0**-24))


def test_tree_plan_fast323_nonuniform(native):
    import tree_cases as TC
    plan, orc = _tree_plan(TC.fast323_nonuniform())
    info = plan.info()
    assert info["leaves"] == 225
    assert info["e_prod"] == float(OF.xi_vector(orc).max())
    assert info["q_sum"] == float(OF.delta_vector(orc).max())
    assert (info["pm"], info["pk"], info["pn"]) == (9, 4, 9)


def test_tree_plan_with_one_rule_per_level_equals_uniform(native):
    # A tree whose levels each repeat one rule is the uniform plan: same
    # leaves, terms, quantities.
    import tree_cases as TC
    for desc, names in ((["S", ["S"] * 7], ["strassen", "strassen"]), (["Wg", ["S"] * 7], ["winograd", "strassen"])):
        t = _tree_plan(desc)[0].info()
        u = _plan(native, names).info()
        assert t == u, (desc, t, u)


def test_tree_plan_mixed_ranks(native):
    import tree_cases as TC
    plan, orc = _tree_plan(TC.mixed_rank())
    info = plan.info()
    assert info["leaves"] == 5 * 7 + 2 * 8
    assert info["e_prod"] == float(OF.xi_vector(orc).max())
    assert info["q_sum"] == float(OF.delta_vector(orc).max())
    # the between-steps scaling needs equal ranks on every level
    assert native.lib().fmm_plan_set_between_scaling(plan.handle, 1) == 10
    assert native.lib().fmm_plan_set_between_scaling(_tree_plan(TC.dalberto())[0].handle, 1) == 0


def test_tree_plan_delta_follows_the_feeding_products(native):
    # max_k delta_k (Sec. 4.5) takes, for each C block, only the products
    # that add into it: here the deep child sits under Winograd's m2, which
    # adds into c11 alone (2 terms), so the maximum is 2 + 12 = 4 + 10 = 14,
    # not the largest gamma plus the largest child (4 + 12 = 16).
    import tree_cases as TC
    plan, orc = _tree_plan(TC.uneven_delta())
    assert float(OF.delta_vector(orc).max()) == 14.0
    assert plan.info()["q_sum"] == 14.0


def test_tree_plan_rejects_bad_trees(native):
    from paper_1507_00687_gb300 import api
    L = native.lib()
    s, f = PR.strassen(), PR.fast323()
    plan = api.Plan([s])  # keeps the rule arrays alive
    arr = plan._rule_array([s, f])
    h = C.c_void_p()
    nodes = (C.c_int32 * 9)(*([0] * 9))
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 2, 8, nodes, 0) == 0
    L.fmm_plan_destroy(h)
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 2, 7, nodes, 0) == 1   # too few nodes
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 2, 9, nodes, 0) == 1   # too many
    bad = (C.c_int32 * 8)(0, 0, 0, 1, 0, 0, 0, 0)                      # <3,2,3> among <2,2,2>
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 2, 8, bad, 0) == 1
    oob = (C.c_int32 * 8)(0, 0, 0, 2, 0, 0, 0, 0)
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 2, 8, oob, 0) == 1
    assert L.fmm_plan_tree(None, 2, arr, 2, 8, nodes, 0) == 1
    assert L.fmm_plan_tree(C.byref(h), 2, arr, 0, 8, nodes, 0) == 1


def test_rotated_rules_accepted_with_invariant_quantities(native):
    # App. A-B: the cyclic rotations of a rule are rules of the rotated
    # shape; Strassen's Q and E are invariant under them.  The library's
    # Brent check accepts the package's rotations, and its Q, E equal the
    # oracle's for the oracle's own rotations.
    import tree_cases as TC
    from paper_1507_00687_gb300 import api
    for lab, shape in (("F_r1", (3, 3, 2)), ("F_r2", (2, 3, 3))):
        pr = TC.package_rule(lab)
        assert (pr.m0, pr.k0, pr.n0) == shape
        info = api.Plan([pr]).info()
        orr = TC.oracle_rule(lab)
        assert info["q_sum"] == OR.principal(orr).Q and info["e_prod"] == OR.principal(orr).E
    s = api.Plan(["strassen"]).info()
    r = api.Plan([PR.rotate(PR.strassen())]).info()
    assert (r["q_sum"], r["e_prod"]) == (s["q_sum"], s["e_prod"])


# ---------------------------------------------------------------- algorithm selection figures (Sec. 5.3)

def test_algorithm_table_matches_table_1(native):
    # Q, E, nnz, R against the Table 1 fixture and the printed stability
    # exponents (two decimals): <2,2,2> classical 1, Strassen 3.58, the
    # Strassen-classical <4,2,2> and <2,4,2> compositions 2.94, <3,2,3> 3.21.
    from paper_1507_00687_gb300 import api
    rows = api.algorithm_table({"classical222": ["classical222"], "strassen": ["strassen"],
                                "strassen*classical211": ["strassen", "classical211"],
                                "strassen*classical121": ["strassen", "classical121"],
                                "fast323": ["fast323"]})
    gold = {r[0]: r for r in (line.split() for line in open(os.path.join(ROOT, "tests", "golden", "table1.txt"))
                              if line.strip() and not line.startswith("#"))}
    printed = {"classical222": 1.0, "strassen": 3.58, "strassen*classical211": 2.94,
               "strassen*classical121": 2.94, "fast323": 3.21}
    for row in rows:
        g = gold[row["name"]]
        assert (row["m0"], row["k0"], row["n0"], row["R"], row["nnz"]) == tuple(int(x) for x in g[1:6])
        assert (row["Q"], row["E"]) == (float(g[6]), float(g[7]))
        assert round(row["stab_exp"], 2) == printed[row["name"]]
        for L in (1, 2, 3, 4):
            base = row["m0"] * row["k0"] * row["n0"]
            assert row["flop_fraction"][L] == pytest.approx((row["R"] / base) ** L)
            assert row["relative_instability"][L] == pytest.approx((row["E"] / row["k0"] ** 2) ** L)


def test_relative_instability_of_plans(native):
    from paper_1507_00687_gb300 import api
    assert api.relative_instability(api.Plan(["strassen", "strassen"])) == 9.0
    assert api.relative_instability(api.Plan(["winograd"])) == 18.0 / 4
    import tree_cases as TC
    lib, orc = TC.two_level(*TC.dalberto())
    assert api.relative_instability(api.Plan.tree(lib)) == 96.0 / 16


def test_package_compose_matches_oracle_compose(native):
    # Package and oracle compose independently; the composite tables (both
    # row-major, product r1 R2 + r2) must agree entry for entry, and the
    # library accepts the composite with the quantities of the two-level plan
    # (same E, leaves, nnz, base case).
    from paper_1507_00687_gb300 import api
    for a, b in (("strassen", "classical211"), ("fast323", "strassen"), ("winograd", "classical121")):
        pc = PR.compose(PR.get(a), PR.get(b))
        oc = OR.compose(_oracle_rule(a), _oracle_rule(b))
        assert np.array_equal(pc.U, oc.U) and np.array_equal(pc.V, oc.V) and np.array_equal(pc.W, oc.W)
        one, two = api.Plan([pc]).info(), api.Plan([a, b]).info()
        for k in ("e_prod", "leaves", "nnz", "pm", "pk", "pn"):
            assert one[k] == two[k], (a, b, k)


# ---------------------------------------------------------------- rule algebra and variants (Sec. 3.4)

def test_rule_algebra_checks_brent(native):
    # The library's transform rejects the D'Alberto variant as printed (it
    # fails the Brent equations, pinned in the oracle tests) and accepts the
    # reading with B's and C's columns exchanged together; permutations
    # must be permutations.
    P = np.array([[0, 1], [1, 0]])
    I2 = np.eye(2)
    s = PR.strassen()
    with pytest.raises(native.FmmError) as e:
        PR.variant(s, np.eye(4), np.kron(P, I2), np.kron(I2, P), "printed")
    assert e.value.code == 2
    good = PR.variant(s, np.eye(4), np.kron(I2, P), np.kron(P, I2), "dalberto")
    # the same rule as exchanging the j blocks
    perm = PR.permute(s, [0, 1], [0, 1], [1, 0], "j-exchanged")
    assert np.array_equal(good.U, perm.U) and np.array_equal(good.V, perm.V) and np.array_equal(good.W, perm.W)
    with pytest.raises(native.FmmError) as e:
        PR.permute(s, [0, 0], [0, 1], [0, 1], "bad")
    assert e.value.code == 1
    with pytest.raises(native.FmmError) as e:
        PR.rotate(PR.variant.__globals__["BaseRule"]("broken", 2, 2, 2, s.U, s.V, -s.W, s.order_a, s.order_b,
                                                       s.order_c))
    assert e.value.code == 2


def test_rotation_matches_oracle(native):
    # the library's rotations are the oracle's (canonical tables equal)
    for name in ("strassen", "winograd", "fast323"):
        lib = PR.get(name)
        orc = _oracle_rule(name)
        for _ in range(3):
            lib, orc = PR.rotate(lib), OR.rotate(orc)
            co = OR.canonical(orc)
            assert (lib.m0, lib.k0, lib.n0) == (co.m0, co.k0, co.n0)
            assert np.array_equal(lib.U, co.U) and np.array_equal(lib.V, co.V) and np.array_equal(lib.W, co.W)


@pytest.mark.parametrize("name", ["strassen", "winograd"])
def test_castrapel_gustafson_variants_match_oracle(native, name):
    from oracle import variants as CG
    for v in range(8):
        lib = PR.castrapel_gustafson(PR.get(name), v)
        orc = OR.canonical(CG.variant(_oracle_rule(name), v))
        assert np.array_equal(lib.U, orc.U) and np.array_equal(lib.V, orc.V) and np.array_equal(lib.W, orc.W), v


@pytest.mark.parametrize("name", ["strassen", "winograd"])
@pytest.mark.parametrize("selection", ["random", "round_robin"])
def test_variant_plans_match_oracle_trees(native, name, selection):
    # fmm_plan_variants picks the same variant per node as the oracle, and
    # its max xi / max delta (Sec. 4.5) equal the oracle's for that tree
    from oracle import variants as CG
    from paper_1507_00687_gb300 import api
    for levels in (1, 2, 3):
        plan = api.Plan.variants(name, levels, selection, seed=1234567, leaf="bf16")
        want = (CG.select_random(7, levels, 1234567) if selection == "random"
                else CG.select_round_robin(7, levels))
        assert plan.chosen == want
        orc = CG.tree(_oracle_rule(name), levels, want)
        info = plan.info()
        assert info["leaves"] == 7**levels
        assert info["e_prod"] == float(OF.xi_vector(orc).max())
        assert info["q_sum"] == float(OF.delta_vector(orc).max())


@pytest.mark.parametrize("name", ["strassen", "winograd"])
def test_matrix_dependent_selection_matches_oracle(native, name):
    # From host block maxima (the values fmm_block_max would give), the
    # library's choice per node equals the oracle's; a dominant block moves
    # the choice away from the variant the uniform input picks.
    import ctypes as C
    from oracle import variants as CG
    from paper_1507_00687_gb300 import api
    g = np.random.default_rng(7)
    rule = PR.get(name)
    for levels in (1, 2, 3):
        n = 1 << levels
        for trial in range(4):
            Amax = g.uniform(0.01, 4.0, (n, n)).astype(np.float32)
            Bmax = g.uniform(0.01, 4.0, (n, n)).astype(np.float32)
            if trial == 1:
                Amax[n - 1, 0] = 1e4
            want = CG.select_matrix(_oracle_rule(name), levels, Amax.astype(np.float64), Bmax.astype(np.float64))
            plan = api.Plan.__new__(api.Plan)
            plan._keep, plan.rules, plan.leaf = [], [rule], "bf16"
            arr = plan._rule_array([rule])
            h = C.c_void_p()
            nodes = sum(7**lv for lv in range(levels))
            chosen = (C.c_int32 * nodes)()
            fp = C.POINTER(C.c_float)
            assert native.lib().fmm_plan_variants(C.byref(h), arr, levels, native.SELECT_MATRIX, 0,
                                                  Amax.ctypes.data_as(fp), Bmax.ctypes.data_as(fp), chosen,
                                                  native.LEAF_BF16) == 0
            plan._h = h
            assert list(chosen) == want, (levels, trial)
    # fmm_plan_variants needs a <2,2,2> base and block maxima for this mode
    h = C.c_void_p()
    holder = api.Plan(["strassen"])  # keeps the rule arrays alive
    arr = holder._rule_array([PR.fast323()])
    assert native.lib().fmm_plan_variants(C.byref(h), arr, 1, 1, 0, None, None, None, 0) == 10
    arr = holder._rule_array([rule])
    assert native.lib().fmm_plan_variants(C.byref(h), arr, 1, native.SELECT_MATRIX, 0, None, None, None, 0) == 1


# ---------------------------------------------------------------- the tables the kernels execute (Eq. 4.4)

def _oracle_flattened(node):
    """[[U, V, W]] of the flattened plan, read off the oracle's recursion
    (Eq. 3.2) itself: one product on operands whose finest blocks are unit
    vectors.  A is pm x (pk P) with block (p, q) = e_(p pk + q)^T (1 x P),
    B is (pk P) x (pn R) with block (p, q) holding e_(p pn + q) in its first
    column, and leaf r records S_r (1 x P: column r of U) and T_r (its first
    column: column r of V) and returns e_r^T (1 x R), so that C block k is
    row k of W.  Every sum is exact (small dyadic coefficients)."""
    pm, pk, pn = OF.dims(node)
    R = _count_leaves(node)
    P = max(pm * pk, pk * pn)
    A = np.zeros((pm, pk * P))
    for p in range(pm):
        for q in range(pk):
            A[p, q * P + p * pk + q] = 1.0
    B = np.zeros((pk * P, pn * R))
    for p in range(pk):
        for q in range(pn):
            B[p * P + p * pn + q, q * R] = 1.0
    Us, Vs = [], []

    def leaf(S, T):
        r = len(Us)
        Us.append(S[0, :pm * pk].copy())
        Vs.append(T[:pk * pn, 0].copy())
        out = np.zeros((1, R))
        out[0, r] = 1.0
        return out
    C = OF.fmm(A, B, node, leaf=leaf)
    assert len(Us) == R
    W = np.stack([C[p, q * R:(q + 1) * R] for p in range(pm) for q in range(pn)])
    return np.stack(Us, axis=1), np.stack(Vs, axis=1), W


def _count_leaves(node):
    if node is None:
        return 1
    return sum(_count_leaves(c) for c in node.children)


def _first_touch(W):
    first = np.zeros(W.shape, np.int32)
    for k in range(W.shape[0]):
        nz = np.nonzero(W[k])[0]
        if nz.size:
            first[k, nz[0]] = 1
    return first


def _plan_cases():
    from paper_1507_00687_gb300 import api
    import tree_cases as TC
    cases = []
    for names in (["strassen"], ["winograd"], ["strassen", "strassen"], ["winograd"] * 3,
                  ["strassen", "classical121", "strassen"], ["fast323"], ["fast323", "strassen"],
                  ["classical121", "winograd"]):
        cases.append((api.Plan(names, "bf16"), OF.uniform([_oracle_rule(n) for n in names])))
    # a rotation (<3,3,2>, A and B grids of different sizes) over Strassen
    cases.append((api.Plan([PR.rotate(PR.get("fast323")), "strassen"], "bf16"),
                  OF.uniform([OR.rotate(OR.fast323()), OR.strassen()])))
    for root, children in (TC.dalberto(), TC.fast323_nonuniform(), TC.mixed_rank(), TC.uneven_delta()):
        lib, orc = TC.two_level(root, children)
        cases.append((api.Plan.tree(lib, "bf16"), orc))
    from oracle import variants as CG
    for name, levels in (("strassen", 2), ("winograd", 3)):
        plan = api.Plan.variants(name, levels, "random", seed=99, leaf="bf16")
        cases.append((plan, CG.tree(_oracle_rule(name), levels, plan.chosen)))
    return cases


def test_kernel_tables_are_the_flattened_rule(native):
    # Every table the kernels read -- the per-leaf descriptors, the per-side
    # term lists and the per-C-block gather lists -- holds exactly the
    # flattened rule of Eq. 4.4 (uniform and non-stationary plans) or of
    # each root-to-leaf path (trees, Castrapel-Gustafson variant trees), in
    # depth-first leaf order, with the first-touch flags the fused epilogue
    # uses; uniform plans also equal the oracle's repeated composition.
    for plan, orc in _plan_cases():
        U0, V0, W0 = _oracle_flattened(orc)
        want_first = _first_touch(W0)
        for table in ("leaves", "lists", "gather"):
            U, V, W, first = plan.flatten(table)
            if table != "gather":
                assert np.array_equal(U, U0) and np.array_equal(V, V0), (plan.rules, table)
            assert np.array_equal(W, W0) and np.array_equal(first, want_first), (plan.rules, table)
        info = plan.info()
        assert info["nnz"] == np.count_nonzero(U0) + np.count_nonzero(V0) + np.count_nonzero(W0)
    # repeated composition (Eq. 4.4) of the oracle's rules for uniform plans
    from paper_1507_00687_gb300 import api
    for names in (["strassen", "strassen"], ["winograd", "classical121", "winograd"]):
        comp = _oracle_rule(names[0])
        for n in names[1:]:
            comp = OR.compose(comp, _oracle_rule(n))
        U, V, W, _ = api.Plan(names, "bf16").flatten()
        assert np.array_equal(U, comp.U) and np.array_equal(V, comp.V) and np.array_equal(W, comp.W)


def test_plan_flatten_rejections(native):
    from paper_1507_00687_gb300 import api
    L = native.lib()
    plan = api.Plan(["strassen"], "bf16")
    assert L.fmm_plan_flatten(None, 0, None, None, None, None) == 1
    assert L.fmm_plan_flatten(plan._h, 3, None, None, None, None) == 1
    assert L.fmm_plan_flatten(plan._h, -1, None, None, None, None) == 1
    assert L.fmm_plan_flatten(plan._h, 2, None, None, None, None) == 0


def _oracle_gradient_tree(node, which):
    """The oracle's tree with every node's rule replaced by its gradient
    rule (rule_for_dA / rule_for_dB), the shape kept."""
    if node is None:
        return None
    f = OR.rule_for_dA if which == "dA" else OR.rule_for_dB
    return OF.Node(f(node.rule), [_oracle_gradient_tree(c, which) for c in node.children])


def test_gradient_plans_are_the_transformed_rules(native):
    # The plan the backward pass runs for dA (dB) is the flattening of the
    # plan's rules transformed to [[W, V^T, U]] ([[U^T, W, V]]) at every
    # level or tree node (Sec. 5.3, App. A-C): Brent-valid, with the grid
    # <pm, pn, pk> (<pk, pm, pn>), and equal, table for table, to the
    # oracle's gradient rules flattened by its own recursion.
    for plan, orc in _plan_cases():
        info = plan.info()
        for which, dims in (("dA", (info["pm"], info["pn"], info["pk"])),
                            ("dB", (info["pk"], info["pm"], info["pn"]))):
            g = plan.gradient(which)
            gi = g.info()
            assert (gi["pm"], gi["pk"], gi["pn"]) == dims and gi["leaves"] == info["leaves"]
            U0, V0, W0 = _oracle_flattened(_oracle_gradient_tree(orc, which))
            for table in ("leaves", "lists"):
                U, V, W, first = g.flatten(table)
                assert np.array_equal(U, U0) and np.array_equal(V, V0) and np.array_equal(W, W0), (which, table)
                assert np.array_equal(first, _first_touch(W0))
    L = native.lib()
    h = C.c_void_p()
    from paper_1507_00687_gb300 import api
    p = api.Plan(["strassen"], "bf16")
    assert L.fmm_plan_gradient(None, 0, C.byref(h)) == 1
    assert L.fmm_plan_gradient(p._h, 2, C.byref(h)) == 1
    assert L.fmm_plan_gradient(p._h, 0, None) == 1


def test_binding_matches_header_signatures(native):
    # Every declaration in include/fmm.h has a ctypes signature with the
    # same number of parameters, each of the same kind and width (the
    # binding is argument marshalling only, so a mismatch would pass wrong
    # values across the C ABI without any error).
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"(?:const\s+char\s*\*|fmm_status)\s*(fmm_\w+)\s*\(([^)]*)\)\s*;", src)
    assert len(decls) == len(header_symbols())
    scalar = {"int": C.c_int, "int64_t": C.c_int64, "size_t": C.c_size_t, "double": C.c_double,
              "uint64_t": C.c_uint64, "fmm_status": C.c_int}
    handles = ("fmm_plan_t", "fmm_batch_t", "fmm_host_t")
    L = native.lib()
    for name, params in decls:
        params = params.strip()
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None and len(argtypes) == len(plist), name
        for p, at in zip(plist, argtypes):
            ptype = re.sub(r"\s*\b\w+$", "", p).replace("const ", "").strip()   # drop the parameter name
            if "*" in ptype or ptype in handles:
                ok = at in (C.c_void_p, C.c_char_p) or hasattr(at, "_type_") and issubclass(at, C._Pointer)
            else:
                ok = at is scalar[ptype]
            assert ok, (name, p, at)


def test_workspace_covers_what_the_pass_schedule_writes(native):
    # fmm_workspace_size must hold, for the forward product and both
    # gradient products, at least what the pass schedule writes: every
    # leaf's combined A and B blocks (16-bit, two planes for bf16 hi+lo; for
    # E4M3 one byte plus one scale byte per 128-block of each row) and, with
    # more than one leaf, the FP32 stored products -- an unpadded lower
    # bound computed here from the plan's grid alone.
    from paper_1507_00687_gb300 import api
    g = np.random.default_rng(17)
    cdiv = lambda a, b: -(-a // b)  # noqa: E731

    def lower(leaf, R, pm, pk, pn, M, K, N):
        bm, bk, bn = cdiv(M, pm), cdiv(K, pk), cdiv(N, pn)
        prods = R * bm * bn * 4 if R > 1 else 0
        if leaf == "e4m3b128":
            return R * (bm + bn) * bk + R * (bm + bn) * cdiv(bk, 128) + prods
        planes = 2 if leaf == "bf16x3" else 1
        return planes * R * (bm + bn) * bk * 2 + prods

    for names in (["winograd"], ["strassen", "classical121"], ["winograd"] * 2, ["fast323"], []):
        for leaf in ("bf16", "bf16x3", "e4m3b128"):
            plan = api.Plan(names, leaf)
            info = plan.info()
            R, pm, pk, pn = info["leaves"], info["pm"], info["pk"], info["pn"]
            for _ in range(6):
                M, K, N = (int(x) for x in g.integers(1, 5000, size=3))
                need = max(lower(leaf, R, pm, pk, pn, M, K, N),     # C = A B
                           lower(leaf, R, pm, pn, pk, M, N, K),     # dA = dC B^T
                           lower(leaf, R, pk, pm, pn, K, M, N))     # dB = A^T dC
                assert api.workspace_bytes(plan, M, K, N) >= need, (names, leaf, M, K, N)
