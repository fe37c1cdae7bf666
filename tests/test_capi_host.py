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
