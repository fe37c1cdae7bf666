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
