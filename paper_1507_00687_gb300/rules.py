"""Built-in base-case rules [[U, V, W]] (Sec. 3.1) in the form fmm_plan takes.

Each rule carries the single-index order of its A, B and C entries; the
library re-indexes and checks the Brent equations itself.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ROW, COL = 0, 1


@dataclass(frozen=True)
class BaseRule:
    name: str
    m0: int
    k0: int
    n0: int
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    order_a: int = ROW
    order_b: int = ROW
    order_c: int = ROW

    @property
    def r(self) -> int:
        return int(self.U.shape[1])


def strassen() -> BaseRule:
    """Strassen <2,2,2;7> with the numbers of App. A.  The table is a
    matrix-multiplication rule when A and B entries are enumerated row-major
    and C entries column-major."""
    U = np.array([[1, 0, 1, 0, 1, -1, 0], [0, 0, 0, 0, 1, 0, 1],
                  [0, 1, 0, 0, 0, 1, 0], [1, 1, 0, 1, 0, 0, -1]], np.float64)
    V = np.array([[1, 1, 0, -1, 0, 1, 0], [0, 0, 1, 0, 0, 1, 0],
                  [0, 0, 0, 1, 0, 0, 1], [1, 0, -1, 0, 1, 0, 1]], np.float64)
    W = np.array([[1, 0, 0, 1, -1, 0, 1], [0, 1, 0, 1, 0, 0, 0],
                  [0, 0, 1, 0, 1, 0, 0], [1, -1, 1, 0, 0, 1, 0]], np.float64)
    return BaseRule("strassen", 2, 2, 2, U, V, W, ROW, ROW, COL)


def winograd() -> BaseRule:
    """Strassen-Winograd <2,2,2;7>: products a11 b11, a12 b21,
    (a11 + a12 - a21 - a22) b22, a22 (b11 - b12 - b21 + b22),
    (a21 + a22)(b12 - b11), (a21 + a22 - a11)(b11 - b12 + b22),
    (a11 - a21)(b22 - b12); c11 = m1 + m2, c12 = m1 + m3 + m5 + m6,
    c21 = m1 - m4 + m6 + m7, c22 = m1 + m5 + m6 + m7 (every shared partial
    sum of the textbook schedule expanded, as the [[U, V, W]] form needs).
    Row-major A, B, C."""
    U = np.array([[1, 0, 1, 0, 0, -1, 1], [0, 1, 1, 0, 0, 0, 0],
                  [0, 0, -1, 0, 1, 1, -1], [0, 0, -1, 1, 1, 1, 0]], np.float64)
    V = np.array([[1, 0, 0, 1, -1, 1, 0], [0, 0, 0, -1, 1, -1, -1],
                  [0, 1, 0, -1, 0, 0, 0], [0, 0, 1, 1, 0, 1, 1]], np.float64)
    W = np.array([[1, 1, 0, 0, 0, 0, 0], [1, 0, 1, 0, 1, 1, 0],
                  [1, 0, 0, -1, 0, 1, 1], [1, 0, 0, 0, 1, 1, 1]], np.float64)
    return BaseRule("winograd", 2, 2, 2, U, V, W)


def classical(m0: int, k0: int, n0: int) -> BaseRule:
    """The classical <m0,k0,n0; m0 k0 n0> rule, one product per (i, k, j)."""
    R = m0 * k0 * n0
    U = np.zeros((m0 * k0, R))
    V = np.zeros((k0 * n0, R))
    W = np.zeros((m0 * n0, R))
    for r, (i, k, j) in enumerate((i, k, j) for i in range(m0) for k in range(k0) for j in range(n0)):
        U[i * k0 + k, r] = V[k * n0 + j, r] = W[i * n0 + j, r] = 1
    return BaseRule(f"classical{m0}{k0}{n0}", m0, k0, n0, U, V, W)


def fast323() -> BaseRule:
    """The rank-15 <3,2,3> rule of App. B (A, B column-major, C row-major)."""
    U = np.array([
        [0, 1, 0, 0, -1, 1, 1, 0, 0, 0, -1, 0, 0, 0, -1],
        [0, 1, 0, 0, 0, 0, 0, -1, 0, -1, 0, 0, 1, -1, 0],
        [0, 0, 0, 1, 0, 0, 0, -1, 0, -1, 1, 0, 0, -1, 0],
        [-1, 0, 1, 0, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1],
        [-1, 0, 0, 0, 0, 1, 0, 1, 0, 1, 0, 1, -1, 0, 0],
        [0, 0, -1, 0, 0, 0, 0, 1, 1, 0, -1, 0, 0, 0, -1]], np.float64)
    V = np.array([
        [0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 1, 1],
        [0, 0, 1, 0, 0, 0, 0, -1, 1, -1, 0, 0, 0, 1, 0],
        [0, -1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 1, 1, -1, 0],
        [-1, 0, 0, 0, 0, 0, 0, 1, 0, 1, 0, 1, 0, -1, 0],
        [0, 1, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1],
        [1, 0, 1, 0, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 1]], np.float64)
    W = np.array([
        [0, 0, 1, 0, 0, 0, -1, 0, 1, 0, 0, 0, 0, 0, -1],
        [1, 0, 0, 0, 1, 1, 0, 0, 0, 0, 0, -1, 0, 0, 0],
        [0, 0, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, -1, 0, 0, 0, 0, 0, -1, 0, 1, 0, -1, 0],
        [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0, 0],
        [0, 1, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 1, 0, 0],
        [0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0, 1, 1, -1, 0, 0, -1, 0, 0],
        [0, 0, 0, -1, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, -1]], np.float64)
    return BaseRule("fast323", 3, 2, 3, U, V, W, COL, COL, ROW)


# ---------------------------------------------------------------- rule algebra
# Rotation, composition, transformation and permutation are computed and
# Brent-checked by the library (fmm_rule_*); these functions marshal the
# tables in and out.  Results are row-major in A, B and C.

def _c_rule(rule: BaseRule, keep: list):
    from . import _native as N
    import ctypes as C
    arrs = [np.ascontiguousarray(X, np.float64) for X in (rule.U, rule.V, rule.W)]
    keep.extend(arrs)
    dp = C.POINTER(C.c_double)
    return N.FmmRule(rule.m0, rule.k0, rule.n0, rule.r, *(a.ctypes.data_as(dp) for a in arrs),
                     rule.order_a, rule.order_b, rule.order_c)


def _c_call(name: str, what: str, shapes, call) -> BaseRule:
    """Run call(U, V, W, out) with output arrays of the given (rows, R)
    shapes and wrap the rule the library wrote."""
    from . import _native as N
    import ctypes as C
    U, V, W = (np.zeros(s, np.float64) for s in shapes)
    dp = C.POINTER(C.c_double)
    out = N.FmmRule()
    N.check(call(U.ctypes.data_as(dp), V.ctypes.data_as(dp), W.ctypes.data_as(dp), C.byref(out)), what)
    assert (out.order_a, out.order_b, out.order_c) == (ROW, ROW, ROW)
    return BaseRule(name, out.m0, out.k0, out.n0, U, V, W, ROW, ROW, ROW)


def rotate(rule: BaseRule) -> BaseRule:
    """The cyclic rotation of a <m0,k0,n0> rule into a <n0,m0,k0> rule
    (App. A-B; fmm_rule_rotate)."""
    from . import _native as N
    import ctypes as C
    keep: list = []
    cr = _c_rule(rule, keep)
    R = rule.r
    shapes = ((rule.n0 * rule.m0, R), (rule.m0 * rule.k0, R), (rule.n0 * rule.k0, R))
    return _c_call(rule.name + "_rot", "fmm_rule_rotate", shapes,
                   lambda U, V, W, o: N.lib().fmm_rule_rotate(C.byref(cr), U, V, W, o))


def compose(outer: BaseRule, inner: BaseRule) -> BaseRule:
    """One rule for two recursion steps (Eq. 4.4 with L = 2; fmm_rule_compose):
    product (r1, r2) is numbered r1 R2 + r2."""
    from . import _native as N
    import ctypes as C
    keep: list = []
    co, ci = _c_rule(outer, keep), _c_rule(inner, keep)
    o, i = outer, inner
    R = o.r * i.r
    shapes = ((o.m0 * i.m0 * o.k0 * i.k0, R), (o.k0 * i.k0 * o.n0 * i.n0, R), (o.m0 * i.m0 * o.n0 * i.n0, R))
    return _c_call(f"{o.name}*{i.name}", "fmm_rule_compose", shapes,
                   lambda U, V, W, out: N.lib().fmm_rule_compose(C.byref(co), C.byref(ci), U, V, W, out))


def variant(rule: BaseRule, XU: np.ndarray, XV: np.ndarray, XW: np.ndarray, name: str) -> BaseRule:
    """[[XU U, XV V, XW W]] with the mixing matrices in the rule's own entry
    order (Sec. 3.4; fmm_rule_transform, which rejects a result that is not
    a matrix-multiplication rule)."""
    from . import _native as N
    import ctypes as C
    keep: list = []
    cr = _c_rule(rule, keep)
    xs = [np.ascontiguousarray(X, np.float64) for X in (XU, XV, XW)]
    dp = C.POINTER(C.c_double)
    R = rule.r
    shapes = ((rule.m0 * rule.k0, R), (rule.k0 * rule.n0, R), (rule.m0 * rule.n0, R))
    return _c_call(name, "fmm_rule_transform", shapes,
                   lambda U, V, W, o: N.lib().fmm_rule_transform(C.byref(cr), *(x.ctypes.data_as(dp) for x in xs),
                                                                 U, V, W, o))


def permute(rule: BaseRule, perm_i, perm_k, perm_j, name: str) -> BaseRule:
    """The rule on A, B blocks relabelled by permutations of the block
    indices i, k, j (fmm_rule_permute); it computes the same product."""
    from . import _native as N
    import ctypes as C
    keep: list = []
    cr = _c_rule(rule, keep)
    ps = [(C.c_int32 * len(p))(*p) for p in (perm_i, perm_k, perm_j)]
    R = rule.r
    shapes = ((rule.m0 * rule.k0, R), (rule.k0 * rule.n0, R), (rule.m0 * rule.n0, R))
    return _c_call(name, "fmm_rule_permute", shapes,
                   lambda U, V, W, o: N.lib().fmm_rule_permute(C.byref(cr), *ps, U, V, W, o))


def castrapel_gustafson(rule: BaseRule, v: int) -> BaseRule:
    """Variant v = 0..7 of a <2,2,2> rule (Sec. 3.4): bit 0 exchanges the i
    blocks (y = 1), bit 1 the k blocks (x = 1), bit 2 the j blocks (z = 1)."""
    sw = lambda b: [1, 0] if v & b else [0, 1]  # noqa: E731
    return permute(rule, sw(1), sw(2), sw(4), f"{rule.name}_cg{v}")


BUILTIN = {"strassen": strassen, "winograd": winograd, "fast323": fast323,
           "classical121": lambda: classical(1, 2, 1), "classical211": lambda: classical(2, 1, 1),
           "classical112": lambda: classical(1, 1, 2), "classical222": lambda: classical(2, 2, 2)}


def get(name: str) -> BaseRule:
    try:
        return BUILTIN[name]()
    except KeyError:
        raise ValueError(f"unknown rule {name!r}; known: {sorted(BUILTIN)}") from None
