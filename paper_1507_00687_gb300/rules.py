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


def _index(p: int, q: int, rows: int, cols: int, order: int) -> int:
    return p * cols + q if order == ROW else q * rows + p


def _to_row_major(X: np.ndarray, rows: int, cols: int, order: int) -> np.ndarray:
    """Rows of X re-indexed so that entry (p, q) of the operand is row p*cols+q."""
    out = np.zeros_like(X)
    for p in range(rows):
        for q in range(cols):
            out[p * cols + q] = X[_index(p, q, rows, cols, order)]
    return out


def rotate(rule: BaseRule) -> BaseRule:
    """The cyclic rotation of a <m0,k0,n0> rule into a <n0,m0,k0> rule
    (Sec. 5.3, App. A-B).  The matrix-multiplication tensor is the sum over
    (i, k, j) of a_ik (x) b_kj (x) c_ij; cycling the factors to
    c_ij (x) a_ik (x) b_kj gives the tensor of a <n0, m0, k0> product whose
    A entry (j, i) is C's entry (i, j), whose B entry (i, k) is A's, and
    whose C entry (j, k) is B's entry (k, j).  So U' = W, V' = U, W' = V,
    with the W and V tables read column-major."""
    U = _to_row_major(rule.U, rule.m0, rule.k0, rule.order_a)
    V = _to_row_major(rule.V, rule.k0, rule.n0, rule.order_b)
    W = _to_row_major(rule.W, rule.m0, rule.n0, rule.order_c)
    return BaseRule(rule.name + "_rot", rule.n0, rule.m0, rule.k0, W, U, V, COL, ROW, COL)


def compose(outer: BaseRule, inner: BaseRule) -> BaseRule:
    """One rule for two recursion steps (Eq. 4.4 with L = 2): block (p1, q1)
    of the outer split, then (p2, q2) of the inner one, is entry
    (p1 m2 + p2, q1 k2 + q2) of the <m1 m2, k1 k2, n1 n2> base case, and
    product (r1, r2) -- numbered r1 R2 + r2 -- has coefficients
    X1[(p1, q1), r1] X2[(p2, q2), r2].  All tables row-major."""
    def flat(X1, rows1, cols1, o1, X2, rows2, cols2, o2):
        A = _to_row_major(X1, rows1, cols1, o1)
        B = _to_row_major(X2, rows2, cols2, o2)
        R1, R2 = A.shape[1], B.shape[1]
        out = np.zeros((rows1 * rows2 * cols1 * cols2, R1 * R2))
        for p1 in range(rows1):
            for q1 in range(cols1):
                for p2 in range(rows2):
                    for q2 in range(cols2):
                        row = (p1 * rows2 + p2) * (cols1 * cols2) + q1 * cols2 + q2
                        out[row] = np.outer(A[p1 * cols1 + q1], B[p2 * cols2 + q2]).reshape(-1)
        return out
    o, i = outer, inner
    return BaseRule(f"{o.name}*{i.name}", o.m0 * i.m0, o.k0 * i.k0, o.n0 * i.n0,
                    flat(o.U, o.m0, o.k0, o.order_a, i.U, i.m0, i.k0, i.order_a),
                    flat(o.V, o.k0, o.n0, o.order_b, i.V, i.k0, i.n0, i.order_b),
                    flat(o.W, o.m0, o.n0, o.order_c, i.W, i.m0, i.n0, i.order_c))


def variant(rule: BaseRule, XU: np.ndarray, XV: np.ndarray, XW: np.ndarray, name: str) -> BaseRule:
    """[[XU U, XV V, XW W]]: the rule with the rows of its tables mixed by XU,
    XV, XW in the rule's own entry order (Sec. 3.4: permutations of the
    entries of A, B and C give equivalent rules with other stability
    vectors).  The library checks the Brent equations of the result."""
    return BaseRule(name, rule.m0, rule.k0, rule.n0, np.asarray(XU, np.float64) @ rule.U,
                    np.asarray(XV, np.float64) @ rule.V, np.asarray(XW, np.float64) @ rule.W,
                    rule.order_a, rule.order_b, rule.order_c)


BUILTIN = {"strassen": strassen, "winograd": winograd, "fast323": fast323,
           "classical121": lambda: classical(1, 2, 1), "classical211": lambda: classical(2, 1, 1),
           "classical112": lambda: classical(1, 1, 2), "classical222": lambda: classical(2, 2, 2)}


def get(name: str) -> BaseRule:
    try:
        return BUILTIN[name]()
    except KeyError:
        raise ValueError(f"unknown rule {name!r}; known: {sorted(BUILTIN)}") from None
