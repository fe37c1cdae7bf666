"""Bilinear base-case rules [[U, V, W]] and their principal quantities.

Oracle module (test infrastructure only; see the package docstring).

A rule <m0, k0, n0; R> multiplies an m0 x k0 matrix by a k0 x n0 matrix with R
active products (Sec. 3.1, Eq. 3.1):

    C_k = sum_r W[k, r] M_r,   M_r = S_r * T_r,
    S_r = sum_i U[i, r] A_i,   T_r = sum_j V[j, r] B_j.

The single indices i, j, k linearise the entries of A, B and C.  The paper
states one ordering (Sec. 3.1: A and B column-major, C row-major) but its own
Strassen table (App. A) only satisfies the Brent equations when A and B are
read row-major and C column-major, while the <3,2,3> table (App. B) satisfies
them under the stated ordering.  Every rule here therefore carries its
ordering explicitly (``order_a``, ``order_b``, ``order_c``) and is converted
to one canonical form -- all three row-major -- by :func:`canonical`.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
import itertools

import numpy as np


@dataclass(frozen=True)
class Rule:
    """One base-case rule [[U, V, W]] for <m0, k0, n0; R> (Sec. 3.1)."""

    name: str
    m0: int
    k0: int
    n0: int
    U: np.ndarray  # (m0*k0, R)
    V: np.ndarray  # (k0*n0, R)
    W: np.ndarray  # (m0*n0, R)
    order_a: str = "row"
    order_b: str = "row"
    order_c: str = "row"
    source: str = field(default="", compare=False)

    @property
    def R(self) -> int:
        return self.U.shape[1]


def _lin(p: int, q: int, rows: int, cols: int, order: str) -> int:
    """Single index of entry (p, q) of a rows x cols matrix."""
    if order == "row":
        return p * cols + q
    if order == "col":
        return q * rows + p
    raise ValueError(order)


def canonical(rule: Rule) -> Rule:
    """Re-index U, V, W so that A, B and C are all read row-major."""
    m0, k0, n0 = rule.m0, rule.k0, rule.n0
    U = np.zeros_like(rule.U)
    V = np.zeros_like(rule.V)
    W = np.zeros_like(rule.W)
    for p in range(m0):
        for q in range(k0):
            U[p * k0 + q] = rule.U[_lin(p, q, m0, k0, rule.order_a)]
    for p in range(k0):
        for q in range(n0):
            V[p * n0 + q] = rule.V[_lin(p, q, k0, n0, rule.order_b)]
    for p in range(m0):
        for q in range(n0):
            W[p * n0 + q] = rule.W[_lin(p, q, m0, n0, rule.order_c)]
    return Rule(rule.name, m0, k0, n0, U, V, W, "row", "row", "row", rule.source)


def brent_violations(rule: Rule) -> int:
    """Number of Brent equations the rule violates (0 means it is a correct
    matrix-multiplication rule).

    The rule computes C = AB exactly for all A, B iff for every A-entry
    (i, k), B-entry (k', j) and C-entry (i', j')
        sum_r U[(i,k), r] V[(k',j), r] W[(i',j'), r] = [i=i'][k=k'][j=j'].
    Checked in exact rational arithmetic.
    """
    c = canonical(rule)
    m0, k0, n0, R = c.m0, c.k0, c.n0, c.R
    Uf = [[Fraction(x).limit_denominator(1 << 20) for x in row] for row in c.U]
    Vf = [[Fraction(x).limit_denominator(1 << 20) for x in row] for row in c.V]
    Wf = [[Fraction(x).limit_denominator(1 << 20) for x in row] for row in c.W]
    bad = 0
    for i, k, k2, j, i2, j2 in itertools.product(range(m0), range(k0), range(k0),
                                                 range(n0), range(m0), range(n0)):
        s = sum(Uf[i * k0 + k][r] * Vf[k2 * n0 + j][r] * Wf[i2 * n0 + j2][r]
                for r in range(R))
        want = 1 if (i == i2 and k == k2 and j == j2) else 0
        if s != want:
            bad += 1
    return bad


# ---------------------------------------------------------------------------
# Tables.  Numbers of App. A (Strassen) and App. B (<3,2,3>) transcribed as
# printed; their index ordering is the reading that satisfies Brent.
# ---------------------------------------------------------------------------

def strassen() -> Rule:
    """Strassen's <2,2,2;7> rule, App. A (coefficients as printed).

    Reading: the printed table satisfies the Brent equations with A and B
    indexed row-major and C column-major (the opposite of the ordering the
    appendix states); with that reading its products are the textbook
    m1..m7 used in Examples 6.1-6.5.
    """
    U = np.array([[1, 0, 1, 0, 1, -1, 0],
                  [0, 0, 0, 0, 1, 0, 1],
                  [0, 1, 0, 0, 0, 1, 0],
                  [1, 1, 0, 1, 0, 0, -1]], dtype=float)
    V = np.array([[1, 1, 0, -1, 0, 1, 0],
                  [0, 0, 1, 0, 0, 1, 0],
                  [0, 0, 0, 1, 0, 0, 1],
                  [1, 0, -1, 0, 1, 0, 1]], dtype=float)
    W = np.array([[1, 0, 0, 1, -1, 0, 1],
                  [0, 1, 0, 1, 0, 0, 0],
                  [0, 0, 1, 0, 1, 0, 0],
                  [1, -1, 1, 0, 0, 1, 0]], dtype=float)
    return Rule("strassen", 2, 2, 2, U, V, W, "row", "row", "col", "App. A")


def strassen_printed_convention() -> Rule:
    """The App. A numbers read with the ordering the appendix states (A, B
    column-major, C row-major).  Kept to pin that this reading is NOT a
    matrix-multiplication rule."""
    s = strassen()
    return Rule("strassen-as-stated", 2, 2, 2, s.U, s.V, s.W, "col", "col", "row", "App. A")


def fast323() -> Rule:
    """The rank-15 <3,2,3> rule of App. B (coefficients as printed), read with
    the stated ordering (A, B column-major, C row-major)."""
    U = np.array([
        [0, 1, 0, 0, -1, 1, 1, 0, 0, 0, -1, 0, 0, 0, -1],
        [0, 1, 0, 0, 0, 0, 0, -1, 0, -1, 0, 0, 1, -1, 0],
        [0, 0, 0, 1, 0, 0, 0, -1, 0, -1, 1, 0, 0, -1, 0],
        [-1, 0, 1, 0, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 1],
        [-1, 0, 0, 0, 0, 1, 0, 1, 0, 1, 0, 1, -1, 0, 0],
        [0, 0, -1, 0, 0, 0, 0, 1, 1, 0, -1, 0, 0, 0, -1]], dtype=float)
    V = np.array([
        [0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 1, 1],
        [0, 0, 1, 0, 0, 0, 0, -1, 1, -1, 0, 0, 0, 1, 0],
        [0, -1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 1, 1, -1, 0],
        [-1, 0, 0, 0, 0, 0, 0, 1, 0, 1, 0, 1, 0, -1, 0],
        [0, 1, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1],
        [1, 0, 1, 0, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 1]], dtype=float)
    W = np.array([
        [0, 0, 1, 0, 0, 0, -1, 0, 1, 0, 0, 0, 0, 0, -1],
        [1, 0, 0, 0, 1, 1, 0, 0, 0, 0, 0, -1, 0, 0, 0],
        [0, 0, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, -1, 0, 0, 0, 0, 0, -1, 0, 1, 0, -1, 0],
        [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0, 0],
        [0, 1, 0, 0, 0, 1, -1, 0, 0, 0, 0, 0, 1, 0, 0],
        [0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0, 1, 1, -1, 0, 0, -1, 0, 0],
        [0, 0, 0, -1, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, -1]], dtype=float)
    return Rule("fast323", 3, 2, 3, U, V, W, "col", "col", "row", "App. B")


def classical(m0: int, k0: int, n0: int) -> Rule:
    """The classical rule <m0,k0,n0; m0 k0 n0>: one product per (i, k, j)."""
    R = m0 * k0 * n0
    U = np.zeros((m0 * k0, R))
    V = np.zeros((k0 * n0, R))
    W = np.zeros((m0 * n0, R))
    r = 0
    for i in range(m0):
        for k in range(k0):
            for j in range(n0):
                U[i * k0 + k, r] = 1
                V[k * n0 + j, r] = 1
                W[i * n0 + j, r] = 1
                r += 1
    return Rule(f"classical{m0}{k0}{n0}", m0, k0, n0, U, V, W, source="classical")


def winograd() -> Rule:
    """The Winograd variant of Strassen's <2,2,2;7> rule in flattened form.

    The paper names this variant (Sec. 2, Sec. 5.2, Sec. 7) without printing
    its coefficients.  Reading: take the textbook definition (sums
    s1 = a21 + a22, s2 = s1 - a11, s3 = a11 - a21, s4 = a12 - s2;
    t1 = b12 - b11, t2 = b22 - t1, t3 = b22 - b12, t4 = t2 - b21;
    products a11 b11, a12 b21, s4 b22, a22 t4, s1 t1, s2 t2, s3 t3;
    c11 = m1 + m2, c12 = m1 + m6 + m5 + m3, c21 = m1 + m6 + m7 - m4,
    c22 = m1 + m6 + m7 + m5) and expand every shared partial sum, so that
    each S_r, T_r and C_k is one linear combination of base entries, as the
    [[U, V, W]] form of Eq. 3.1 requires.  Indices are row-major for A, B
    and C.  Its Brent equations are checked in the tests; its principal
    quantities are Q = 10, E = 18, nnz = 42.
    """
    # columns r = m1..m7; rows a11, a12, a21, a22
    U = np.array([[1, 0, 1, 0, 0, -1, 1],
                  [0, 1, 1, 0, 0, 0, 0],
                  [0, 0, -1, 0, 1, 1, -1],
                  [0, 0, -1, 1, 1, 1, 0]], dtype=float)
    # rows b11, b12, b21, b22
    V = np.array([[1, 0, 0, 1, -1, 1, 0],
                  [0, 0, 0, -1, 1, -1, -1],
                  [0, 1, 0, -1, 0, 0, 0],
                  [0, 0, 1, 1, 0, 1, 1]], dtype=float)
    # rows c11, c12, c21, c22
    W = np.array([[1, 1, 0, 0, 0, 0, 0],
                  [1, 0, 1, 0, 1, 1, 0],
                  [1, 0, 0, -1, 0, 1, 1],
                  [1, 0, 0, 0, 1, 1, 1]], dtype=float)
    return Rule("winograd", 2, 2, 2, U, V, W, source="Strassen-Winograd variant")


# ---------------------------------------------------------------------------
# Principal quantities (Sec. 4.1, Eqs. 4.1-4.2, Defs. 4.1-4.2)
# ---------------------------------------------------------------------------

@dataclass
class Principal:
    alpha: np.ndarray   # nnz of columns of U
    beta: np.ndarray    # nnz of columns of V
    gamma: np.ndarray   # nnz of rows of W
    a: np.ndarray       # column 1-norms of U
    b: np.ndarray       # column 1-norms of V
    q: np.ndarray       # prefactor vector (Def. 4.1)
    e: np.ndarray       # stability vector (Def. 4.2)
    Q: float
    E: float
    nnz: int


def principal(rule: Rule) -> Principal:
    """alpha, beta, gamma, a, b (Eqs. 4.1-4.2), q and Q (Def. 4.1), e and E
    (Def. 4.2), and nnz(U)+nnz(V)+nnz(W).  Entries of q and e follow the row
    order of W in the rule as given."""
    U, V, W = rule.U, rule.V, rule.W
    alpha = (U != 0).sum(axis=0)
    beta = (V != 0).sum(axis=0)
    gamma = (W != 0).sum(axis=1)
    a = np.abs(U).sum(axis=0)
    b = np.abs(V).sum(axis=0)
    q = np.array([gamma[k] + max((alpha[r] + beta[r]) * (W[k, r] != 0)
                                 for r in range(rule.R))
                  for k in range(W.shape[0])], dtype=float)
    e = np.array([sum(a[r] * b[r] * abs(W[k, r]) for r in range(rule.R))
                  for k in range(W.shape[0])], dtype=float)
    nnz = int((U != 0).sum() + (V != 0).sum() + (W != 0).sum())
    return Principal(alpha, beta, gamma, a, b, q, e, float(q.max()), float(e.max()), nnz)


# ---------------------------------------------------------------------------
# Rule transforms
# ---------------------------------------------------------------------------

def compose(outer: Rule, inner: Rule) -> Rule:
    """The single rule <m1 m2, k1 k2, n1 n2; R1 R2> equal to one level of
    ``outer`` followed by one level of ``inner`` (the flattening of
    Eq. 4.4 for L = 2).  Both rules are taken in canonical form.  Entry
    (p, q) of the composite A lies in outer block (p // m2, q // k2) at inner
    position (p % m2, q % k2); the composite product index is r1 * R2 + r2."""
    o, i = canonical(outer), canonical(inner)
    m0, k0, n0 = o.m0 * i.m0, o.k0 * i.k0, o.n0 * i.n0
    R = o.R * i.R

    def kron(Mo, Mi, ro, co, ri, ci):
        rows, cols = ro * ri, co * ci
        out = np.zeros((rows * cols, R))
        for p in range(rows):
            for q in range(cols):
                io = (p // ri) * co + (q // ci)
                ii = (p % ri) * ci + (q % ci)
                out[p * cols + q] = np.kron(Mo[io], Mi[ii])
        return out

    U = kron(o.U, i.U, o.m0, o.k0, i.m0, i.k0)
    V = kron(o.V, i.V, o.k0, o.n0, i.k0, i.n0)
    W = kron(o.W, i.W, o.m0, o.n0, i.m0, i.n0)
    return Rule(f"{o.name}*{i.name}", m0, k0, n0, U, V, W, source="composition")


def transpose_index(M: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """Rows of M re-indexed from a row-major rows x cols matrix to the
    row-major cols x rows transpose (the vec-permutation of App. C)."""
    out = np.zeros_like(M)
    for p in range(rows):
        for q in range(cols):
            out[q * rows + p] = M[p * cols + q]
    return out


def rule_for_dA(rule: Rule) -> Rule:
    """Rule for dA = dC B^T, an <m0, n0, k0> product, obtained from the
    cyclic symmetry of the matrix-multiplication tensor (the transforms of
    Sec. 5.3 / App. A-C): the dC operand takes the W coefficients, B^T the V
    coefficients re-indexed by transposition, and the result dA the U
    coefficients."""
    c = canonical(rule)
    return Rule(c.name + "^dA", c.m0, c.n0, c.k0,
                c.W.copy(), transpose_index(c.V, c.k0, c.n0), c.U.copy(),
                source="transform")


def rule_for_dB(rule: Rule) -> Rule:
    """Rule for dB = A^T dC, a <k0, m0, n0> product: A^T takes the U
    coefficients re-indexed by transposition, dC the W coefficients and the
    result dB the V coefficients."""
    c = canonical(rule)
    return Rule(c.name + "^dB", c.k0, c.m0, c.n0,
                transpose_index(c.U, c.m0, c.k0), c.W.copy(), c.V.copy(),
                source="transform")


def to_stated_order(rule: Rule) -> Rule:
    """Re-index a rule into the ordering Sec. 3.1 states (A, B column-major,
    C row-major)."""
    c = canonical(rule)
    m0, k0, n0 = c.m0, c.k0, c.n0
    U, V, W = np.zeros_like(c.U), np.zeros_like(c.V), c.W.copy()
    for p in range(m0):
        for q in range(k0):
            U[q * m0 + p] = c.U[p * k0 + q]
    for p in range(k0):
        for q in range(n0):
            V[q * k0 + p] = c.V[p * n0 + q]
    return Rule(c.name, m0, k0, n0, U, V, W, "col", "col", "row", c.source)


def rotate(rule: Rule) -> Rule:
    """The cyclic rotation [[W, U, V]] (App. A, App. B).  With the stated
    ordering the three index vectors are those of A, B and C^T, all
    column-major, and tr(ABC^T) is invariant under cycling the three
    operands; so [[W, U, V]] of a <m0,k0,n0> rule is a <n0,m0,k0> rule in the
    same ordering."""
    s = to_stated_order(rule)
    return Rule(s.name + "^rot", s.n0, s.m0, s.k0, s.W.copy(), s.U.copy(),
                s.V.copy(), "col", "col", "row", "rotation")
