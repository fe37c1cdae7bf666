"""Pins for the oracle's rules, principal quantities and rule transforms.

Every expected value is printed in the paper (golden files cite where) or
follows from the Brent equations (exact rational check).
"""
import os

import numpy as np
import pytest

from oracle import fmm as F
from oracle import rules as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


RULES = {
    "classical222": lambda: R.classical(2, 2, 2),
    "strassen": R.strassen,
    "strassen*classical211": lambda: R.compose(R.strassen(), R.classical(2, 1, 1)),
    "strassen*classical121": lambda: R.compose(R.strassen(), R.classical(1, 2, 1)),
    "fast323": R.fast323,
    "fast323^rot": lambda: R.rotate(R.fast323()),
}


@pytest.mark.parametrize("row", _golden("table1.txt"), ids=lambda r: r[0])
def test_table1_principal_quantities(row):
    name, m0, k0, n0, Rk, nnz, Q, E = row
    rule = RULES[name]()
    p = R.principal(rule)
    assert (rule.m0, rule.k0, rule.n0, rule.R) == (int(m0), int(k0), int(n0), int(Rk))
    assert p.nnz == int(nnz)
    assert p.Q == float(Q)
    assert p.E == float(E)
    assert R.brent_violations(rule) == 0


def test_stability_vectors_printed():
    g = {r[0]: [float(x) for x in r[1:]] for r in _golden("stability_vectors.txt")}
    assert list(R.principal(R.strassen()).e) == g["strassen"]
    # <3,2,3>: W rows are row-major C; the printed vector lists column-major C
    e = R.principal(R.fast323()).e.reshape(3, 3)
    assert list(e.T.reshape(-1)) == g["fast323_colmajor"]


@pytest.mark.parametrize("make", [R.strassen, R.winograd, R.fast323,
                                  lambda: R.classical(2, 2, 2),
                                  lambda: R.classical(1, 2, 1),
                                  lambda: R.classical(2, 1, 1),
                                  lambda: R.classical(2, 3, 4)])
def test_brent_holds(make):
    assert R.brent_violations(make()) == 0


def test_strassen_stated_ordering_is_not_matmul():
    # The App. A numbers under the ordering App. A states violate Brent; this
    # pins the index-order reading used everywhere else.
    assert R.brent_violations(R.strassen_printed_convention()) == 12


def test_brent_catches_planted_mistakes():
    s = R.strassen()
    for which in ("U", "V", "W"):
        M = getattr(s, which).copy()
        M[0, 0] = -M[0, 0]
        bad = R.Rule("bad", 2, 2, 2, *(M if w == which else getattr(s, w) for w in "UVW"),
                     s.order_a, s.order_b, s.order_c)
        assert R.brent_violations(bad) > 0
    # swapped columns of W only (a transposed output assignment)
    W = s.W[:, [1, 0, 2, 3, 4, 5, 6]]
    assert R.brent_violations(R.Rule("bad", 2, 2, 2, s.U, s.V, W, "row", "row", "col")) > 0


def test_winograd_quantities():
    # Not printed in the paper; Sec. 5.2 only says its stability factor is
    # slightly larger than Strassen's 12.  Q, E, nnz of the flattened form.
    p = R.principal(R.winograd())
    assert (p.Q, p.E, p.nnz) == (10.0, 18.0, 42)
    assert p.E > R.principal(R.strassen()).E
    assert list(p.alpha) == [1, 1, 4, 1, 2, 3, 2]


@pytest.mark.parametrize("make", [R.strassen, R.winograd, R.fast323])
def test_gradient_rules_brent(make):
    r = make()
    dA, dB = R.rule_for_dA(r), R.rule_for_dB(r)
    assert (dA.m0, dA.k0, dA.n0) == (r.m0, r.n0, r.k0)
    assert (dB.m0, dB.k0, dB.n0) == (r.k0, r.m0, r.n0)
    assert R.brent_violations(dA) == 0
    assert R.brent_violations(dB) == 0


def test_rotations_are_rules():
    f = R.fast323()
    r1 = R.rotate(f)
    r2 = R.rotate(r1)
    assert (r1.m0, r1.k0, r1.n0) == (3, 3, 2)
    assert (r2.m0, r2.k0, r2.n0) == (2, 3, 3)
    assert R.brent_violations(r1) == 0 and R.brent_violations(r2) == 0
    # cyclic invariance of Strassen's Q and E (App. A)
    s = R.principal(R.strassen())
    for rr in (R.rotate(R.strassen()), R.rotate(R.rotate(R.strassen()))):
        p = R.principal(rr)
        assert (p.Q, p.E) == (s.Q, s.E)


def _variant(rule, XU, XV, XW, name):
    return R.Rule(name, rule.m0, rule.k0, rule.n0, XU @ rule.U, XV @ rule.V, XW @ rule.W,
                  rule.order_a, rule.order_b, rule.order_c)


def test_dalberto_two_level_factor():
    g = {r[0]: float(r[1]) for r in _golden("stability_vectors.txt") if len(r) == 2}
    s = R.strassen()
    P, I = np.array([[0, 1], [1, 0]]), np.eye(2)
    # Reading: permute the columns of B and the columns of C together; in the
    # effective ordering of App. A that is (I x P) V and (P x I) W.  The
    # printed (P x I) V, (I x P) W fails Brent but has the same factor.
    valid = _variant(s, np.eye(4), np.kron(I, P), np.kron(P, I), "dalberto")
    printed = _variant(s, np.eye(4), np.kron(P, I), np.kron(I, P), "printed")
    assert R.brent_violations(valid) == 0
    assert R.brent_violations(printed) > 0
    for v in (valid, printed):
        tree = F.Node(s, [F.Node(v if r in (0, 2, 3) else s, [None] * 7) for r in range(7)])
        assert F.xi_vector(tree).max() == g["strassen_L2_dalberto"]
    assert F.xi_vector(F.uniform([s, s])).max() == g["strassen_L2_stationary"]


def test_fast323_nonuniform_two_level_factor():
    g = {r[0]: float(r[1]) for r in _golden("stability_vectors.txt") if len(r) == 2}
    f = R.fast323()
    I2 = np.eye(2)
    P = np.array([[1, 0, 0], [0, 0, 1], [0, 1, 0]])
    Pp = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]])
    v1 = _variant(f, np.kron(I2, P), np.kron(P, I2), np.kron(P, P), "v1")
    v2 = _variant(f, np.kron(I2, Pp), np.kron(Pp, I2), np.kron(Pp, Pp), "v2")
    assert R.brent_violations(v1) == 0 and R.brent_violations(v2) == 0
    node_rule = {n: f for n in (2, 6, 8, 14, 15)}
    node_rule.update({n: v1 for n in (1, 3, 10, 11)})
    node_rule.update({n: v2 for n in (4, 5, 7, 9, 12, 13)})
    tree = F.Node(f, [F.Node(node_rule[r + 1], [None] * 15) for r in range(15)])
    assert F.xi_vector(tree).max() == g["fast323_L2_nonuniform"]
    assert F.xi_vector(F.uniform([f, f])).max() == g["fast323_L2_stationary"]


def test_uniform_tree_quantities_reduce_to_theorem_4_2():
    # For uniform plans the Sec. 4.5 recursions reduce to sum Q and prod E.
    s, w, c = R.strassen(), R.winograd(), R.classical(1, 2, 1)
    for rules in ([s], [s, s], [w, c, w], [s, w], [w, w, w]):
        tree = F.uniform(rules)
        Qs = sum(R.principal(r).Q for r in rules)
        Es = np.prod([R.principal(r).E for r in rules])
        assert F.delta_vector(tree).max() == Qs
        assert F.xi_vector(tree).max() == Es


def test_composition_matches_two_levels():
    # A composed rule equals two levels of recursion (flattening, Eq. 4.4).
    s, c = R.strassen(), R.classical(1, 2, 1)
    comp = R.compose(s, c)
    assert R.brent_violations(comp) == 0
    g = np.random.default_rng(0)
    A = g.integers(-3, 4, size=(8, 16)).astype(float)
    B = g.integers(-3, 4, size=(16, 8)).astype(float)
    one = F.fmm(A, B, F.uniform([comp]))
    two = F.fmm(A, B, F.uniform([s, c]))
    assert np.array_equal(one, A @ B) and np.array_equal(two, A @ B)
    pc = R.principal(comp)
    assert pc.E == R.principal(s).E * R.principal(c).E


def test_stated_order_reindexing():
    # Sec. 3.1 states A and B column-major and C row-major.  App. B's table
    # is read in that order, so re-indexing it changes nothing; Strassen's
    # second product (a21 + a22) b11 puts a21 at index 2 row-major and at
    # index 1 column-major.  Every rule keeps its canonical form and Brent.
    f = R.fast323()
    s = R.to_stated_order(f)
    assert np.array_equal(s.U, f.U) and np.array_equal(s.V, f.V) and np.array_equal(s.W, f.W)
    st = R.to_stated_order(R.strassen())
    assert list(R.canonical(R.strassen()).U[:, 1]) == [0, 0, 1, 1]
    assert list(st.U[:, 1]) == [0, 1, 0, 1] and list(st.V[:, 1]) == [1, 0, 0, 0]
    for r in (R.strassen(), R.winograd(), R.classical(2, 3, 4), R.fast323(), R.rotate(R.fast323())):
        s = R.to_stated_order(r)
        assert (s.order_a, s.order_b, s.order_c) == ("col", "col", "row")
        assert R.brent_violations(s) == 0
        c0, c1 = R.canonical(r), R.canonical(s)
        assert np.array_equal(c0.U, c1.U) and np.array_equal(c0.V, c1.V) and np.array_equal(c0.W, c1.W)


def _flattened_by_recursion(rules):
    """[[U, V, W]] of L levels read off the recursion of Eq. 3.2 itself:
    one product whose finest blocks are unit vectors, with a leaf that
    records S_r and T_r and returns e_r (so C block k holds row k of W)."""
    node = F.uniform(rules)
    pm, pk, pn = F.dims(node)
    R_ = int(np.prod([r.R for r in rules]))
    P = max(pm * pk, pk * pn)
    A = np.zeros((pm, pk * P))
    for p in range(pm):
        for q in range(pk):
            A[p, q * P + p * pk + q] = 1.0
    B = np.zeros((pk * P, pn * R_))
    for p in range(pk):
        for q in range(pn):
            B[p * P + p * pn + q, q * R_] = 1.0
    Us, Vs = [], []

    def leaf(S, T):
        out = np.zeros((1, R_))
        out[0, len(Us)] = 1.0
        Us.append(S[0, :pm * pk].copy())
        Vs.append(T[:pk * pn, 0].copy())
        return out
    C = F.fmm(A, B, node, leaf=leaf)
    W = np.stack([C[p, q * R_:(q + 1) * R_] for p in range(pm) for q in range(pn)])
    return np.stack(Us, axis=1), np.stack(Vs, axis=1), W


@pytest.mark.parametrize("pair", [("strassen", "classical121"), ("winograd", "strassen"),
                                  ("fast323", "classical211"), ("classical121", "fast323")])
def test_composition_is_the_recursions_flattening(pair):
    # Eq. 4.4: leaf (r1, r2) of two levels multiplies S = sum U[i1,r1]
    # U[i2,r2] A_(i1,i2) by T likewise and adds W[k1,r1] W[k2,r2] times the
    # product into C block (k1,k2); the recursion visits r2 fastest, so the
    # composite's product r1 R2 + r2 must be the recursion's leaf number
    # r1 R2 + r2, entry for entry.
    mk = {"strassen": R.strassen, "winograd": R.winograd, "fast323": R.fast323,
          "classical121": lambda: R.classical(1, 2, 1), "classical211": lambda: R.classical(2, 1, 1)}
    outer, inner = mk[pair[0]](), mk[pair[1]]()
    comp = R.compose(outer, inner)
    U, V, W = _flattened_by_recursion([outer, inner])
    assert np.array_equal(comp.U, U) and np.array_equal(comp.V, V) and np.array_equal(comp.W, W)


def test_principal_quantities_under_product_rescaling():
    # Scaling product r's A-combination by c_r and its output row by 1/c_r
    # (U_r -> c_r U_r, W_r -> W_r / c_r) or its B-combination likewise gives
    # another rule for the same product: the nonzero counts (alpha, beta,
    # gamma, Q, nnz) stay, a_r (b_r) = ||u_r||_1 (||v_r||_1) scales by
    # |c_r|, and every e_k = sum_r a_r b_r |w_kr| is unchanged (Defs.
    # 4.1-4.2).  Powers of two keep every product exact.
    s = R.canonical(R.strassen())
    p0 = R.principal(s)
    c = np.array([2.0, 0.5, 4.0, 1.0, 0.25, 2.0, 8.0])
    for which in ("U", "V"):
        U, V = s.U.copy(), s.V.copy()
        if which == "U":
            U = U * c[None, :]
        else:
            V = V * c[None, :]
        r = R.Rule("rescaled", 2, 2, 2, U, V, s.W / c[None, :], "row", "row", "row", "test")
        assert R.brent_violations(r) == 0
        p = R.principal(r)
        assert np.array_equal(p.alpha, p0.alpha) and np.array_equal(p.beta, p0.beta)
        assert p.Q == p0.Q and p.nnz == p0.nnz
        scaled = p.a if which == "U" else p.b
        same = p.b if which == "U" else p.a
        base = p0.a if which == "U" else p0.b
        assert np.array_equal(scaled, base * c) and np.array_equal(same, p0.b if which == "U" else p0.a)
        assert np.allclose(p.e, p0.e) and p.E == p0.E
