"""Pins for the oracle's Castrapel-Gustafson variants and node selections
(Sec. 3.4).

Pinned against: the Brent equations of every variant, the identity variant,
the closed form of a variant's stability vector (a permutation of the
rule's, since the variant relabels the blocks of C), exactness against the
classical product on integer inputs for a tree mixing all eight variants,
the published reference outputs of SplitMix64, brute-force minimality of
the matrix-dependent choice, and its equivariance: exchanging the block rows
of A (the block columns of B, both k halves) permutes the node's eight
costs by v -> v xor 1 (v xor 4, v xor 2); the bounds passed to a node's
children hold on real matrices and are attained by sign-matched constant
blocks.
"""
import itertools

import numpy as np
import pytest

from oracle import fmm as F
from oracle import rules as R
from oracle import variants as CG
from paper_1507_00687_gb300 import inputs

BASES = {"strassen": R.strassen, "winograd": R.winograd}


@pytest.mark.parametrize("name", sorted(BASES))
def test_every_variant_is_a_rule_and_v0_is_the_rule(name):
    base = BASES[name]()
    for v in range(8):
        assert R.brent_violations(CG.variant(base, v)) == 0, v
    c0, cb = R.canonical(CG.variant(base, 0)), R.canonical(base)
    assert np.array_equal(c0.U, cb.U) and np.array_equal(c0.V, cb.V) and np.array_equal(c0.W, cb.W)
    # eight distinct variants
    tabs = {R.canonical(CG.variant(base, v)).U.tobytes() + R.canonical(CG.variant(base, v)).V.tobytes()
            + R.canonical(CG.variant(base, v)).W.tobytes() for v in range(8)}
    assert len(tabs) == 8


@pytest.mark.parametrize("name", sorted(BASES))
def test_variant_stability_vector_is_the_permuted_one(name):
    # A variant multiplies the blocks of A, B relabelled by the exchanges of
    # i (y = 1) and j (z = 1) -- and of k, which C does not see -- so its
    # stability vector e (indexed by C's entries, row-major) is the rule's
    # with C's block indices relabelled: e_v(i, j) = e(i xor y1, j xor z1).
    base = BASES[name]()
    e = R.principal(R.canonical(base)).e.reshape(2, 2)
    for v in range(8):
        x, y, z = CG.exponents(v)
        ev = R.principal(R.canonical(CG.variant(base, v))).e.reshape(2, 2)
        si, sj = int(y == 1), int(z == 1)
        for i, j in itertools.product(range(2), range(2)):
            assert ev[i, j] == e[i ^ si, j ^ sj], (v, i, j)
        assert R.principal(CG.variant(base, v)).E == R.principal(base).E


def test_splitmix64_reference_outputs():
    # The first outputs of SplitMix64 from state 0, as printed with the
    # generator's reference implementation.
    assert [CG.splitmix64(0, n) for n in range(4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                       0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_random_and_round_robin_selections():
    assert CG.select_round_robin(7, 2) == [n % 8 for n in range(8)]
    sel = CG.select_random(7, 3, seed=99)
    assert len(sel) == 1 + 7 + 49 and all(0 <= v < 8 for v in sel)
    assert sel == [CG.splitmix64(99, n) >> 61 for n in range(57)]
    assert CG.select_random(7, 3, seed=99) == sel and CG.select_random(7, 3, seed=100) != sel


@pytest.mark.parametrize("name", sorted(BASES))
def test_variant_trees_exact_on_integers(name):
    # a two-level tree using all eight variants computes A B exactly on
    # small integers, like the classical product
    base = BASES[name]()
    chosen = CG.select_round_robin(7, 2)
    assert set(chosen) == set(range(8))
    tree = CG.tree(base, 2, chosen)
    A = inputs.integers((36, 44), -4, 4, seed=5)
    B = inputs.integers((44, 28), -4, 4, seed=6)
    assert np.array_equal(F.fmm(A, B, tree), F.classical(A, B))


def _costs(base, levels, Amax, Bmax):
    cs = []
    chosen = CG.select_matrix(base, levels, Amax, Bmax, costs=cs)
    return chosen, cs


@pytest.mark.parametrize("name", sorted(BASES))
def test_matrix_selection_minimal_at_every_node(name):
    base = BASES[name]()
    g = np.random.default_rng(3)
    for levels in (1, 2):
        n = 1 << levels
        Amax = g.integers(1, 50, (n, n)).astype(float)
        Bmax = g.integers(1, 50, (n, n)).astype(float)
        chosen, costs = _costs(base, levels, Amax, Bmax)
        assert len(chosen) == CG.node_count(7, levels) == len(costs)
        for v, cs in zip(chosen, costs):
            assert cs[v] == min(cs) and v == cs.index(min(cs))
        # the root's costs by brute force over the tables: max over C blocks
        # of sum_r |w| (sum_i |u| a_i)(sum_j |v| b_j)
        qa = [Amax[p * n // 2:(p + 1) * n // 2, q * n // 2:(q + 1) * n // 2].max() for p in (0, 1) for q in (0, 1)]
        qb = [Bmax[p * n // 2:(p + 1) * n // 2, q * n // 2:(q + 1) * n // 2].max() for p in (0, 1) for q in (0, 1)]
        for v in range(8):
            c = R.canonical(CG.variant(base, v))
            s = np.abs(c.U).T @ np.array(qa)
            t = np.abs(c.V).T @ np.array(qb)
            assert costs[0][v] == float((np.abs(c.W) @ (s * t)).max())
        if levels == 2:
            # the children's costs by brute force too: child r of the
            # chosen root variant multiplies sum_i U_ir A_i by sum_j V_jr
            # B_j, whose 2 x 2 block bounds are sum_i |U_ir| (quadrant i of
            # Amax) and sum_j |V_jr| (quadrant j of Bmax)
            root = R.canonical(CG.variant(base, chosen[0]))
            for r in range(root.R):
                Ab = sum(abs(root.U[i, r]) * Amax[(i // 2) * 2:(i // 2) * 2 + 2, (i % 2) * 2:(i % 2) * 2 + 2]
                         for i in range(4))
                Bb = sum(abs(root.V[j, r]) * Bmax[(j // 2) * 2:(j // 2) * 2 + 2, (j % 2) * 2:(j % 2) * 2 + 2]
                         for j in range(4))
                qa2 = [Ab[p, q] for p in (0, 1) for q in (0, 1)]
                qb2 = [Bb[p, q] for p in (0, 1) for q in (0, 1)]
                for v in range(8):
                    c = R.canonical(CG.variant(base, v))
                    s2 = np.abs(c.U).T @ np.array(qa2)
                    t2 = np.abs(c.V).T @ np.array(qb2)
                    assert costs[1 + r][v] == float((np.abs(c.W) @ (s2 * t2)).max()), (r, v)


@pytest.mark.parametrize("name", sorted(BASES))
def test_matrix_selection_equivariance(name):
    # Variant v on relabelled blocks is variant v xor (the relabelling) on
    # the original ones, so the node costs permute exactly (integer block
    # maxima keep every cost exact): exchanging A's block rows (i) maps cost
    # v to v xor 1, A's block columns with B's block rows (k) to v xor 2,
    # B's block columns (j) to v xor 4.  (Strassen's costs are also
    # invariant under v -> v xor 7, its own symmetry, so ties are common.)
    base = BASES[name]()
    g = np.random.default_rng(11)
    for _ in range(20):
        Amax = g.integers(1, 100, (2, 2)).astype(float)
        Bmax = g.integers(1, 100, (2, 2)).astype(float)
        _, (cs,) = _costs(base, 1, Amax, Bmax)
        for (Ap, Bp), flip in (((Amax[::-1, :], Bmax), 1), ((Amax[:, ::-1], Bmax[::-1, :]), 2),
                               ((Amax, Bmax[:, ::-1]), 4)):
            _, (cp,) = _costs(base, 1, Ap, Bp)
            assert [cp[v] for v in range(8)] == [cs[v ^ flip] for v in range(8)], flip
        # the choice is the lowest index among the minima
        v = CG.select_matrix(base, 1, Amax, Bmax)[0]
        assert cs[v] == min(cs) and all(cs[u] > cs[v] for u in range(v))


def test_block_max_definition():
    X = np.arange(35, dtype=float).reshape(5, 7) - 17.0
    out = CG.block_max(X, 2, 3)   # blocks of 3 x 3, edge blocks 2 rows / 1 column
    assert out.shape == (2, 3)
    assert out[0, 0] == 17.0 and out[1, 2] == 17.0 and out[0, 2] == 11.0 and out[1, 0] == 13.0
    assert CG.block_max(np.zeros((3, 3)), 4, 4)[3, 3] == 0.0


@pytest.mark.parametrize("name", sorted(BASES))
def test_child_bounds_hold_and_are_attained(name):
    # The matrix-dependent selection passes bounds on the finest blocks of
    # each product's operands, S_r = sum_i U_ir A_i and T_r = sum_j V_jr B_j
    # (quadrants row-major, canonical tables), down the tree.  By the
    # triangle inequality max|block of S_r| <= sum_i |U_ir| max|block of
    # A_i|: checked on real matrices with random signs, and attained when
    # every quadrant is a sign-matched constant-block matrix.
    base = BASES[name]()
    g = np.random.default_rng(21)
    n, b = 4, 3                                   # a 4 x 4 grid of 3 x 3 blocks
    h = n * b // 2
    quad = lambda X, i: X[(i // 2) * h:(i // 2 + 1) * h, (i % 2) * h:(i % 2 + 1) * h]  # noqa: E731
    for v in range(8):
        c = R.canonical(CG.variant(base, v))
        for T in (c.U, c.V):
            for _ in range(5):
                X = g.standard_normal((n * b, n * b)) * np.exp2(g.integers(-3, 4, (n * b, n * b)))
                Xmax = CG.block_max(X, n, n)
                for r in range(c.R):
                    S = sum(float(T[i, r]) * quad(X, i) for i in range(4))
                    assert np.all(CG.block_max(S, 2, 2) <= CG.child_bounds(T, Xmax, r) * (1 + 1e-15))
            Xmax = g.integers(1, 50, (n, n)).astype(float)
            for r in range(c.R):
                X = np.kron(Xmax, np.ones((b, b)))
                for i in range(4):
                    quad(X, i)[...] *= np.sign(T[i, r]) if T[i, r] != 0 else 1.0
                S = sum(float(T[i, r]) * quad(X, i) for i in range(4))
                assert np.array_equal(CG.block_max(S, 2, 2), CG.child_bounds(T, Xmax, r))


def test_tree_nodes_in_level_order():
    # node n of the level-order list runs variant chosen[n]; a node's
    # children follow in product order, level by level: at three levels,
    # the child r2 of the root's child r1 is node 1 + R + R r1 + r2
    base = R.strassen()
    chosen = CG.select_random(7, 3, seed=5)
    t = CG.tree(base, 3, chosen)
    same = lambda a, b: (np.array_equal(a.U, b.U) and np.array_equal(a.V, b.V)  # noqa: E731
                         and np.array_equal(a.W, b.W))
    v = [CG.variant(base, k) for k in range(8)]
    assert same(t.rule, v[chosen[0]])
    for r1 in range(7):
        assert same(t.children[r1].rule, v[chosen[1 + r1]])
        for r2 in range(7):
            node = t.children[r1].children[r2]
            assert same(node.rule, v[chosen[8 + 7 * r1 + r2]]) and node.children == [None] * 7
