"""Pins for the oracle's recursive fast multiplication and its bounds.

Pinned against: exact integer arithmetic (brute force and classical), exact
rational brute force on tiny inputs, Theorem 4.1 / 4.2 and the componentwise
first-order bound from the proof of Theorem 4.1, and Example 6.1.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import fmm as F
from oracle import precision as P
from oracle import rules as R
from paper_1507_00687_gb300 import inputs

S, Wg, C121 = R.strassen(), R.winograd(), R.classical(1, 2, 1)


@pytest.mark.parametrize("rules", [[S, S], [Wg], [Wg, Wg, Wg], [S, C121, S],
                                   [R.fast323()], [S, R.fast323()]],
                         ids=["S2", "W1", "W3", "S-C121-S", "f323", "S-f323"])
def test_integer_inputs_exact(rules):
    # n=16, entries in [-4, 4]: every intermediate is a small integer, so the
    # fast algorithm must equal the classical product exactly.
    A = inputs.integers((16, 16), -4, 4, seed=1)
    B = inputs.integers((16, 16), -4, 4, seed=2)
    assert np.array_equal(F.fmm(A, B, F.uniform(rules)), A @ B)


@pytest.mark.parametrize("shape", [(13, 7, 9), (1, 1, 1), (5, 3, 2), (17, 33, 8), (0, 4, 3)])
def test_ragged_shapes_padding_exact(shape):
    M, K, N = shape
    A = inputs.integers((M, K), -3, 3, seed=3)
    B = inputs.integers((K, N), -3, 3, seed=4)
    for rules in ([S], [S, S], [Wg, C121]):
        out = F.fmm(A, B, F.uniform(rules))
        assert out.shape == (M, N)
        assert np.array_equal(out, A @ B)


def test_brute_force_all_sign_patterns_2x2():
    # Every A, B in {-1, 1}^{2x2}: compare with the exact rational product.
    tree = F.uniform([S])
    for bits in itertools.product((-1, 1), repeat=8):
        A = np.array(bits[:4], float).reshape(2, 2)
        B = np.array(bits[4:], float).reshape(2, 2)
        exact = F.classical_exact([[Fraction(int(x)) for x in r] for r in A],
                                  [[Fraction(int(x)) for x in r] for r in B])
        assert np.array_equal(F.fmm(A, B, tree), np.array(exact, dtype=float))


def test_brute_force_rationals_4x4():
    g = np.random.default_rng(5)
    for trial in range(20):
        A = [[Fraction(int(g.integers(-9, 10)), int(g.integers(1, 5))) for _ in range(4)] for _ in range(4)]
        B = [[Fraction(int(g.integers(-9, 10)), int(g.integers(1, 5))) for _ in range(4)] for _ in range(4)]
        exact = np.array(F.classical_exact(A, B), dtype=float)
        got = F.fmm(np.array(A, float), np.array(B, float), F.uniform([Wg, S]))
        assert np.max(np.abs(got - exact)) <= 64 * 2.0**-53 * np.max(np.abs(exact)) + 1e-300


def _fixed(shape, seed, bits=48):
    # U[-1,1] rounded to 48 fractional bits, so classical_exact_fixed gives
    # the exact product.
    X = inputs.uniform(shape, -1.0, 1.0, seed)
    return np.round(X * 2**bits) / 2**bits


def test_exact_fixed_product_against_fractions():
    A = _fixed((5, 7), 1)
    B = _fixed((7, 3), 2)
    want = F.classical_exact([[Fraction(x) for x in r] for r in A], [[Fraction(x) for x in r] for r in B])
    got = F.classical_exact_fixed(A, B)
    den = 1 << 96
    assert all(Fraction(int(got[i, j]), den) == want[i][j] for i in range(5) for j in range(3))


def test_theorem_4_1_config_small():
    # Strassen, L = 2, n = 256, FP64, A, B ~ U[-1, 1]; bound of Theorem 4.1:
    # (K/K0^L + Q L)(K/K0^L) E^L ||A|| ||B|| eps = (64 + 16) 64 144 eps.
    A = _fixed((256, 256), 11)
    B = _fixed((256, 256), 12)
    C = F.exact_to_float(F.classical_exact_fixed(A, B))
    got = F.fmm(A, B, F.uniform([S, S]))
    eps = 2.0**-53
    bound = F.bound_uniform([S, S], 256, np.abs(A).max(), np.abs(B).max(), eps)
    assert bound == pytest.approx((64 + 16) * 64 * 144 * eps * np.abs(A).max() * np.abs(B).max())
    assert bound <= 8.2e-11
    err = F.err_max(got, C)
    assert 0 < err <= bound
    # componentwise form from the proof: |E_k| <= delta eps G (first order)
    G = F.growth(A, B, F.uniform([S, S]))
    delta = 256 / 4 + 2 * R.principal(S).Q
    assert np.all(np.abs(got - C) <= delta * eps * G * (1 + 1e-6))


@pytest.mark.parametrize("rules", [[Wg, C121, Wg], [S, Wg], [R.fast323(), S]],
                         ids=["W-C-W", "S-W", "323-S"])
def test_theorem_4_2_uniform_nonstationary(rules):
    tree = F.uniform(rules)
    pm, pk, pn = F.dims(tree)
    A = _fixed((pm * 8, pk * 8), 21)
    B = _fixed((pk * 8, pn * 8), 22)
    C = F.exact_to_float(F.classical_exact_fixed(A, B))
    got = F.fmm(A, B, tree)
    bound = F.bound_uniform(rules, A.shape[1], np.abs(A).max(), np.abs(B).max(), 2.0**-53)
    assert F.err_max(got, C) <= bound
    assert F.bound_tree(tree, A.shape[1], np.abs(A).max(), np.abs(B).max(), 2.0**-53) == pytest.approx(bound)


def test_theorem_special_cases():
    # L = 0: K^2 ||A|| ||B|| eps (Sec. 4.3 remark)
    assert F.bound_uniform([], 100, 1.0, 1.0, 1.0) == 100**2
    # full recursion, square: (1 + Q L) E^L ||A|| ||B|| eps
    L = 5
    assert F.bound_uniform([S] * L, 2**L, 1.0, 1.0, 1.0) == (1 + 8 * L) * 12.0**L


def test_growth_bound_relation():
    # G <= (K/K0^L) E^L ||A|| ||B|| entrywise (last step of the proof)
    A = inputs.uniform((32, 32), -1, 1, 31)
    B = inputs.uniform((32, 32), -1, 1, 32)
    for rules in ([S], [S, S], [Wg, Wg]):
        G = F.growth(A, B, F.uniform(rules))
        E = np.prod([R.principal(r).E for r in rules])
        assert G.max() <= (32 / 2**len(rules)) * E * np.abs(A).max() * np.abs(B).max() * (1 + 1e-12)
        assert np.all(G >= np.abs(A) @ np.abs(B) * (1 - 1e-12))


def test_example_6_1_relative_error():
    # Example 6.1: Strassen's c11 has relative error O(eps/z) without scaling,
    # O(eps) with outside scaling.  Small perturbations make the roundings
    # real (the example's own remark).
    z = 1.2345e-9
    A = np.array([[1.0, 1.0 + 2**-30], [1.0 - 2**-31, 1.0]])
    B = np.array([[z, 1.0 + 2**-29], [z * (1 + 2**-28), 1.0]])
    C = np.array(F.classical_exact([[Fraction(x) for x in r] for r in A],
                                   [[Fraction(x) for x in r] for r in B]), dtype=float)
    plain = F.fmm(A, B, F.uniform([S]))
    rel_plain = abs(plain[0, 0] - C[0, 0]) / abs(C[0, 0])
    from oracle import scaling as Sc
    st = Sc.repeated(A, B, "O")
    scaled = Sc.unscale(F.fmm(st.A, st.B, F.uniform([S])), st)
    rel_scaled = abs(scaled[0, 0] - C[0, 0]) / abs(C[0, 0])
    assert rel_plain > 1e3 * 2.0**-53
    assert rel_scaled < 8 * 2.0**-53


def test_emulated_leaf_formats_bracket():
    # bf16x3 emulation is far closer to the exact product than bf16.
    A = inputs.uniform((64, 64), -1, 1, 41)
    B = inputs.uniform((64, 64), -1, 1, 42)
    C = A @ B
    tree = F.uniform([S])
    e16 = F.err_max(F.fmm(A, B, tree, leaf=F.leaf_rounded("bf16"), dtype=np.float32), C)
    ex3 = F.err_max(F.fmm(A, B, tree, leaf=F.leaf_bf16x3, dtype=np.float32), C)
    assert ex3 < e16 / 64
    G = F.growth(A, B, tree)
    assert ex3 <= (3 * 2.0**-16 + 8 * 2.0**-24) * G.max()


def test_flop_count():
    f = F.flop_count(F.uniform([S, S]), 4096, 4096, 4096)
    assert f["leaves"] == 49
    assert f["leaf"] == 2.0 * 49 * 1024**3


# ---------------------------------------------------------------- scaling between recursive steps

def test_between_scaling_is_exact_on_integers():
    # Power-of-two scaling of each root product's pair cancels exactly: with
    # exact arithmetic the result is still the classical product.
    from oracle import rules as OR
    rng = np.random.default_rng(5)
    for rules in ([OR.strassen(), OR.strassen()], [OR.winograd(), OR.winograd()], [OR.strassen(), OR.fast323()]):
        tree = F.uniform(rules)
        A = rng.integers(-4, 5, size=(24, 20)).astype(np.float64)
        B = rng.integers(-4, 5, size=(20, 18)).astype(np.float64)
        # spread the magnitudes so that nonzero exponents occur
        A *= np.exp2(rng.integers(-6, 7, size=(1, 20)))
        B *= np.exp2(rng.integers(-6, 7, size=(20, 1)))
        assert np.array_equal(F.fmm(A, B, tree, between=True), A @ B)


def test_between_exponents_balance_each_pair():
    # After the scaling, e(max |T_r[k, :]|) - e(max |S_r[:, k]|) is 0 or 1
    # for every root product r and column k with both sides nonzero (the
    # I-step property, Sec. 6.2), and d is 0 where a side is zero.
    from oracle import rules as OR
    from oracle.rules import canonical
    rng = np.random.default_rng(9)
    rules = [OR.winograd(), OR.strassen()]
    tree = F.uniform(rules)
    A = rng.uniform(-1, 1, size=(16, 16)) * np.exp2(rng.integers(-20, 21, size=(1, 16)))
    B = rng.uniform(-1, 1, size=(16, 16)) * np.exp2(rng.integers(-20, 21, size=(16, 1)))
    A[:, 3] = 0.0  # a zero column of A: its S columns vanish for some r
    d = F.between_exponents(A, B, tree)
    r = canonical(rules[0])
    kb = 8
    Ab = [A[p * 8:(p + 1) * 8, q * 8:(q + 1) * 8].astype(np.float32) for p in range(2) for q in range(2)]
    Bb = [B[p * 8:(p + 1) * 8, q * 8:(q + 1) * 8].astype(np.float32) for p in range(2) for q in range(2)]
    checked = 0
    for j in range(r.R):
        S = sum(np.float32(r.U[i, j]) * Ab[i] for i in range(4) if r.U[i, j] != 0)
        T = sum(np.float32(r.V[i, j]) * Bb[i] for i in range(4) if r.V[i, j] != 0)
        for k in range(kb):
            cs, rt = np.abs(S[:, k]).max(), np.abs(T[k, :]).max()
            if cs == 0 or rt == 0:
                assert d[j][k] == 0
                continue
            es = np.frexp(cs * 2.0 ** d[j][k])[1]
            et = np.frexp(rt * 2.0 ** -d[j][k])[1]
            assert et - es in (0, 1), (j, k, et - es)
            checked += 1
    assert checked > 20


def _R(name):
    return {"strassen": R.strassen, "winograd": R.winograd, "fast323": R.fast323,
            "classical121": lambda: R.classical(1, 2, 1), "classical211": lambda: R.classical(2, 1, 1)}[name]()


@pytest.mark.parametrize("names", [["strassen"], ["winograd", "classical121"], ["strassen", "fast323"],
                                   ["winograd", "classical121", "strassen", "classical211"]])
def test_growth_entries_equal_full_growth(names):
    # The sampled-entry growth (flattened rule, Eq. 4.4) against the
    # recursive evaluation of Eq. 3.2 on |A|, |B|, including padded edges.
    rules = [_R(n) for n in names]
    g = np.random.default_rng(7)
    M, K, N = 37, 53, 41
    A = g.uniform(-1, 1, size=(M, K))
    B = g.uniform(-1, 1, size=(K, N))
    full = F.growth(A, B, F.uniform(rules))
    rows = g.integers(0, M, size=40)
    cols = g.integers(0, N, size=40)
    part = F.growth_entries(A, B, rules, rows, cols)
    assert np.allclose(part, full[rows, cols], rtol=1e-12, atol=0)
    # the growth of a product of nonnegative matrices is the product itself
    # when every coefficient is nonnegative and each entry lies in one term
    Ac, Bc = np.abs(A), np.abs(B)
    assert np.allclose(F.growth_entries(Ac, Bc, [R.classical(1, 2, 1)], rows, cols), (Ac @ Bc)[rows, cols])


def test_error_norms_on_a_hand_computed_case():
    # Sec. 6.5 measures the componentwise relative error max |c_hat - c| / |c|
    # over the entries with c != 0.  Worked by hand on a 2 x 2 case:
    #   c = 2,  c_hat = 2.2  -> 0.2 / 2 = 0.1
    #   c = 0,  c_hat = 7    -> skipped (the ratio is undefined there)
    #   c = -4, c_hat = -3   -> 1 / 4  = 0.25   (dividing by |c_hat| would give 1/3)
    #   c = 1,  c_hat = 1    -> 0
    # so the componentwise error is 0.25 and the max-norm error is 7.  A
    # version that divides by |c_hat| gives 1.0 (the skipped entry's 7/7),
    # one that keeps zero entries gives inf, one that drops the absolute
    # value of the denominator gives -0.25 or 0.1.
    C = np.array([[2.0, 0.0], [-4.0, 1.0]])
    C_hat = np.array([[2.2, 7.0], [-3.0, 1.0]])
    assert F.err_componentwise(C_hat, C) == pytest.approx(0.25, rel=1e-15)
    assert F.err_max(C_hat, C) == 7.0
    # all-zero reference: no entry defines a ratio
    assert F.err_componentwise(np.ones((2, 2)), np.zeros((2, 2))) == 0.0
    # invariant: scaling both by the same nonzero factor leaves the
    # componentwise error unchanged and scales the max-norm error
    assert F.err_componentwise(-8.0 * C_hat, -8.0 * C) == pytest.approx(0.25, rel=1e-15)
    assert F.err_max(-8.0 * C_hat, -8.0 * C) == 56.0


def test_sums_follow_index_order_in_the_working_precision():
    # Eq. 4.3's model: S_r, T_r and C_k are sequential sums in index order,
    # each step rounded to the working precision.  In FP32, 1 + 2^-24 is a
    # tie that rounds to 1 (even), so 1 + 2^-24 + 2^-24 stays 1 in index
    # order but is 1 + 2^-23 if the two small terms meet first.  Winograd
    # (flattened, row-major): S_2 = a11 + a12 - a21 - a22,
    # T_5 = b11 - b12 + b22, c12 = m1 + m3 + m5 + m6.
    u = 2.0 ** -24
    A = np.array([[1.0, u], [-u, 0.0]])
    B = np.array([[1.0, -u], [0.0, u]])
    M = {0: 1.0, 2: u, 4: u, 5: 0.0}
    rec = []

    def leaf(S, T):
        rec.append((float(S[0, 0]), float(T[0, 0])))
        return np.array([[M.get(len(rec) - 1, 0.0)]])
    C = F.fmm(A, B, F.uniform([Wg]), leaf=leaf, dtype=np.float32)
    assert rec[2][0] == 1.0 and rec[5][1] == 1.0 and C[0, 1] == 1.0
    rec.clear()
    C = F.fmm(A, B, F.uniform([Wg]), leaf=leaf, dtype=np.float64)
    assert rec[2][0] == 1 + 2 * u and rec[5][1] == 1 + 2 * u and C[0, 1] == 1 + 2 * u


def test_between_exponents_come_from_fp32_sums():
    # The between-steps exponents are taken from the root's sums formed in
    # FP32, the precision the operand sums are formed in: T_1 of Strassen's
    # first product is b11 + b22 = 0.75 + (0.25 - 2^-26), which is 1 - 2^-26
    # exactly (frexp exponent 0) but 1 in FP32 (exponent 1); with
    # S_1 = a11 + a22 = 1, d = floor((e(T) - e(S)) / 2) is 0, not -1.
    A = np.array([[1.0, 0.0], [0.0, 0.0]])
    B = np.array([[0.75, 0.0], [0.0, 0.25 - 2.0 ** -26]])
    d = F.between_exponents(A, B, F.uniform([S, S]))
    assert list(d[0]) == [0]


def test_flop_count_on_a_rectangular_plan():
    # <2,1,1> over the rotated <3,3,2>: pm = 6, pk = 3, pn = 2, 2 x 15
    # leaves; leaf flops 2 R^L (Mp/pm)(Kp/pk)(Np/pn) on the padded shape.
    plan = F.uniform([R.classical(2, 1, 1), R.rotate(R.fast323())])
    assert F.dims(plan) == (6, 3, 2)
    f = F.flop_count(plan, 12, 9, 4)
    assert f["leaves"] == 30 and f["leaf"] == 2.0 * 30 * 2 * 3 * 2 and f["classical"] == 2.0 * 12 * 9 * 4
    assert F.flop_count(plan, 13, 9, 5)["leaf"] == 2.0 * 30 * 3 * 3 * 3


def test_delta_vector_entries_of_one_level():
    # Sec. 4.5 / Def. 4.1 for one Strassen level: delta_k = gamma_k + max
    # over the products feeding C block k of alpha_r + beta_r (canonical
    # order c11, c12, c21, c22): c11 = m1 + m4 - m5 + m7 -> 4 + 4,
    # c12 = m3 + m5 -> 2 + 3, c21 = m2 + m4 -> 2 + 3, c22 = m1 - m2 + m3 + m6
    # -> 4 + 4.  Two levels add each path's counts: max is 8 + 8.
    assert list(F.delta_vector(F.uniform([S]))) == [8.0, 5.0, 5.0, 8.0]
    assert F.delta_vector(F.uniform([S, S])).max() == 16.0


def test_rounded_leaves_round_both_operands():
    # 1 + 2^-8 is a bf16 tie (and 1 + 2^-11 an fp16 one) that rounds to 1:
    # the leaf multiplies the rounded S and T, so the product is exactly 1.
    for fmt, u in (("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)):
        x = np.array([[1.0 + u]])
        assert F.leaf_rounded(fmt)(x, x)[0, 0] == 1.0


def test_growth_with_between_scaling_assembled_by_hand():
    # With scaling between recursive steps, root product r's absolute sums
    # |S_r| = sum_i |U_ir| |A_i| and |T_r| = sum_j |V_jr| |B_j| are scaled by
    # 2^d (columns of S_r) and 2^-d (rows of T_r), d from the root's signed
    # sums; the lower levels' growth of that scaled pair, weighted by |W|,
    # gives G.  Assembled here block by block from the growth of the lower
    # plan, with inputs whose exponents are not all zero.
    g = np.random.default_rng(8)
    n = 16
    A = g.uniform(-1, 1, (n, n)) * np.exp2(g.integers(-6, 7, (1, n)))
    B = g.uniform(-1, 1, (n, n)) * np.exp2(g.integers(-6, 7, (n, 1)))
    plan = F.uniform([S, Wg])
    d = F.between_exponents(A, B, plan)
    assert any(np.any(v != 0) for v in d)
    c = R.canonical(S)
    h = n // 2
    Ab = [np.abs(A[p * h:(p + 1) * h, q * h:(q + 1) * h]) for p in (0, 1) for q in (0, 1)]
    Bb = [np.abs(B[p * h:(p + 1) * h, q * h:(q + 1) * h]) for p in (0, 1) for q in (0, 1)]
    G = np.zeros((n, n))
    for r in range(7):
        Sr = sum(abs(c.U[i, r]) * Ab[i] for i in range(4)) * np.exp2(d[r].astype(float))[None, :]
        Tr = sum(abs(c.V[j, r]) * Bb[j] for j in range(4)) * np.exp2(-d[r].astype(float))[:, None]
        Gr = F.growth(Sr, Tr, F.uniform([Wg]))
        for k in range(4):
            p, q = divmod(k, 2)
            G[p * h:(p + 1) * h, q * h:(q + 1) * h] += abs(c.W[k, r]) * Gr
    assert np.allclose(F.growth(A, B, plan, between=True), G, rtol=1e-14, atol=0)
    assert not np.allclose(F.growth(A, B, plan), G, rtol=1e-6, atol=0)
