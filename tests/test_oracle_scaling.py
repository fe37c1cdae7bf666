"""Pins for the oracle's diagonal scaling (Sec. 6, App. D).

Pinned against: the worked examples' scaled matrices (Examples 6.2-6.5, with
z = 2^-2m so every square root is exact), Propositions 6.1 and 6.2,
Theorem 6.4 monotonicity, the closed forms of Lemma D.4, and exactness of
power-of-two scale / unscale.
"""
import numpy as np
import pytest

from oracle import scaling as Sc
from paper_1507_00687_gb300 import inputs

z = 2.0**-20
rz = 2.0**-10  # sqrt(z)


def test_example_6_1_outside():
    A = np.ones((2, 2))
    B = np.array([[z, 1], [z, 1]])
    st = Sc.repeated(A, B, "O")
    assert np.array_equal(st.A, np.ones((2, 2)))
    assert np.array_equal(st.B, np.ones((2, 2)))


def test_example_6_2_inside():
    A = np.array([[1, z], [1, z]])
    B = np.array([[z, z], [1, 1]])
    assert np.array_equal(Sc.repeated(A, B, "O").A, A)   # outside does nothing
    st = Sc.repeated(A, B, "I")
    assert np.array_equal(st.d, [rz, 1 / rz])
    assert np.array_equal(st.A, np.full((2, 2), rz))
    assert np.array_equal(st.B, np.full((2, 2), rz))


def test_example_6_3_order():
    A = np.array([[1, 1 / z], [1, 1]])
    B = np.array([[z, 1], [z, 1]])
    oi = Sc.repeated(A, B, "OI")
    assert np.array_equal(oi.A, [[z, 1], [1, 1]])
    assert np.array_equal(oi.B, np.ones((2, 2)))
    io = Sc.repeated(A, B, "IO")
    assert np.array_equal(io.A, [[rz, 1], [1, rz]])
    assert np.array_equal(io.B, [[rz, rz], [1, 1]])
    # Reading: the printed C' (1,1) entry "1 + z^(1/4)" is 1 + z.
    assert np.allclose(io.A @ io.B, [[1 + z, 1 + z], [2 * rz, 2 * rz]], rtol=0, atol=0)


def test_example_6_4_order():
    A = np.array([[1, z], [z, z]])
    B = np.array([[z, 1], [1, 1 / z]])
    io = Sc.repeated(A, B, "IO")
    assert np.array_equal(io.A, [[1, 1], [z, 1]])
    assert np.array_equal(io.B, np.ones((2, 2)))
    # Reading: the printed O-then-I matrices do not follow from Alg. 3 on
    # these A, B; Alg. 3 gives the following (pinned by hand).
    oi = Sc.repeated(A, B, "OI")
    assert np.array_equal(oi.A, [[rz, z], [rz, 1]])
    assert np.array_equal(oi.B, [[rz, rz], [1, 1]])


def test_example_6_5_unchanged():
    A = np.array([[1, z], [z, 1]])
    for steps in ("O", "I", "OI", "IO", "OIOI"):
        st = Sc.repeated(A, A, steps)
        assert np.array_equal(st.A, A) and np.array_equal(st.B, A)
        # power-of-two mode: the O step maps the unit row maxima to 1/2 and
        # nothing else changes (all scales are powers of two already)
        p2 = Sc.pow2_repeated(A, A, steps)
        assert np.array_equal(p2.A, A / (2.0 if "O" in steps else 1.0))


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_propositions_6_1_6_2(kind):
    A, B = inputs.paper_distribution(kind, 64, seed=kind)
    o = Sc.repeated(A, B, "O")
    assert np.allclose(np.abs(o.A).max(axis=1), 1.0) and np.allclose(np.abs(o.B).max(axis=0), 1.0)
    i = Sc.repeated(A, B, "I")
    assert np.allclose(np.abs(i.A).max(axis=0), np.abs(i.B).max(axis=1))
    # Prop 6.2: ||A'|| ||B'|| = max_{i,k,j} |a_ik||b_kj|
    assert np.isclose(np.abs(i.A).max() * np.abs(i.B).max(),
                      np.max(np.abs(A).max(axis=0) * np.abs(B).max(axis=1)))
    # unscale recovers C exactly in exact arithmetic
    for steps in ("O", "I", "OI", "IO", "OIOI"):
        st = Sc.repeated(A, B, steps)
        assert np.allclose(Sc.unscale(st.A @ st.B, st), A @ B, rtol=1e-12, atol=0)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_pow2_scaling_invariants(kind):
    A, B = inputs.paper_distribution(kind, 48, seed=10 + kind)
    o = Sc.pow2_repeated(A, B, "O")
    ra = np.abs(o.A).max(axis=1)
    assert np.all((ra >= 0.5) & (ra < 1.0))
    cb = np.abs(o.B).max(axis=0)
    assert np.all((cb >= 0.5) & (cb < 1.0))
    i = Sc.pow2_repeated(A, B, "I")
    ratio = np.abs(i.B).max(axis=1) / np.abs(i.A).max(axis=0)
    assert np.all((ratio > 0.5) & (ratio < 4.0))
    for steps in ("O", "I", "OI", "IO", "OIOI", "IOIO"):
        st = Sc.pow2_repeated(A, B, steps)
        Ap, Bp = Sc.pow2_apply(A, B, st.eA, st.d, st.eB)
        assert np.array_equal(Ap, st.A) and np.array_equal(Bp, st.B)   # exact
        assert np.allclose(Sc.pow2_unscale(st.A @ st.B, st.eA, st.eB), A @ B, rtol=1e-12, atol=0)


def test_pow2_zero_rows_and_cols():
    A = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0]])
    B = np.array([[0.0, 5.0], [0.0, 0.25], [0.0, 1.0]])
    st = Sc.pow2_repeated(A, B, "OIOI")
    assert st.eA[0] == 0 and st.eB[0] == 0
    assert np.all(np.isfinite(st.A)) and np.all(np.isfinite(st.B))
    # an I step with one side zero leaves d_k = 0, whatever the other side
    # holds: column 0 of A is zero while row 0 of B is large, row 1 of B is
    # zero while column 1 of A is large; k = 2 has both sides, max 2 in A
    # (frexp exponent 2) and 1 in B (exponent 1): floor((1 - 2) / 2) = -1
    A = np.array([[0.0, 64.0, 1.0], [0.0, 32.0, 2.0]])
    B = np.array([[64.0, 128.0], [0.0, 0.0], [1.0, 0.5]])
    st = Sc.pow2_repeated(A, B, "I")
    assert list(st.d) == [0, 0, -1]
    # the real-valued steps give zero rows / columns the scale 1 as well
    A = np.array([[0.0, 0.0], [3.0, 1.0]])
    B = np.array([[0.0, 2.0], [0.0, 5.0]])
    st = Sc.repeated(A, B, "OI")
    assert st.r[0] == 1.0 and st.s[0] == 1.0 and st.r[1] == 3.0 and st.s[1] == 5.0


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_theorem_6_4_monotone(kind):
    A, B = inputs.paper_distribution(kind, 40, seed=20 + kind)
    for first in ("O", "I"):
        st = Sc.start(A, B)
        prev = np.outer(st.r, st.s) * np.abs(st.A).max() * np.abs(st.B).max()
        for t in range(12):
            st = Sc.o_step(st) if (t % 2 == 0) == (first == "O") else Sc.i_step(st)
            cur = np.outer(st.r, st.s) * np.abs(st.A).max() * np.abs(st.B).max()
            assert np.all(cur <= prev * (1 + 1e-12))
            prev = cur


def test_lemma_D4_closed_forms():
    # A = [[1, 0], [1, 2^(-2^v)]], B = I, starting with an O step (t0 = 0):
    # A^(t) = [[1, 0], [1, 2^(-2^(v - t/2))]], r = [1, 1],
    # s = [1, 2^(-2^v (1 - 2^(-t/2)))], B^(t) = I for even t;
    # A^(t+1) = [[1,0],[1, 2^(-2^(v-t/2-1))]], B^(t+1) = diag(1, same).
    v = 6
    A = np.array([[1.0, 0.0], [1.0, 2.0 ** -(2**v)]])
    B = np.eye(2)
    st = Sc.start(A, B)
    st = Sc.o_step(st)  # t = 1 is the first O step's result; t0 = 1 in this count
    for h in range(v):  # h = (t - t0)/2
        assert np.array_equal(st.A, [[1, 0], [1, 2.0 ** -(2 ** (v - h))]])
        assert np.array_equal(st.B, np.eye(2))
        assert np.array_equal(st.r, [1, 1])
        assert np.array_equal(st.s, [1, 2.0 ** -(2**v * (1 - 2.0 ** -h))])
        st = Sc.i_step(st)
        assert np.array_equal(st.A, [[1, 0], [1, 2.0 ** -(2 ** (v - h - 1))]])
        assert np.array_equal(st.B, [[1, 0], [0, 2.0 ** -(2 ** (v - h - 1))]])
        st = Sc.o_step(st)


# ---------------------------------------------------------------- adaptive Alg. 3 (tau stopping criterion)

def _lemma_d4_stop(v, L):
    # In the Lemma D.4 example (first O step at t = 1) the I step after h
    # O-I rounds has factor 2^(2^(v-h-1)) on the second column and the O step
    # after it the column factor 2^(-2^(v-h-1)) on B; with 1 + tau = 2^L the
    # I test holds iff 2^(v-h-1) <= L/4 and the O test iff 2^(v-h-1) <= L/2.
    # The O step at t = 2h+1 (h >= 1) tests the same inequality as the I step
    # at 2h+2, so the first pass is t = 2 (I test at h = 0) or t = 2h*+3.
    if 2 ** (v - 1) <= L / 4:
        return 2
    h = 0
    while 2 ** (v - h - 1) > L / 2:
        h += 1
    return 2 * h + 3


@pytest.mark.parametrize("L", [4, 8, 16, 64])
def test_adaptive_stop_step_closed_form_lemma_d4(L):
    v = 6
    A = np.array([[1.0, 0.0], [1.0, 2.0 ** -(2**v)]])
    B = np.eye(2)
    tau = 2.0**L - 1
    want = _lemma_d4_stop(v, L)
    assert want <= 2 * (v - 2) + 3  # every exponent along the way is an integer
    _, t = Sc.adaptive(A, B, tau, 40)
    assert t == want
    _, t2 = Sc.pow2_adaptive(A, B, tau, 40)
    assert t2 == want
    # a cap below the stopping step returns the cap
    _, t3 = Sc.adaptive(A, B, tau, want - 1)
    assert t3 == want - 1


def _mu_max(st, lim):
    # relative distance of r_i s_j ||A'|| ||B'|| from its limit (Sec. 6.3)
    cur = np.outer(st.r, st.s) * np.abs(st.A).max() * np.abs(st.B).max()
    ref = np.outer(lim.r, lim.s) * np.abs(lim.A).max() * np.abs(lim.B).max()
    return float(np.max(np.abs(cur - ref) / np.abs(ref)))


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("tau", [0.5, 1e-2, 1e-4])
@pytest.mark.parametrize("first", ["O", "I"])
def test_adaptive_stopping_theorem(kind, tau, first):
    # The theorem of Sec. 6.3: once the test passes, the products
    # r_i s_j ||A'|| ||B'|| are within relative distance tau of their limit.
    # The limit is approximated by continuing the same alternation until the
    # scales stop moving.
    A, B = inputs.paper_distribution(kind, 40, seed=40 + kind)
    st, t = Sc.adaptive(A, B, tau, 200, first)
    assert t < 200
    kinds = Sc._kinds(first, 4000)
    lim = st
    for k in kinds[t:t + 3000]:
        lim = Sc.o_step(lim) if k == "O" else Sc.i_step(lim)
    assert _mu_max(st, lim) <= tau * (1 + 1e-6)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_pow2_adaptive_stops_at_a_fixed_point(kind):
    # With tau < 3 no power-of-two factor other than 1 passes the I test, and
    # an O factor passes only if it is >= 1; an I step that passes changes no
    # exponent, after which further steps change nothing either.
    A, B = inputs.paper_distribution(kind, 64, seed=60 + kind)
    st, t = Sc.pow2_adaptive(A, B, 1e-3, 60)
    assert t < 60
    nxt = Sc.pow2_o_step(st) if t % 2 == 0 else Sc.pow2_i_step(st)
    if t % 2 == 0:  # the last step was an I step
        for s in (Sc.pow2_o_step(st), Sc.pow2_i_step(Sc.pow2_o_step(st))):
            assert np.array_equal(s.eA, st.eA) and np.array_equal(s.d, st.d) and np.array_equal(s.eB, st.eB)
    else:  # an O step: no exponent went down
        prev = Sc.pow2_repeated(A, B, Sc._kinds("O", t - 1))
        assert np.all(st.eA >= prev.eA) and np.all(st.eB >= prev.eB)
    assert nxt is not None
    # the result equals the fixed sequence of the same length
    ref = Sc.pow2_repeated(A, B, Sc._kinds("O", t))
    assert np.array_equal(ref.eA, st.eA) and np.array_equal(ref.d, st.d) and np.array_equal(ref.eB, st.eB)


def test_adaptive_zero_steps_and_no_o_step():
    A, B = inputs.paper_distribution(2, 16, seed=1)
    st, t = Sc.pow2_adaptive(A, B, 0.1, 0)
    assert t == 0 and not st.eA.any() and not st.d.any() and not st.eB.any()
    # a single I step is never tested (no O step before it)
    _, t = Sc.pow2_adaptive(A, B, 1e9, 1, "I")
    assert t == 1
    # with a huge tau the first tested step passes: t0 + 1
    _, t = Sc.pow2_adaptive(A, B, 1e30, 10, "O")
    assert t == 2
    _, t = Sc.pow2_adaptive(A, B, 1e30, 10, "I")
    assert t == 3
