"""Diagonal scaling of Sec. 6: outside (Alg. 1), inside (Alg. 2) and
repeated outside-inside (Alg. 3), real-valued and rounded to powers of two.

Oracle module (test infrastructure only; see the package docstring).

State after any sequence of steps (Eq. 6.3 with D_A, D_B, D diagonal):
    A' = D_A^{-1} A D,   B' = D^{-1} B D_B^{-1},   C = D_A (A' B') D_B.
Power-of-two mode (reading of the remark in Sec. 6 that the scales can be
rounded to powers of two so that applying them is exact):
  O step: the row scale of A' is 2^e with e the frexp exponent of the row's
          max-abs (so the scaled row max lies in [1/2, 1)); likewise for the
          columns of B'.
  I step: d_k = floor((e(max_j |B'_kj|) - e(max_i |A'_ik|)) / 2) with e the
          frexp exponent -- the power of two nearest below-or-at the square
          root of Eq. 6.6 in exponent arithmetic.
  All-zero rows / columns (excluded by Sec. 6.1) get scale 1 (exponent 0);
  an I step with either side all-zero gets d_k = 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _fexp(x: np.ndarray) -> np.ndarray:
    """frexp exponent e with x = f 2^e, 1/2 <= f < 1 (x > 0)."""
    return np.frexp(x)[1].astype(np.int64)


@dataclass
class Scaled:
    A: np.ndarray            # A'
    B: np.ndarray            # B'
    r: np.ndarray            # diag of D_A
    s: np.ndarray            # diag of D_B
    d: np.ndarray            # diag of the cumulative inside scale D
    history: list = field(default_factory=list)  # (kind, factors) per step


# ---------------------------------------------------------------------------
# Real-valued (the algorithms as stated)
# ---------------------------------------------------------------------------

def o_step(st: Scaled) -> Scaled:
    """O step of Alg. 3 (Alg. 1 when applied once to unscaled inputs)."""
    rp = np.max(np.abs(st.A), axis=1) if st.A.shape[1] else np.zeros(st.A.shape[0])
    sp = np.max(np.abs(st.B), axis=0) if st.B.shape[0] else np.zeros(st.B.shape[1])
    rp = np.where(rp > 0, rp, 1.0)
    sp = np.where(sp > 0, sp, 1.0)
    A = st.A / rp[:, None]
    B = st.B / sp[None, :]
    return Scaled(A, B, st.r * rp, sp * st.s, st.d, st.history + [("O", (rp, sp))])


def i_step(st: Scaled) -> Scaled:
    """I step of Alg. 3 (Alg. 2 when applied once): D = diag(sqrt(
    max_j |B'_kj| / max_i |A'_ik|)) (Eq. 6.6), A' <- A' D, B' <- D^{-1} B'."""
    ca = np.max(np.abs(st.A), axis=0) if st.A.shape[0] else np.zeros(st.A.shape[1])
    rb = np.max(np.abs(st.B), axis=1) if st.B.shape[1] else np.zeros(st.B.shape[0])
    ok = (ca > 0) & (rb > 0)
    D = np.ones_like(ca)
    D[ok] = np.sqrt(rb[ok] / ca[ok])
    return Scaled(st.A * D[None, :], st.B / D[:, None], st.r, st.s, st.d * D,
                  st.history + [("I", (D,))])


def start(A, B) -> Scaled:
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return Scaled(A.copy(), B.copy(), np.ones(A.shape[0]), np.ones(B.shape[1]),
                  np.ones(A.shape[1]))


def repeated(A, B, steps: str) -> Scaled:
    """Alg. 3 with a fixed step sequence, e.g. "O" (Alg. 1), "I" (Alg. 2),
    "OI" (outside then inside), "OIOI" (2-times repeated outside-inside)."""
    st = start(A, B)
    for s in steps:
        st = o_step(st) if s == "O" else i_step(st)
    return st


def unscale(Cp: np.ndarray, st: Scaled) -> np.ndarray:
    """C = D_A C' D_B (last line of Algs. 1 and 3)."""
    return st.r[:, None] * Cp * st.s[None, :]


# ---------------------------------------------------------------------------
# Power-of-two mode
# ---------------------------------------------------------------------------

@dataclass
class Pow2:
    A: np.ndarray     # A' = 2^{-eA_i} A_ik 2^{d_k}
    B: np.ndarray     # B' = 2^{-d_k} B_kj 2^{-eB_j}
    eA: np.ndarray    # int64, cumulative row exponents (D_A = diag 2^eA)
    d: np.ndarray     # int64, cumulative inside exponents (D = diag 2^d)
    eB: np.ndarray    # int64, cumulative column exponents (D_B = diag 2^eB)


def pow2_start(A, B) -> Pow2:
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return Pow2(A.copy(), B.copy(), np.zeros(A.shape[0], np.int64),
                np.zeros(A.shape[1], np.int64), np.zeros(B.shape[1], np.int64))


def pow2_o_step(st: Pow2) -> Pow2:
    rmax = np.max(np.abs(st.A), axis=1) if st.A.shape[1] else np.zeros(st.A.shape[0])
    cmax = np.max(np.abs(st.B), axis=0) if st.B.shape[0] else np.zeros(st.B.shape[1])
    e = np.where(rmax > 0, _fexp(np.where(rmax > 0, rmax, 1.0)), 0)
    f = np.where(cmax > 0, _fexp(np.where(cmax > 0, cmax, 1.0)), 0)
    A = np.ldexp(st.A, -e[:, None])
    B = np.ldexp(st.B, -f[None, :])
    return Pow2(A, B, st.eA + e, st.d, st.eB + f)


def pow2_i_step(st: Pow2) -> Pow2:
    ca = np.max(np.abs(st.A), axis=0) if st.A.shape[0] else np.zeros(st.A.shape[1])
    rb = np.max(np.abs(st.B), axis=1) if st.B.shape[1] else np.zeros(st.B.shape[0])
    ok = (ca > 0) & (rb > 0)
    diff = _fexp(np.where(ok, rb, 1.0)) - _fexp(np.where(ok, ca, 1.0))
    dk = np.where(ok, np.floor_divide(diff, 2), 0)
    A = np.ldexp(st.A, dk[None, :])
    B = np.ldexp(st.B, -dk[:, None])
    return Pow2(A, B, st.eA, st.d + dk, st.eB)


def pow2_repeated(A, B, steps: str) -> Pow2:
    """Alg. 3 with power-of-two scales and a fixed step sequence."""
    st = pow2_start(A, B)
    for s in steps:
        st = pow2_o_step(st) if s == "O" else pow2_i_step(st)
    return st


def pow2_apply(A, B, eA, d, eB):
    """A' = 2^{-eA} A 2^{d}, B' = 2^{-d} B 2^{-eB} (exact)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return (np.ldexp(A, (-np.asarray(eA)[:, None] + np.asarray(d)[None, :])),
            np.ldexp(B, (-np.asarray(d)[:, None] - np.asarray(eB)[None, :])))


def pow2_unscale(Cp, eA, eB):
    """C = 2^{eA_i} C'_ij 2^{eB_j} (exact)."""
    return np.ldexp(np.asarray(Cp, np.float64), np.asarray(eA)[:, None] + np.asarray(eB)[None, :])


# ---------------------------------------------------------------------------
# Adaptive repeated scaling: Alg. 3 with the tau stopping criterion (Sec. 6.3)
# ---------------------------------------------------------------------------
#
# Steps alternate, starting with `first`.  t0 is the index (1-based) of the
# first O step; every step after it is tested on the factors it computes:
#   O step: every row factor of A' and column factor of B' >= (1+tau)^(-1/2)
#   I step: every inside factor in [(1+tau)^(-1/4), (1+tau)^(1/4)]
# and the iteration stops after the first step that passes (its result is
# kept: the theorem bounds the distance from the limit after that step), or
# after max_steps steps.  In power-of-two mode the factors tested are the
# powers of two the step applies (2^(new - old exponent)).

def _kinds(first: str, max_steps: int) -> str:
    other = "I" if first == "O" else "O"
    return "".join(first if t % 2 == 0 else other for t in range(max_steps))


def adaptive(A, B, tau: float, max_steps: int, first: str = "O"):
    """Real-valued adaptive Alg. 3; returns (state, steps taken)."""
    st = start(A, B)
    kinds = _kinds(first, max_steps)
    t0 = kinds.index("O") + 1 if "O" in kinds else max_steps + 1
    for t, kind in enumerate(kinds, start=1):
        st = o_step(st) if kind == "O" else i_step(st)
        if t <= t0:
            continue
        if kind == "O":
            rp, sp = st.history[-1][1]
            ok = np.all(rp >= (1 + tau) ** -0.5) and np.all(sp >= (1 + tau) ** -0.5)
        else:
            (D,) = st.history[-1][1]
            ok = np.all(D >= (1 + tau) ** -0.25) and np.all(D <= (1 + tau) ** 0.25)
        if ok:
            return st, t
    return st, len(kinds)


def pow2_adaptive(A, B, tau: float, max_steps: int, first: str = "O"):
    """Power-of-two adaptive Alg. 3; returns (state, steps taken)."""
    st = pow2_start(A, B)
    kinds = _kinds(first, max_steps)
    t0 = kinds.index("O") + 1 if "O" in kinds else max_steps + 1
    for t, kind in enumerate(kinds, start=1):
        prev = st
        st = pow2_o_step(st) if kind == "O" else pow2_i_step(st)
        if t <= t0:
            continue
        if kind == "O":
            f = np.exp2(np.concatenate([st.eA - prev.eA, st.eB - prev.eB]).astype(np.float64))
            ok = np.all(f >= (1 + tau) ** -0.5)
        else:
            f = np.exp2((st.d - prev.d).astype(np.float64))
            ok = np.all(f >= (1 + tau) ** -0.25) and np.all(f <= (1 + tau) ** 0.25)
        if ok:
            return st, t
    return st, len(kinds)
