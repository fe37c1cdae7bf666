"""Classical and recursive fast matrix multiplication, and the error bounds.

Oracle module (test infrastructure only; see the package docstring).

A *plan* is a recursion tree.  ``Node(rule, children)`` applies ``rule`` at
this node; ``children[r]`` is the node that computes product M_r one level
down (``None`` = classical product at the base case).  Stationary and uniform
non-stationary plans (Sec. 3.2, 3.3) are trees with one rule per level
(:func:`uniform`); non-uniform plans (Sec. 3.4) give every node its own rule.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional, Sequence

import numpy as np

from . import precision
from .rules import Rule, canonical, principal


@dataclass
class Node:
    rule: Rule
    children: list  # length R, entries Node or None


def uniform(rules: Sequence[Rule]) -> Optional[Node]:
    """Tree of a uniform non-stationary plan: ``rules[l]`` at every node of
    level l+1 (Sec. 3.3).  Stationary = the same rule repeated (Sec. 3.2)."""
    if not rules:
        return None
    child = uniform(rules[1:])
    return Node(rules[0], [child] * rules[0].R)


def dims(node: Optional[Node]):
    """(prod m0, prod k0, prod n0) along one root-to-leaf path (all paths of a
    plan partition alike, Sec. 3.4)."""
    if node is None:
        return 1, 1, 1
    m, k, n = dims(node.children[0])
    return node.rule.m0 * m, node.rule.k0 * k, node.rule.n0 * n


def depth(node: Optional[Node]) -> int:
    return 0 if node is None else 1 + depth(node.children[0])


# ---------------------------------------------------------------------------
# Products
# ---------------------------------------------------------------------------

def classical(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = AB by the classical algorithm in float64 (the base case of
    Eq. 3.2); the inner products are evaluated by the BLAS matmul."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def classical_exact(A, B):
    """C = AB with Python integers / Fractions, for brute force on tiny
    inputs."""
    M, K = len(A), len(A[0])
    N = len(B[0])
    return [[sum(A[i][k] * B[k][j] for k in range(K)) for j in range(N)] for i in range(M)]


def classical_exact_fixed(A: np.ndarray, B: np.ndarray, frac_bits: int = 48):
    """Exact C = AB for inputs that are multiples of 2^-frac_bits with
    |entries| < 2 (fixed point), returned as an object array of Python
    integers holding C * 2^(2 frac_bits).  Each input is split into four
    16-bit integer limbs; the limb products are exact in int64 (K up to
    2^20), and Python integers add them with their shifts."""
    sa = np.round(np.asarray(A, np.float64) * 2.0**frac_bits)
    sb = np.round(np.asarray(B, np.float64) * 2.0**frac_bits)
    assert np.array_equal(sa / 2.0**frac_bits, A) and np.array_equal(sb / 2.0**frac_bits, B)
    ia, ib = sa.astype(np.int64), sb.astype(np.int64)

    def limbs(X):
        sgn = np.sign(X)
        X = np.abs(X)
        return [sgn * ((X >> (16 * t)) & 0xFFFF) for t in range(4)]

    la, lb = limbs(ia), limbs(ib)
    out = np.zeros((A.shape[0], B.shape[1]), dtype=object)
    for s, a in enumerate(la):
        for t, b in enumerate(lb):
            if not a.any() or not b.any():
                continue
            p = (a @ b).astype(object)
            out = out + p * (1 << (16 * (s + t)))
    return out


def exact_to_float(Cint, frac_bits: int = 48) -> np.ndarray:
    """Round the exact fixed-point result of classical_exact_fixed to float64."""
    from fractions import Fraction
    den = 1 << (2 * frac_bits)
    return np.vectorize(lambda v: float(Fraction(int(v), den)))(Cint).astype(np.float64)


def _seq_sum(terms, dtype):
    """Sequential sum c_1 X_1 + c_2 X_2 + ... in the order given, each step
    rounded to ``dtype`` (the summation model of Eq. 4.3)."""
    acc = None
    for c, X in terms:
        t = (dtype(c) * X).astype(dtype)
        acc = t if acc is None else (acc + t).astype(dtype)
    return acc


def _pad(X: np.ndarray, rows: int, cols: int) -> np.ndarray:
    if X.shape == (rows, cols):
        return X
    out = np.zeros((rows, cols), dtype=X.dtype)
    out[: X.shape[0], : X.shape[1]] = X
    return out


def _recurse(A, B, node, leaf, dtype, dvecs=None):
    """One node of Eq. 3.2.  ``dvecs`` (root node only): per product r an
    integer vector d, applied as S_r <- S_r 2^d (columns), T_r <- 2^-d T_r
    (rows) before recursing -- the between-steps scaling."""
    if node is None:
        return leaf(A, B)
    r = canonical(node.rule)
    m0, k0, n0 = r.m0, r.k0, r.n0
    mb, kb, nb = A.shape[0] // m0, A.shape[1] // k0, B.shape[1] // n0
    Ab = [A[p * mb:(p + 1) * mb, q * kb:(q + 1) * kb] for p in range(m0) for q in range(k0)]
    Bb = [B[p * kb:(p + 1) * kb, q * nb:(q + 1) * nb] for p in range(k0) for q in range(n0)]
    Ms = []
    for j in range(r.R):
        # S_r, T_r: sequential sums in index order (Eq. 3.2)
        S = _seq_sum([(r.U[i, j], Ab[i]) for i in range(m0 * k0) if r.U[i, j] != 0], dtype)
        T = _seq_sum([(r.V[i, j], Bb[i]) for i in range(k0 * n0) if r.V[i, j] != 0], dtype)
        if S is None:
            S = np.zeros((mb, kb), dtype)
        if T is None:
            T = np.zeros((kb, nb), dtype)
        if dvecs is not None:
            S = (S * np.exp2(dvecs[j].astype(np.float64))[None, :]).astype(dtype)
            T = (T * np.exp2(-dvecs[j].astype(np.float64))[:, None]).astype(dtype)
        Ms.append(_recurse(S, T, node.children[j], leaf, dtype))
    C = np.zeros((m0 * mb, n0 * nb), dtype=dtype)
    for k in range(m0 * n0):
        p, q = divmod(k, n0)
        # C_k = sum_r W[k, r] M_r, r in order (Eq. 3.2)
        blk = _seq_sum([(r.W[k, j], Ms[j]) for j in range(r.R) if r.W[k, j] != 0], dtype)
        if blk is not None:
            C[p * mb:(p + 1) * mb, q * nb:(q + 1) * nb] = blk
    return C


def _frexp_exp(x: np.ndarray) -> np.ndarray:
    """frexp exponent e (x = f 2^e, 1/2 <= |f| < 1) of each entry; None-like
    sentinel -2^30 for zeros."""
    f, e = np.frexp(x)
    return np.where(x == 0, -(1 << 30), e).astype(np.int64)


def between_exponents(A: np.ndarray, B: np.ndarray, node: Node) -> list:
    """Scaling between recursive steps (the reading used here: after the
    root node's sums, before the next level's).  For each root product r,
    the pair (S_r, T_r) is inside-scaled as its own product A B (Alg. 2 in
    power-of-two form): d_k = floor((e(max_j |T_r[k, j]|) - e(max_i
    |S_r[i, k]|)) / 2), 0 where either side is zero.  S_r, T_r are the
    root node's sequential sums in index order in FP32 (the precision the
    operand sums are formed in); A, B already padded."""
    r = canonical(node.rule)
    m0, k0, n0 = r.m0, r.k0, r.n0
    A32, B32 = np.asarray(A, np.float32), np.asarray(B, np.float32)
    mb, kb, nb = A32.shape[0] // m0, A32.shape[1] // k0, B32.shape[1] // n0
    Ab = [A32[p * mb:(p + 1) * mb, q * kb:(q + 1) * kb] for p in range(m0) for q in range(k0)]
    Bb = [B32[p * kb:(p + 1) * kb, q * nb:(q + 1) * nb] for p in range(k0) for q in range(n0)]
    out = []
    for j in range(r.R):
        S = _seq_sum([(r.U[i, j], Ab[i]) for i in range(m0 * k0) if r.U[i, j] != 0], np.float32)
        T = _seq_sum([(r.V[i, j], Bb[i]) for i in range(k0 * n0) if r.V[i, j] != 0], np.float32)
        if S is None or T is None or S.shape[0] == 0 or T.shape[1] == 0:
            out.append(np.zeros(kb, np.int64))
            continue
        eS = _frexp_exp(np.abs(S).max(axis=0).astype(np.float64))
        eT = _frexp_exp(np.abs(T).max(axis=1).astype(np.float64))
        zero = (eS <= -(1 << 29)) | (eT <= -(1 << 29))
        out.append(np.where(zero, 0, np.floor_divide(eT - eS, 2)).astype(np.int64))
    return out


def fmm(A: np.ndarray, B: np.ndarray, plan: Optional[Node],
        leaf: Optional[Callable] = None, dtype=np.float64, between: bool = False) -> np.ndarray:
    """C = AB by the recursive fast algorithm of Eq. 3.2 with the given plan.

    A and B are zero-padded once, up front, so that every level partitions
    evenly (Sec. 3.2 pads with zeros; reading: pad M, K, N to the next
    multiple of the product of the base-case dimensions along the tree).
    S_r, T_r and C_k are sequential sums in index order computed in
    ``dtype``; the leaves call ``leaf(S, T)`` (default: classical float64).
    """
    leaf = leaf or classical
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    pm, pk, pn = dims(plan)
    Mp, Kp, Np = -(-M // pm) * pm, -(-K // pk) * pk, -(-N // pn) * pn
    Ap = _pad(np.asarray(A, dtype=dtype), Mp, Kp)
    Bp = _pad(np.asarray(B, dtype=dtype), Kp, Np)
    if M == 0 or N == 0:
        return np.zeros((M, N), dtype=dtype)
    dvecs = between_exponents(Ap, Bp, plan) if between and depth(plan) >= 2 else None
    return _recurse(Ap, Bp, plan, leaf, dtype, dvecs)[:M, :N]


def abs_plan(node: Optional[Node]) -> Optional[Node]:
    """Same tree with |U|, |V|, |W|."""
    if node is None:
        return None
    r = node.rule
    ar = Rule(r.name + "|abs|", r.m0, r.k0, r.n0, np.abs(r.U), np.abs(r.V), np.abs(r.W),
              r.order_a, r.order_b, r.order_c)
    return Node(ar, [abs_plan(c) for c in node.children])


def growth(A: np.ndarray, B: np.ndarray, plan: Optional[Node], between: bool = False) -> np.ndarray:
    """Componentwise growth quantity of the proof of Theorem 4.1:
        G_ij = sum_r |W-product| (sum_i |U-product| |A_i|) (sum_j |V-product| |B_j|)
    evaluated entrywise (before the max-norms are taken).  The proof bounds
    |C_k - fl(C_k)| by delta_k * eps * G to first order, and G <= (K/K0^L)
    E^L ||A|| ||B||.  Computed as the fast algorithm run on |A|, |B| with
    |U|, |V|, |W| in float64.  With ``between``, the root products' scaling
    exponents (from the signed operands) scale the absolute sums the same
    way."""
    if not (between and depth(plan) >= 2):
        return fmm(np.abs(A), np.abs(B), abs_plan(plan))
    M, K = A.shape
    N = B.shape[1]
    pm, pk, pn = dims(plan)
    Mp, Kp, Np = -(-M // pm) * pm, -(-K // pk) * pk, -(-N // pn) * pn
    Ap = _pad(np.asarray(A, dtype=np.float64), Mp, Kp)
    Bp = _pad(np.asarray(B, dtype=np.float64), Kp, Np)
    if M == 0 or N == 0:
        return np.zeros((M, N))
    dvecs = between_exponents(Ap, Bp, plan)
    return _recurse(np.abs(Ap), np.abs(Bp), abs_plan(plan), classical, np.float64, dvecs)[:M, :N]


def growth_entries(A: np.ndarray, B: np.ndarray, rules: Sequence[Rule], rows, cols) -> np.ndarray:
    """``growth`` of the uniform plan ``rules`` at the entries (rows[s],
    cols[s]) only, from the flattened rule of Eq. 4.4 (the levels composed
    into one <pm, pk, pn; R^L> rule): with A, B zero-padded to the block
    grid, entry (i, j) of C block (bi, bj) at position (li, lj) is
        G_ij = sum_r |W_(bi,bj),r| (sum_(p,q) |U_(p,q),r| |A_(p bm + li, q block)|)
                                   . (sum_(p,q) |V_(p,q),r| |B_(p block, q bn + lj)|)
    -- the same sums as the recursive evaluation, since every term is
    nonnegative.  Each sample costs O(R^L K / pk) instead of a full product,
    so it serves products too large for ``growth``."""
    from .rules import compose
    comp = canonical(rules[0])
    for r in rules[1:]:
        comp = compose(comp, r)
    pm, pk, pn = comp.m0, comp.k0, comp.n0
    M, K = A.shape
    N = B.shape[1]
    bm, bk, bn = -(-M // pm), -(-K // pk), -(-N // pn)
    Ua, Va, Wa = np.abs(comp.U), np.abs(comp.V), np.abs(comp.W)
    out = np.zeros(len(rows))
    for s, (i, j) in enumerate(zip(rows, cols)):
        bi, li = divmod(int(i), bm)
        bj, lj = divmod(int(j), bn)
        # |A| row segments of every block: (pm pk) x bk, zero past the edge
        Aseg = np.zeros((pm, pk * bk))
        for p in range(pm):
            r_ = p * bm + li
            if r_ < M:
                Aseg[p, :K] = np.abs(A[r_, :])
        Aseg = Aseg.reshape(pm * pk, bk)
        Bseg = np.zeros((pn, pk * bk))
        for q in range(pn):
            c_ = q * bn + lj
            if c_ < N:
                Bseg[q, :K] = np.abs(B[:, c_])
        # B block (p, q) at flattened index p pn + q holds column lj of block column q
        Bseg = Bseg.reshape(pn, pk, bk).transpose(1, 0, 2).reshape(pk * pn, bk)
        S = Ua.T @ Aseg          # R x bk
        T = Va.T @ Bseg          # R x bk
        Mr = np.einsum("rk,rk->r", S, T)
        out[s] = Wa[bi * pn + bj] @ Mr
    return out


# ---------------------------------------------------------------------------
# Leaf products in reduced precision (emulation of the leaf formats)
# ---------------------------------------------------------------------------

def leaf_rounded(fmt: str) -> Callable:
    """Leaf product with S and T rounded to ``fmt`` ('bf16', 'fp16') and the
    product formed exactly (float64)."""
    def leaf(S, T):
        return classical(precision.round_to(S, fmt), precision.round_to(T, fmt))
    return leaf


def quantize_e4m3_blocks(X: np.ndarray, axis: int, block: int = 128):
    """E4M3 with power-of-two block scales along ``axis`` (blocks of
    ``block`` consecutive entries of each row (axis 1) or column (axis 0)):
    each block is scaled by 2^-s with s = e(max |block|) - 8 (the frexp
    exponent; s = 0 for an all-zero block), so that its largest magnitude
    lies in [128, 256), rounded to E4M3 (ties to even), and scaled back.
    The scale is a UE8M0 number (2^-127 .. 2^127), so s is raised to -127
    for blocks whose largest magnitude is below 2^-120 (which then use the
    E4M3 subnormals).
    Returns (the represented values, the exponents s per block)."""
    X = np.asarray(X, dtype=np.float64)
    Xt = X if axis == 1 else X.T
    rows, cols = Xt.shape
    nb = -(-cols // block)
    out = np.zeros_like(Xt)
    scales = np.zeros((rows, nb), dtype=np.int64)
    for b in range(nb):
        blk = Xt[:, b * block:(b + 1) * block]
        m = np.abs(blk).max(axis=1)
        e = np.frexp(m)[1]
        s_ = np.where(m > 0, np.maximum(e - 8, -127), 0)
        scales[:, b] = s_
        f = np.exp2(s_.astype(np.float64))[:, None]
        out[:, b * block:(b + 1) * block] = precision.round_to(blk / f, "e4m3") * f
    return (out if axis == 1 else out.T), (scales if axis == 1 else scales.T)


def leaf_e4m3_b128(S, T):
    """Leaf product with S quantized to E4M3 in 128-blocks along K per row
    and T per column (quantize_e4m3_blocks), the product formed exactly."""
    return classical(quantize_e4m3_blocks(S, axis=1)[0], quantize_e4m3_blocks(T, axis=0)[0])


def leaf_bf16x3(S, T):
    """Leaf product with S = hi + lo, T = hi' + lo' split into bf16 parts and
    the three products hi hi' + hi lo' + lo hi' formed exactly (float64)."""
    sh, sl = precision.split_bf16(S)
    th, tl = precision.split_bf16(T)
    return classical(sh, th) + classical(sh, tl) + classical(sl, th)


# ---------------------------------------------------------------------------
# Bounds (Theorems 4.1, 4.2; Sec. 4.5)
# ---------------------------------------------------------------------------

def bound_uniform(rules: Sequence[Rule], K: int, normA: float, normB: float,
                  eps: float) -> float:
    """Theorem 4.2 (Theorem 4.1 when all rules are equal), first order:
        (K/prod K0 + sum_l Q_l) (K/prod K0) (prod_l E_l) ||A|| ||B|| eps
    with ||.|| the max-norm.  K is the (padded) inner dimension."""
    pk = int(np.prod([r.k0 for r in rules])) if rules else 1
    kl = K / pk
    Qs = sum(principal(r).Q for r in rules)
    Es = float(np.prod([principal(r).E for r in rules])) if rules else 1.0
    return (kl + Qs) * kl * Es * normA * normB * eps


def delta_vector(node: Optional[Node], chi: float = 0.0) -> np.ndarray:
    """Accumulation counts delta_k of Sec. 4.5 without the K/prod K0 term,
    over the flattened output blocks k = (k_1, ..., k_L) (k_1 slowest):
    delta^{[l]}_k = gamma_{k_l} + max_{r: W[k_l, r] != 0} delta^{[l+1, r]}_k
    with chi (the alpha + beta counts along the path) at the leaves."""
    if node is None:
        return np.array([chi])
    r = canonical(node.rule)
    p = principal(r)
    subs = [delta_vector(node.children[j], chi + p.alpha[j] + p.beta[j]) for j in range(r.R)]
    out = []
    for k in range(r.m0 * r.n0):
        cands = [subs[j] for j in range(r.R) if r.W[k, j] != 0]
        out.append(p.gamma[k] + np.max(np.stack(cands), axis=0))
    return np.concatenate(out)


def xi_vector(node: Optional[Node]) -> np.ndarray:
    """Growth factors xi_k of Sec. 4.5 (simplified form), flattened over
    k = (k_1, ..., k_L): xi = sum_r |W[k_1, r]| a_r b_r xi^{child r}."""
    if node is None:
        return np.array([1.0])
    r = canonical(node.rule)
    p = principal(r)
    subs = [xi_vector(node.children[j]) for j in range(r.R)]
    out = []
    for k in range(r.m0 * r.n0):
        acc = np.zeros_like(subs[0])
        for j in range(r.R):
            if r.W[k, j] != 0:
                acc = acc + abs(r.W[k, j]) * p.a[j] * p.b[j] * subs[j]
        out.append(acc)
    return np.concatenate(out)


def bound_tree(plan: Optional[Node], K: int, normA: float, normB: float, eps: float) -> float:
    """Sec. 4.5 bound for any plan: (K/prod K0 + max_k delta_k)(K/prod K0)
    max_k xi_k ||A|| ||B|| eps (first order)."""
    _, pk, _ = dims(plan)
    kl = K / pk
    return (kl + float(delta_vector(plan).max())) * kl * float(xi_vector(plan).max()) \
        * normA * normB * eps


def flop_count(plan: Optional[Node], M: int, K: int, N: int) -> dict:
    """Leaf flops 2 * R^L * (M/pm)(K/pk)(N/pn) of the padded problem and the
    classical 2MKN."""
    pm, pk, pn = dims(plan)
    leaves = 1
    node = plan
    while node is not None:
        leaves *= node.rule.R
        node = node.children[0]
    Mp, Kp, Np = -(-M // pm) * pm, -(-K // pk) * pk, -(-N // pn) * pn
    return {"leaf": 2.0 * leaves * (Mp // pm) * (Kp // pk) * (Np // pn),
            "classical": 2.0 * M * K * N, "leaves": leaves}


# ---------------------------------------------------------------------------
# Errors (Sec. 6.5)
# ---------------------------------------------------------------------------

def err_max(C_hat: np.ndarray, C: np.ndarray) -> float:
    return float(np.max(np.abs(np.asarray(C_hat, np.float64) - C))) if C.size else 0.0


def err_componentwise(C_hat: np.ndarray, C: np.ndarray) -> float:
    """max_ij |c_hat - c| / |c| over entries with c != 0 (Sec. 6.5)."""
    C_hat = np.asarray(C_hat, np.float64)
    nz = C != 0
    if not nz.any():
        return 0.0
    return float(np.max(np.abs(C_hat[nz] - C[nz]) / np.abs(C[nz])))
