"""Castrapel-Gustafson variants of a <2,2,2> rule and per-node selection of
them in a recursion tree (Sec. 3.4).

Oracle module (test infrastructure only; see the package docstring).

The eight variants are [[(P^x (x) P^y) U, (P^z (x) P^x) V, (P^y (x) P^z) W]]
with x, y, z in {1, 2} and P the 2 x 2 exchange (P^2 = I), written in the
entry order the paper states (A, B column-major, C row-major).  Variant
v = 0..7 takes x = 1 when bit 1 of v is set, y = 1 when bit 0 is set,
z = 1 when bit 2 is set (else 2), so v = 0 is the rule itself.

The paper names random, round-robin and matrix-dependent selection without
defining them; the readings here:
  random        node n (level order) takes the top three bits of output n
                of SplitMix64 stream `seed` (Steele, Lea, Flood, OOPSLA 2014);
  round-robin   node n takes variant n mod 8;
  matrix        level by level, each node takes the variant minimising the
                one-level growth factor of the proof of Theorem 4.1 on its
                own operands, max_k sum_r |W_kr| (sum_i |U_ir| a_i)
                (sum_j |V_jr| b_j), with a_i, b_j bounds on the max-abs of
                its operands' quadrants (ties: the lowest v); its children's
                bounds follow from the triangle inequality.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .fmm import Node
from .rules import Rule, canonical, to_stated_order

_P = np.array([[0.0, 1.0], [1.0, 0.0]])
_I = np.eye(2)
MASK64 = (1 << 64) - 1


def exponents(v: int):
    """(x, y, z) of variant v."""
    return (1 if v & 2 else 2, 1 if v & 1 else 2, 1 if v & 4 else 2)


def variant(rule: Rule, v: int) -> Rule:
    """Variant v of a <2,2,2> rule: the Kronecker factors of Sec. 3.4 applied
    to the rule's tables in the stated entry order."""
    assert (rule.m0, rule.k0, rule.n0) == (2, 2, 2)
    x, y, z = exponents(v)
    pw = lambda e: _P if e == 1 else _I  # noqa: E731  (P^2 = I)
    s = to_stated_order(rule)
    U = np.kron(pw(x), pw(y)) @ s.U
    V = np.kron(pw(z), pw(x)) @ s.V
    W = np.kron(pw(y), pw(z)) @ s.W
    return Rule(f"{rule.name}_cg{v}", 2, 2, 2, U, V, W, "col", "col", "row", "Castrapel-Gustafson variant")


def splitmix64(seed: int, n: int) -> int:
    """Output n (0-based) of SplitMix64 started at state `seed`: the state
    advances by the golden gamma 0x9E3779B97F4A7C15 before each output,
    which is the state mixed by two xor-shift-multiply rounds and a final
    xor-shift."""
    z = (seed + (n + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def node_count(R: int, levels: int) -> int:
    return sum(R**lvl for lvl in range(levels))


def select_round_robin(R: int, levels: int) -> List[int]:
    return [n % 8 for n in range(node_count(R, levels))]


def select_random(R: int, levels: int, seed: int) -> List[int]:
    return [splitmix64(seed, n) >> 61 for n in range(node_count(R, levels))]


def block_max(X: np.ndarray, nrb: int, ncb: int) -> np.ndarray:
    """Max-abs of each block of the nrb x ncb grid of ceil(rows/nrb) x
    ceil(cols/ncb) blocks (zero for empty edge blocks)."""
    rows, cols = X.shape
    br, bc = -(-rows // nrb), -(-cols // ncb)
    out = np.zeros((nrb, ncb))
    for p in range(nrb):
        for q in range(ncb):
            blk = X[p * br:(p + 1) * br, q * bc:(q + 1) * bc]
            out[p, q] = float(np.abs(blk).max()) if blk.size else 0.0
    return out


def _quadrants(Bd: np.ndarray) -> List[float]:
    """Max over each quadrant (row-major 11, 12, 21, 22) of a bound grid."""
    h = Bd.shape[0] // 2
    return [float(Bd[p * h:(p + 1) * h, q * h:(q + 1) * h].max()) for p in (0, 1) for q in (0, 1)]


def node_cost(rule: Rule, Ab: np.ndarray, Bb: np.ndarray) -> float:
    """max_k sum_r |W_kr| (sum_i |U_ir| a_i)(sum_j |V_jr| b_j) on the
    quadrant bounds, every sum in ascending index order (canonical form:
    A, B, C row-major)."""
    c = canonical(rule)
    qa, qb = _quadrants(Ab), _quadrants(Bb)
    sa, sb = [], []
    for r in range(c.R):
        x = 0.0
        for i in range(4):
            x += abs(float(c.U[i, r])) * qa[i]
        y = 0.0
        for j in range(4):
            y += abs(float(c.V[j, r])) * qb[j]
        sa.append(x)
        sb.append(y)
    worst = 0.0
    for k in range(4):
        e = 0.0
        for r in range(c.R):
            e += abs(float(c.W[k, r])) * (sa[r] * sb[r])
        worst = max(worst, e)
    return worst


def child_bounds(T: np.ndarray, Bd: np.ndarray, r: int) -> np.ndarray:
    """Bounds on the finest blocks of sum_i T[i, r] X_i (X_i the quadrants
    of an operand whose finest-block bounds are Bd): sum_i |T_ir| Bd_i."""
    h = Bd.shape[0] // 2
    out = np.zeros((h, h))
    for s in range(h):
        for t in range(h):
            acc = 0.0
            for i in range(4):
                acc += abs(float(T[i, r])) * float(Bd[(i // 2) * h + s, (i % 2) * h + t])
            out[s, t] = acc
    return out


def select_matrix(rule: Rule, levels: int, Amax: np.ndarray, Bmax: np.ndarray, costs: Optional[list] = None):
    """Variant per node by the matrix-dependent reading (module docstring);
    Amax, Bmax: the 2^levels x 2^levels block max-abs grids of A and B.
    When ``costs`` is a list, each node's eight costs are appended to it."""
    variants = [variant(rule, v) for v in range(8)]
    canon = [canonical(v) for v in variants]
    level = [(np.asarray(Amax, np.float64), np.asarray(Bmax, np.float64))]
    chosen = []
    for lvl in range(levels):
        nxt = []
        for Ab, Bb in level:
            cs = [node_cost(variants[v], Ab, Bb) for v in range(8)]
            if costs is not None:
                costs.append(cs)
            best = min(range(8), key=lambda v: (cs[v], v))
            chosen.append(best)
            if lvl + 1 < levels:
                c = canon[best]
                for r in range(c.R):
                    nxt.append((child_bounds(c.U, Ab, r), child_bounds(c.V, Bb, r)))
        level = nxt
    return chosen


def tree(rule: Rule, levels: int, chosen: Sequence[int]) -> Node:
    """The recursion tree whose node n (level order) runs variant chosen[n]."""
    variants = [variant(rule, v) for v in range(8)]
    R = rule.R
    it = iter(chosen)
    # level by level, children attached in product order
    roots = [Node(variants[next(it)], [None] * R)]
    level = roots
    for _ in range(1, levels):
        nxt = []
        for node in level:
            for r in range(R):
                child = Node(variants[next(it)], [None] * R)
                node.children[r] = child
                nxt.append(child)
        level = nxt
    return roots[0]
