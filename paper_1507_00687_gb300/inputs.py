"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random-number generation only -- none of the method's
arithmetic -- so that the CUDA path's tests and benchmarks and the CPU
oracle's checks draw the same inputs.  All generators are numpy PCG64 streams
keyed by an integer seed; every function returns float64 arrays (callers cast
to the storage dtype they test).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform(shape, lo: float, hi: float, seed: int) -> np.ndarray:
    """iid Uniform[lo, hi)."""
    return rng(seed).uniform(lo, hi, size=shape)


def integers(shape, lo: int, hi: int, seed: int) -> np.ndarray:
    """iid integers uniform in {lo, ..., hi} (as float64)."""
    return rng(seed).integers(lo, hi + 1, size=shape).astype(np.float64)


def diag_scaled_pair(M: int, K: int, N: int, seed: int, span: float = 12.0,
                     integer_exponents: bool = False):
    """A = D1 X D2 and B = D3 Y D4 with X, Y iid Uniform[0, 1) and the
    diagonal entries of D1..D4 equal to 2^u, u ~ Uniform(-span, span)
    (continuous by default, so the diagonal is not itself a power of two)."""
    g = rng(seed)
    X = g.uniform(0.0, 1.0, size=(M, K))
    Y = g.uniform(0.0, 1.0, size=(K, N))

    def d(n):
        u = g.uniform(-span, span, size=n)
        if integer_exponents:
            u = np.floor(u)
        return np.exp2(u)

    d1, d2, d3, d4 = d(M), d(K), d(K), d(N)
    return d1[:, None] * X * d2[None, :], d3[:, None] * Y * d4[None, :]


def paper_distribution(kind: int, n: int, seed: int):
    """The three N x N test distributions of the scaling experiments
    (Sec. 6.5), with 1-based index conditions i < n/2, j > n/2 read on
    0-based arrays as i + 1 < n/2, j + 1 > n/2.
      1: A, B iid Uniform(0, 1)
      2: A_ij ~ U(0, 1/n^2) if j > n/2 else U(0, 1);
         B_ij ~ U(0, 1/n^2) if i < n/2 else U(0, 1)
      3: A_ij ~ U(0, n^2) if i < n/2 and j > n/2 else U(0, 1);
         B_ij ~ U(0, 1/n^2) if j < n/2 else U(0, 1)
    """
    g = rng(seed)
    A = g.uniform(0.0, 1.0, size=(n, n))
    B = g.uniform(0.0, 1.0, size=(n, n))
    idx = np.arange(n) + 1
    half = n / 2.0
    if kind == 2:
        A[:, idx > half] *= 1.0 / n**2
        B[idx < half, :] *= 1.0 / n**2
    elif kind == 3:
        A[np.ix_(idx < half, idx > half)] *= float(n) ** 2
        B[:, idx < half] *= 1.0 / n**2
    elif kind != 1:
        raise ValueError(kind)
    return A, B


def log_uniform_dims(count: int, lo: int, hi: int, step: int, seed: int) -> np.ndarray:
    """``count`` x 3 problem dimensions, each exp(Uniform(ln lo, ln hi))
    rounded to a multiple of ``step`` and clipped to [lo, hi]."""
    g = rng(seed)
    x = np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    x = np.clip(np.round(x / step) * step, lo, hi)
    return x.astype(np.int64)
