"""Shared helpers of the GPU parity tests: building the library, running the
oracle on the same inputs, and the elementwise tolerance.

Tolerance (first-order, per output entry), derived from the arithmetic of
the CUDA path on top of the exact float64 result of the oracle:
  |C_gpu - C| <= (u_leaf + (K_leaf + 2 t_max + 8) 2^-23) * G
with G the growth quantity of the proof of Theorem 4.1 evaluated entrywise
(sum_r |W| |S_r| |T_r| with absolute coefficients, unscaled by 2^(eA+eB)),
u_leaf the relative error of one leaf product from rounding S and T
(bf16: 2^-7 + 2^-16, fp16: 2^-10 + 2^-22, bf16 hi+lo with three products:
3 * 2^-16, E4M3 with 128-block scales: 2^-3 + 2^-8), K_leaf FP32 accumulations in the tensor core, and at most
t_max FP32 roundings each for forming S, forming T and adding into C
(counted with the conservative 2^-23 per operation).
"""
import numpy as np
import pytest
import torch

from oracle import fmm as OF
from oracle import rules as OR
from oracle import scaling as OS

U_LEAF = {"bf16": 2.0**-7 + 2.0**-16, "fp16": 2.0**-10 + 2.0**-22, "bf16x3": 3 * 2.0**-16,
          "e4m3b128": 2.0**-3 + 2.0**-8}

ORACLE_RULES = {"strassen": OR.strassen, "winograd": OR.winograd, "fast323": OR.fast323,
                "classical121": lambda: OR.classical(1, 2, 1), "classical211": lambda: OR.classical(2, 1, 1),
                "classical222": lambda: OR.classical(2, 2, 2)}

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_00687_gb300 import build
    build.build()
    from paper_1507_00687_gb300 import api
    return api


def oracle_tree(names):
    return OF.uniform([ORACLE_RULES[n]() for n in names])


def to_dev(X64: np.ndarray, dt: str) -> torch.Tensor:
    return torch.from_numpy(X64).to(TORCH_DT[dt]).cuda()


def dev_values(T: torch.Tensor) -> np.ndarray:
    """The exact float64 values of a device tensor."""
    return T.detach().to(torch.float64).cpu().numpy()


def max_terms(names) -> int:
    t = 1
    for n in names:
        r = ORACLE_RULES[n]()
        p = OR.principal(r)
        t *= int(max(p.alpha.max(), p.beta.max(), (r.W != 0).sum(axis=0).max()))
    return t


def oracle_reference(A64, B64, names, eA=None, d=None, eB=None):
    """(C, G): the exact-arithmetic fast product (float64) of the scaled
    operands, unscaled, and its growth quantity."""
    tree = oracle_tree(names)
    if eA is not None:
        Ap, Bp = OS.pow2_apply(A64, B64, eA, d, eB)
        C = OS.pow2_unscale(OF.fmm(Ap, Bp, tree), eA, eB)
        G = OS.pow2_unscale(OF.growth(Ap, Bp, tree), eA, eB)
    else:
        C = OF.fmm(A64, B64, tree)
        G = OF.growth(A64, B64, tree)
    return C, G


def tolerance(G, names, K, leaf):
    tree = oracle_tree(names)
    _, pk, _ = OF.dims(tree)
    kl = -(-K // pk)
    return (U_LEAF[leaf] + (kl + 2 * max_terms(names) + 8) * 2.0**-23) * G


def assert_within(C_gpu, C, G, names, K, leaf, what=""):
    tol = tolerance(G, names, K, leaf)
    err = np.abs(C_gpu - C)
    bad = err > tol
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} entries outside tolerance; first {tuple(i)}: "
                             f"gpu={C_gpu[tuple(i)]!r} oracle={C[tuple(i)]!r} tol={tol[tuple(i)]!r}")
    return float((err / np.where(tol > 0, tol, 1)).max())
