"""PyTorch-facing wrappers over the C ABI (device memory and streams only;
every step of the computation runs in the library's CUDA kernels)."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence, Union

import numpy as np
import torch

from . import _native as N
from .rules import BaseRule, get as get_rule

LEAF = {"bf16": N.LEAF_BF16, "fp16": N.LEAF_F16, "bf16x3": N.LEAF_BF16X3, "e4m3b128": N.LEAF_E4M3B128}
SCHEDULE = {"auto": N.SCHEDULE_AUTO, "load_stage": N.SCHEDULE_LOAD_STAGE, "pass": N.SCHEDULE_PASS,
            "pass_epilogue": N.SCHEDULE_PASS_EPILOGUE, "pass_products": N.SCHEDULE_PASS_PRODUCTS,
            "pass_accumulate": N.SCHEDULE_PASS_ACCUMULATE}
DTYPE = {torch.float32: N.DT_F32, torch.bfloat16: N.DT_BF16, torch.float16: N.DT_F16}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _rowmajor(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.shape[0] > 0 and t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return max(t.stride(0), t.shape[1], 1)


def _check_exponents(vectors, lengths, device) -> None:
    """Exponent vectors are read as int32 arrays of a fixed length: anything
    else would have the kernels read past them or misread them."""
    for name, v in vectors.items():
        if v is None:
            continue
        n = lengths[name]
        if (not isinstance(v, torch.Tensor) or v.dtype != torch.int32 or v.dim() != 1 or v.numel() != n
                or not v.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous 1-D int32 tensor of length {n}")
        if v.device != device:
            raise ValueError(f"{name} must be on {device}, like the operands")


def _check_out(out: torch.Tensor, M: int, Ncols: int, device) -> None:
    """The kernels write M x Ncols float32 values through ``out``."""
    if out.dtype != torch.float32 or tuple(out.shape) != (M, Ncols):
        raise ValueError(f"out must be a float32 tensor of shape ({M}, {Ncols})")
    if out.device != device:
        raise ValueError(f"out must be on {device}, like the operands")


@dataclass
class TreeNode:
    """One node of a non-uniform plan: ``rule`` (a rule or its name) applied
    here; ``children[r]`` the node computing product r, None at the leaves."""
    rule: Union[str, BaseRule]
    children: list


class Plan:
    """A flattened uniform non-stationary plan (fmm_plan): ``rules[l]`` at
    level l+1, classical leaves, leaf products in ``leaf`` format.
    ``schedule`` (fmm_plan_set_schedule): "auto", "load_stage" (S_r, T_r
    formed in the multiply kernel's load stage) or "pass" (formed by a
    combination pass into the workspace; "pass_epilogue" / "pass_products"
    force where the output combination runs).  ``between``: scaling between
    recursive steps (fmm_plan_set_between_scaling)."""

    def __init__(self, rules: Sequence[Union[str, BaseRule]], leaf: str = "bf16x3", schedule: str = "auto",
                 between: bool = False, node_rule: Optional[Sequence[int]] = None, levels: int = 0):
        self.rules = [get_rule(r) if isinstance(r, str) else r for r in rules]
        self.leaf = leaf
        self._keep = []
        arr = self._rule_array(self.rules)
        h = C.c_void_p()
        if node_rule is None:
            N.check(N.lib().fmm_plan(C.byref(h), len(self.rules), arr, LEAF[leaf]), "fmm_plan")
        else:
            nodes = (C.c_int32 * max(1, len(node_rule)))(*node_rule)
            N.check(N.lib().fmm_plan_tree(C.byref(h), len(self.rules), arr, levels, len(node_rule), nodes,
                                          LEAF[leaf]), "fmm_plan_tree")
        self.node_rule = None if node_rule is None else list(node_rule)
        self._h = h
        self.schedule = schedule
        N.check(N.lib().fmm_plan_set_schedule(h, SCHEDULE[schedule]), "fmm_plan_set_schedule")
        self.between = between
        if between:
            N.check(N.lib().fmm_plan_set_between_scaling(h, 1), "fmm_plan_set_between_scaling")

    def _rule_array(self, rules):
        arr = (N.FmmRule * max(1, len(rules)))()
        for i, r in enumerate(rules):
            U = np.ascontiguousarray(r.U, np.float64)
            V = np.ascontiguousarray(r.V, np.float64)
            W = np.ascontiguousarray(r.W, np.float64)
            self._keep += [U, V, W]
            dp = C.POINTER(C.c_double)
            arr[i] = N.FmmRule(r.m0, r.k0, r.n0, r.r, U.ctypes.data_as(dp), V.ctypes.data_as(dp),
                               W.ctypes.data_as(dp), r.order_a, r.order_b, r.order_c)
        return arr

    @classmethod
    def tree(cls, root: "TreeNode", leaf: str = "bf16x3", schedule: str = "auto", between: bool = False):
        """A non-uniform plan (fmm_plan_tree) from a recursion tree whose
        nodes are ``TreeNode(rule, children)`` (children[r] computes product
        r one level down; None below the last level)."""
        table, index, node_rule = [], {}, []
        level, levels = [root], 0
        while level and level[0] is not None:
            levels += 1
            nxt = []
            for node in level:
                key = id(node.rule)
                if key not in index:
                    index[key] = len(table)
                    table.append(get_rule(node.rule) if isinstance(node.rule, str) else node.rule)
                node_rule.append(index[key])
                nxt.extend(node.children)
            if any(c is None for c in nxt) and not all(c is None for c in nxt):
                raise ValueError("every leaf of the tree must sit at the same depth")
            level = nxt
        return cls(table, leaf=leaf, schedule=schedule, between=between, node_rule=node_rule, levels=levels)

    @classmethod
    def variants(cls, base: Union[str, BaseRule], levels: int, selection: str = "round_robin", seed: int = 0,
                 A: Optional[torch.Tensor] = None, B: Optional[torch.Tensor] = None, leaf: str = "bf16x3",
                 schedule: str = "auto", stream=None) -> "Plan":
        """A non-uniform plan whose every node runs one of the eight
        Castrapel-Gustafson variants of a <2,2,2> rule (Sec. 3.4;
        fmm_plan_variants), chosen per node by ``selection``: "random"
        (SplitMix64 stream ``seed``), "round_robin", or "matrix" (from the
        block max-abs of the device operands A and B, found by
        fmm_block_max).  The chosen variant of each node (level order) is
        in ``plan.chosen``."""
        rule = get_rule(base) if isinstance(base, str) else base
        sel = {"random": N.SELECT_RANDOM, "round_robin": N.SELECT_ROUND_ROBIN, "matrix": N.SELECT_MATRIX}[selection]
        g = 1 << levels
        fa = fb = None
        if sel == N.SELECT_MATRIX:
            if A is None or B is None:
                raise ValueError("matrix-dependent selection needs the operands A and B")
            fa, fb = block_max(A, g, g, stream), block_max(B, g, g, stream)
            torch.cuda.synchronize(A.device)
            fa = fa.cpu().contiguous()
            fb = fb.cpu().contiguous()
        nodes = sum(rule.r**lvl for lvl in range(levels))
        chosen = (C.c_int32 * nodes)()
        self = cls.__new__(cls)
        self.rules = [rule]
        self.leaf = leaf
        self._keep = []
        arr = self._rule_array([rule])
        h = C.c_void_p()
        fp = C.POINTER(C.c_float)
        N.check(N.lib().fmm_plan_variants(C.byref(h), arr, levels, sel, C.c_uint64(seed & ((1 << 64) - 1)),
                                          None if fa is None else C.cast(fa.data_ptr(), fp),
                                          None if fb is None else C.cast(fb.data_ptr(), fp), chosen, LEAF[leaf]),
                "fmm_plan_variants")
        self._h = h
        self.node_rule = list(chosen)
        self.chosen = list(chosen)
        self.schedule = schedule
        N.check(N.lib().fmm_plan_set_schedule(h, SCHEDULE[schedule]), "fmm_plan_set_schedule")
        self.between = False
        return self

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        q, e = C.c_double(), C.c_double()
        leaves, nnz, pm, pk, pn = (C.c_int64() for _ in range(5))
        N.check(N.lib().fmm_plan_info(self._h, C.byref(q), C.byref(e), C.byref(leaves), C.byref(nnz),
                                      C.byref(pm), C.byref(pk), C.byref(pn)), "fmm_plan_info")
        return {"q_sum": q.value, "e_prod": e.value, "leaves": leaves.value, "nnz": nnz.value,
                "pm": pm.value, "pk": pk.value, "pn": pn.value}

    def flatten(self, table: str = "leaves"):
        """The flattened rule (Eq. 4.4) read back from one of the plan's
        kernel tables (fmm_plan_flatten): "leaves" (the tensor-core kernels'
        leaf descriptors), "lists" (the combination and output passes' term
        lists) or "gather" (the gather output pass's per-C-block lists: U and
        V come back as None).  Returns numpy arrays U (pm pk x leaves),
        V (pk pn x leaves), W (pm pn x leaves) and first (int32, W's shape:
        1 where the leaf is the first to add into the C block)."""
        t = {"leaves": N.TABLE_LEAVES, "lists": N.TABLE_LISTS, "gather": N.TABLE_GATHER}[table]
        inf = self.info()
        R = inf["leaves"]
        U = None if t == N.TABLE_GATHER else np.zeros((inf["pm"] * inf["pk"], R))
        V = None if t == N.TABLE_GATHER else np.zeros((inf["pk"] * inf["pn"], R))
        W = np.zeros((inf["pm"] * inf["pn"], R))
        first = np.zeros(W.shape, np.int32)
        ptr = lambda a: None if a is None else C.c_void_p(a.ctypes.data)  # noqa: E731
        N.check(N.lib().fmm_plan_flatten(self._h, t, ptr(U), ptr(V), ptr(W), ptr(first)), "fmm_plan_flatten")
        return U, V, W, first

    def gradient(self, which: str) -> "Plan":
        """The plan fmm_multiply_backward runs for "dA" (dC B^T, [[W, V^T, U]]
        per level or node) or "dB" (A^T dC, [[U^T, W, V]]), as a plan of its
        own (fmm_plan_gradient)."""
        w = {"dA": N.GRAD_A, "dB": N.GRAD_B}[which]
        h = C.c_void_p()
        N.check(N.lib().fmm_plan_gradient(self._h, w, C.byref(h)), "fmm_plan_gradient")
        g = Plan.__new__(Plan)
        g._keep, g.rules, g.leaf, g.node_rule = [], [], self.leaf, self.node_rule
        g.schedule, g.between, g._h = self.schedule, False, h
        return g

    def bound(self, K: int, normA: float, normB: float, eps: float) -> float:
        b = C.c_double()
        N.check(N.lib().fmm_plan_bound(self._h, K, normA, normB, eps, C.byref(b)), "fmm_plan_bound")
        return b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib().fmm_plan_destroy(h)
            except Exception:
                pass
            self._h = None


def block_max(X: torch.Tensor, nrb: int, ncb: int, stream=None) -> torch.Tensor:
    """Max-abs of each block of the nrb x ncb grid of ceil(rows/nrb) x
    ceil(cols/ncb) blocks of X (fmm_block_max): a float32 device tensor."""
    rows, cols = X.shape
    ld = _rowmajor(X, "X")
    out = torch.empty((nrb, ncb), dtype=torch.float32, device=X.device)
    N.check(N.lib().fmm_block_max(_ptr(X), DTYPE[X.dtype], rows, cols, ld, nrb, ncb, _ptr(out), _stream(stream)),
            "fmm_block_max")
    return out


def scale(A: torch.Tensor, B: torch.Tensor, steps: str, stream=None):
    """Alg. 3 with power-of-two scales and a fixed step sequence ("O", "I",
    "OI", "IO", "OIOI", ...); returns int32 device tensors (eA, d, eB)."""
    M, K = A.shape
    K2, Nn = B.shape
    assert K == K2 and A.dtype == B.dtype
    lda, ldb = _rowmajor(A, "A"), _rowmajor(B, "B")
    dev = A.device
    eA = torch.empty(M, dtype=torch.int32, device=dev)
    d = torch.empty(K, dtype=torch.int32, device=dev)
    eB = torch.empty(Nn, dtype=torch.int32, device=dev)
    N.check(N.lib().fmm_scale(steps.encode(), _ptr(A), _ptr(B), DTYPE[A.dtype], M, K, Nn, lda, ldb,
                              _ptr(eA), _ptr(d), _ptr(eB), _stream(stream)), "fmm_scale")
    return eA, d, eB


def scale_adaptive(A: torch.Tensor, B: torch.Tensor, tau: float, max_steps: int, first: str = "O", stream=None):
    """Adaptive Alg. 3 with the tau stopping test (fmm_scale_adaptive);
    returns int32 device tensors (eA, d, eB, steps) with steps[0] the number
    of steps applied (decided on the device, read it when needed)."""
    M, K = A.shape
    K2, Nn = B.shape
    assert K == K2 and A.dtype == B.dtype
    if first not in ("O", "I"):
        raise ValueError("first must be 'O' or 'I'")
    lda, ldb = _rowmajor(A, "A"), _rowmajor(B, "B")
    dev = A.device
    eA = torch.empty(M, dtype=torch.int32, device=dev)
    d = torch.empty(K, dtype=torch.int32, device=dev)
    eB = torch.empty(Nn, dtype=torch.int32, device=dev)
    steps = torch.empty(1, dtype=torch.int32, device=dev)
    ws = torch.empty(M + K + Nn + 64, dtype=torch.int32, device=dev)
    N.check(N.lib().fmm_scale_adaptive(_ptr(A), _ptr(B), DTYPE[A.dtype], M, K, Nn, lda, ldb, float(tau), max_steps,
                                       1 if first == "I" else 0, _ptr(eA), _ptr(d), _ptr(eB), _ptr(steps), _ptr(ws),
                                       ws.numel() * 4, _stream(stream)), "fmm_scale_adaptive")
    return eA, d, eB, steps


def scale_outside(A, B, d=None, eA=None, eB=None, stream=None):
    """One O step (Alg. 1 when d is None); returns (eA, eB)."""
    M, K = A.shape
    Nn = B.shape[1]
    _check_exponents({"d": d, "eA": eA, "eB": eB}, {"d": K, "eA": M, "eB": Nn}, A.device)
    eA = eA if eA is not None else torch.empty(M, dtype=torch.int32, device=A.device)
    eB = eB if eB is not None else torch.empty(Nn, dtype=torch.int32, device=A.device)
    N.check(N.lib().fmm_scale_outside(_ptr(A), _ptr(B), DTYPE[A.dtype], M, K, Nn, _rowmajor(A, "A"),
                                      _rowmajor(B, "B"), _ptr(d), _ptr(eA), _ptr(eB), _stream(stream)),
            "fmm_scale_outside")
    return eA, eB


def scale_inside(A, B, eA=None, eB=None, d=None, stream=None):
    """One I step (Alg. 2 when eA, eB are None); returns d."""
    M, K = A.shape
    Nn = B.shape[1]
    _check_exponents({"eA": eA, "eB": eB, "d": d}, {"eA": M, "eB": Nn, "d": K}, A.device)
    d = d if d is not None else torch.empty(K, dtype=torch.int32, device=A.device)
    N.check(N.lib().fmm_scale_inside(_ptr(A), _ptr(B), DTYPE[A.dtype], M, K, Nn, _rowmajor(A, "A"),
                                     _rowmajor(B, "B"), _ptr(eA), _ptr(eB), _ptr(d), _stream(stream)),
            "fmm_scale_inside")
    return d


def workspace_bytes(plan: Plan, M: int, K: int, Ncols: int) -> int:
    """Bytes of device workspace a scaled multiply of this shape needs."""
    b = C.c_size_t()
    N.check(N.lib().fmm_workspace_size(plan.handle, M, K, Ncols, C.byref(b)), "fmm_workspace_size")
    return b.value


_WS = {}


def _workspace(plan: Plan, M: int, K: int, Ncols: int, device) -> torch.Tensor:
    """A cached device workspace of at least workspace_bytes() bytes."""
    need = workspace_bytes(plan, M, K, Ncols)
    key = torch.device(device).index
    ws = _WS.get(key)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
        _WS[key] = ws
    return ws


def multiply(plan: Plan, A: torch.Tensor, B: torch.Tensor, eA=None, d=None, eB=None,
             out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """C = A B (float32) by the plan's fast algorithm on the scaled operands
    (C = D_A (A' B') D_B when exponents are given).  ``ws`` is a uint8 device
    tensor of workspace_bytes() used for operand copies (scaled, padded or
    realigned); a cached one is used when not given."""
    M, K = A.shape
    K2, Nn = B.shape
    if K != K2 or A.dtype != B.dtype or B.device != A.device:
        raise ValueError("shape / dtype / device mismatch")
    _check_exponents({"eA": eA, "d": d, "eB": eB}, {"eA": M, "d": K, "eB": Nn}, A.device)
    if out is None:
        out = torch.empty((M, Nn), dtype=torch.float32, device=A.device)
    _check_out(out, M, Nn, A.device)
    if ws is None:
        ws = _workspace(plan, M, K, Nn, A.device)
    N.check(N.lib().fmm_multiply(plan.handle, _ptr(A), _rowmajor(A, "A"), _ptr(B), _rowmajor(B, "B"),
                                 _ptr(out), _rowmajor(out, "C"), M, K, Nn, DTYPE[A.dtype], _ptr(eA), _ptr(d),
                                 _ptr(eB), _ptr(ws), ws.numel(), _stream(stream)), "fmm_multiply")
    return out


def multiply_backward(plan: Plan, dC: torch.Tensor, A: torch.Tensor, B: torch.Tensor, need_a: bool = True,
                      need_b: bool = True, ws: Optional[torch.Tensor] = None, stream=None):
    """(dA, dB) = (dC B^T, A^T dC) by the permuted fast rules."""
    M, K = A.shape
    Nn = B.shape[1]
    if B.shape[0] != K or tuple(dC.shape) != (M, Nn) or A.dtype != B.dtype:
        raise ValueError("dC must be M x N for A (M x K) and B (K x N) of one dtype")
    if B.device != A.device or dC.device != A.device:
        raise ValueError("dC, A and B must be on one device")
    dC = dC.contiguous().float()
    if ws is None:
        ws = _workspace(plan, M, K, Nn, A.device)
    dA = torch.empty((M, K), dtype=torch.float32, device=A.device) if need_a else None
    dB = torch.empty((K, Nn), dtype=torch.float32, device=A.device) if need_b else None
    N.check(N.lib().fmm_multiply_backward(plan.handle, _ptr(dC), _rowmajor(dC, "dC"), _ptr(A),
                                          _rowmajor(A, "A"), _ptr(B), _rowmajor(B, "B"), _ptr(dA),
                                          K if dA is not None else 0, _ptr(dB),
                                          Nn if dB is not None else 0, M, K, Nn, DTYPE[A.dtype], _ptr(ws),
                                          ws.numel(), _stream(stream)), "fmm_multiply_backward")
    return dA, dB


class HostPipeline:
    """Products of one shape whose operands and results live in host memory
    (fmm_host_*): ``submit`` enqueues the copies in, the scaling steps and
    the multiply, and the copy out, and returns at once; ``wait`` blocks
    until every submitted product is back.  Host tensors must stay untouched
    until then (or until ``depth`` further submissions); pinned tensors let
    the copies of one product overlap the computation of the next."""

    def __init__(self, plan: "Plan", M: int, K: int, Ncols: int, dtype=torch.float32, steps: str = "OI",
                 depth: int = 2):
        self.plan = plan
        self.shape = (M, K, Ncols)
        self.dtype = dtype
        h = C.c_void_p()
        N.check(N.lib().fmm_host_create(C.byref(h), plan.handle, M, K, Ncols, DTYPE[dtype], steps.encode(), depth),
                "fmm_host_create")
        self._h = h
        self._held = []
        self.depth = depth

    def submit(self, A: torch.Tensor, B: torch.Tensor, C_out: torch.Tensor) -> None:
        M, K, Ncols = self.shape
        for t, shp, dt, name in ((A, (M, K), self.dtype, "A"), (B, (K, Ncols), self.dtype, "B"),
                                 (C_out, (M, Ncols), torch.float32, "C")):
            if t.is_cuda or tuple(t.shape) != shp or t.dtype != dt or (t.shape[1] > 1 and t.stride(1) != 1):
                raise ValueError(f"{name}: host row-major {dt} tensor of shape {shp} required")
        N.check(N.lib().fmm_host_submit(self._h, C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(B.data_ptr()),
                                        B.stride(0), C.c_void_p(C_out.data_ptr()), C_out.stride(0)),
                "fmm_host_submit")
        self._held = (self._held + [(A, B, C_out)])[-(self.depth + 1):]

    def wait(self) -> None:
        N.check(N.lib().fmm_host_wait(self._h), "fmm_host_wait")
        self._held = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib().fmm_host_destroy(h)
            except Exception:
                pass
            self._h = None


def partition_batch(dims, parts: int) -> list:
    """Indices of the products of each part when a batch of products with
    sizes ``dims`` ((M, K, N) rows) is split over ``parts`` GPUs
    (fmm_batch_partition: longest-processing-time by flops)."""
    d = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
    n = len(d)
    M, K, Nn = (np.ascontiguousarray(d[:, j]) for j in range(3))
    out = np.zeros(n, dtype=np.int32)
    i64p = C.POINTER(C.c_int64)
    N.check(N.lib().fmm_batch_partition(M.ctypes.data_as(i64p), K.ctypes.data_as(i64p), Nn.ctypes.data_as(i64p), n,
                                        parts, out.ctypes.data_as(C.POINTER(C.c_int32))), "fmm_batch_partition")
    return [np.flatnonzero(out == q).tolist() for q in range(parts)]


class Batch:
    """Many independent products C_i = A_i B_i, each with its own plan, run
    as one fixed launch sequence (fmm_batch_create / fmm_batch_run): batched
    scaling reductions, one combination pass, one persistent tensor-core
    launch over every product's work units, one output pass.  ``problems``
    is a sequence of (plan, A, B, C) with row-major device tensors of one
    element type and float32 C; ``steps`` is "", "O", "I" or "OI".  The
    workspace is allocated here; ``run`` launches only (capturable in a CUDA
    graph) and recomputes every C from the current A and B."""

    def __init__(self, problems, steps: str = "OI", ws: Optional[torch.Tensor] = None):
        self._keep = list(problems)
        dt = problems[0][1].dtype
        arr = (N.FmmProblem * len(problems))()
        for i, (plan, A, B, Cm) in enumerate(problems):
            M, K = A.shape
            K2, Nn = B.shape
            if K != K2 or A.dtype != dt or B.dtype != dt or tuple(Cm.shape) != (M, Nn) or Cm.dtype != torch.float32:
                raise ValueError(f"problem {i}: shape / dtype mismatch")
            arr[i] = N.FmmProblem(plan.handle.value, A.data_ptr(), _rowmajor(A, "A"), B.data_ptr(),
                                  _rowmajor(B, "B"), Cm.data_ptr(), _rowmajor(Cm, "C"), M, K, Nn)
        self._arr = arr
        self.steps = steps
        need = C.c_size_t()
        N.check(N.lib().fmm_batch_workspace_size(arr, len(problems), DTYPE[dt], steps.encode(), C.byref(need)),
                "fmm_batch_workspace_size")
        self.ws = ws if ws is not None else torch.empty(max(need.value, 256), dtype=torch.uint8,
                                                        device=problems[0][1].device)
        h = C.c_void_p()
        N.check(N.lib().fmm_batch_create(C.byref(h), arr, len(problems), DTYPE[dt], steps.encode(), _ptr(self.ws),
                                         self.ws.numel()), "fmm_batch_create")
        self._h = h

    def run(self, stream=None) -> None:
        N.check(N.lib().fmm_batch_run(self._h, _stream(stream)), "fmm_batch_run")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib().fmm_batch_destroy(h)
            except Exception:
                pass
            self._h = None


# Candidate plans the autotuner chooses from: rules per level (depth = the
# list's length; the recursion cutoff is the smallest leaf block allowed).
AUTOTUNE_CANDIDATES = ((), ("strassen",), ("winograd",), ("winograd", "winograd"), ("strassen", "strassen"))


class Autotuner:
    """Chooses, per product shape, the rule sequence (algorithm and
    recursion depth) with the shortest measured time.  It times every
    candidate on a ladder of square sizes on the current GPU (once; results
    kept in ``self.table``), then, for a shape (M, K, N), predicts each
    candidate's time from the ladder point nearest to the shape's geometric
    mean size scaled by the candidate's flop count, and skips candidates
    whose leaf blocks would be smaller than ``cutoff``."""

    def __init__(self, leaf: str = "bf16", dtype=torch.bfloat16, sizes=(512, 1024, 2048, 4096),
                 candidates=AUTOTUNE_CANDIDATES, cutoff: int = 256, reps: int = 5, scaling: str = "OI"):
        self.leaf, self.dtype, self.sizes, self.cutoff = leaf, dtype, tuple(sizes), cutoff
        self.candidates = tuple(tuple(c) for c in candidates)
        self.table = {}
        self._plans = {c: Plan(list(c), leaf) for c in self.candidates}
        gen = torch.Generator(device="cuda").manual_seed(1507)
        for n in self.sizes:
            A = (torch.rand((n, n), generator=gen, device="cuda") * 2 - 1).to(dtype)
            B = (torch.rand((n, n), generator=gen, device="cuda") * 2 - 1).to(dtype)
            out = torch.empty((n, n), device="cuda")
            for c in self.candidates:
                if not self._fits(c, n, n, n):
                    continue
                plan = self._plans[c]
                eA, d, eB = scale(A, B, scaling) if scaling else (None, None, None)
                multiply(plan, A, B, eA, d, eB, out=out)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    multiply(plan, A, B, eA, d, eB, out=out)
                e1.record()
                torch.cuda.synchronize()
                self.table[(c, n)] = e0.elapsed_time(e1) / reps
            del A, B, out
        sync_status()

    def _fits(self, c, M, K, N) -> bool:
        p = self._plans[c].info()
        return min(M // p["pm"], K // p["pk"], N // p["pn"]) >= self.cutoff or not c

    def predict(self, c, M, K, N) -> float:
        """Predicted ms of candidate c on (M, K, N): the nearest ladder time
        scaled by the ratio of the products' classical flop counts."""
        g = (M * K * N) ** (1.0 / 3.0)
        pts = [n for n in self.sizes if (c, n) in self.table]
        if not pts:
            return float("inf")
        n = min(pts, key=lambda s: abs(np.log(s / g)))
        return self.table[(c, n)] * (M * K * N) / float(n ** 3)

    def choose(self, M, K, N, max_instability: Optional[float] = None):
        """Fastest predicted candidate; with ``max_instability``, only among
        candidates whose relative instability (the factor over the classical
        error bound, :func:`relative_instability`) is at most that value --
        the accuracy axis of the choice."""
        ok = [c for c in self.candidates if self._fits(c, M, K, N) and
              (max_instability is None or not c or relative_instability(self._plans[c]) <= max_instability)]
        best = min(ok, key=lambda c: self.predict(c, M, K, N))
        return list(best)

    def plan(self, M, K, N, max_instability: Optional[float] = None) -> "Plan":
        return self._plans[tuple(self.choose(M, K, N, max_instability))]


def relative_instability(plan: "Plan") -> float:
    """Factor by which the plan's first-order error bound exceeds the
    classical one for large K (Sec. 5.3): prod E / (prod k0)^2 for a uniform
    plan (max_k xi_k / (prod k0)^2 for a tree)."""
    info = plan.info()
    return info["e_prod"] / float(info["pk"]) ** 2


def algorithm_table(algorithms: dict, levels=(1, 2, 3, 4)) -> list:
    """Stability and cost figures of Sec. 5.3 for candidate algorithms.

    ``algorithms`` maps a name to a rule sequence; several rules are
    composed into one base-case rule (e.g. Strassen then a classical <2,1,1>
    step is a <4,2,2;14> rule).  Per algorithm: the base case <m0,k0,n0>,
    rank R, nnz, Q and E of that rule from the library's plan compiler; the
    stability exponent log_{m0 k0 n0} of E E' E'' with E', E'' those of its
    two cyclic rotations (for a square base case the three are equal, giving
    log_{n0} E); and per number of recursion steps L the fraction of
    classical flops (R / (m0 k0 n0))^L and the relative instability
    (E / k0^2)^L.  Host computation only (no GPU work)."""
    from .rules import compose, rotate
    rows = []
    for name, seq in algorithms.items():
        rules = [get_rule(r) if isinstance(r, str) else r for r in seq]
        rule = rules[0]
        for r in rules[1:]:
            rule = compose(rule, r)
        info = Plan([rule], "bf16").info()
        m0, k0, n0 = info["pm"], info["pk"], info["pn"]
        e_cyc = info["e_prod"]
        rot = rule
        for _ in range(2):
            rot = rotate(rot)
            e_cyc *= Plan([rot], "bf16").info()["e_prod"]
        R = info["leaves"]
        base = m0 * k0 * n0
        rows.append({"name": name, "m0": m0, "k0": k0, "n0": n0, "R": R, "nnz": info["nnz"], "Q": info["q_sum"],
                     "E": info["e_prod"], "stab_exp": float(np.log(e_cyc) / np.log(base)) if base > 1 else 0.0,
                     "flop_fraction": {L: (R / base) ** L for L in levels},
                     "relative_instability": {L: (info["e_prod"] / k0**2) ** L for L in levels}})
    return rows


TIMING_KINDS = {"scale": 2, "prepare": 4, "combine": 8, "multiply": 16}


def kernel_timing(enable: bool, kinds: Sequence[str] = ()) -> None:
    """Start (discarding earlier records) or stop per-kernel event timing;
    ``kinds`` restricts the recording to those kinds (default: all)."""
    mask = (sum(TIMING_KINDS[k] for k in kinds) if kinds else 1) if enable else 0
    N.check(N.lib().fmm_kernel_timing(mask), "fmm_kernel_timing")


def kernel_timing_read(kind: str = "") -> tuple:
    """(total ms, launches) of the recorded kernels of one kind ("scale",
    "prepare", "combine", "multiply") or of all kinds."""
    ms, n = C.c_double(), C.c_int64()
    N.check(N.lib().fmm_kernel_timing_read(kind.encode(), C.byref(ms), C.byref(n)), "fmm_kernel_timing_read")
    return ms.value, n.value


def sync_status(stream=None) -> None:
    """Synchronise and raise FmmError if a kernel recorded a device error."""
    N.check(N.lib().fmm_sync_status(_stream(stream)), "device status")


class FastMatmul(torch.autograd.Function):
    """C = A B with the plan's fast algorithm forward and the permuted fast
    rules backward (dA = dC B^T, dB = A^T dC)."""

    @staticmethod
    def forward(ctx, A, B, plan):
        ctx.save_for_backward(A, B)
        ctx.plan = plan
        return multiply(plan, A.contiguous(), B.contiguous())

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dA, dB = multiply_backward(ctx.plan, dC, A.contiguous(), B.contiguous(),
                                   ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        if dA is not None:
            dA = dA.to(A.dtype)
        if dB is not None:
            dB = dB.to(B.dtype)
        return dA, dB, None


def fast_matmul(A, B, plan):
    return FastMatmul.apply(A, B, plan)
