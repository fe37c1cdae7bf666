"""Host-detectable argument errors of the C ABI return at once, with the
status code the header gives, and launch nothing.

Run where no CUDA device exists: there every call that reached the CUDA
runtime would fail with FMM_ERR_CUDA, so a status of FMM_ERR_ARG, _SHAPE,
_DTYPE, _WORKSPACE or _UNSUPPORTED shows that the call stopped on the host
first.  Some cases pass stand-in addresses for operands that the call must
reject before reading, so the module skips itself where a GPU is visible.
"""
import ctypes as C
import math

import pytest
import torch

from paper_1507_00687_gb300 import build as Bld

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host-side rejections are exercised where no device exists")

ARG, NOT_MATMUL, SHAPE, DTYPE, WORKSPACE, UNSUPPORTED = 1, 2, 3, 5, 6, 10
FAKE = C.c_void_p(0x100000)   # never dereferenced: every call below must stop before


@pytest.fixture(scope="module")
def L():
    Bld.build()
    from paper_1507_00687_gb300 import _native
    return _native.lib()


@pytest.fixture(scope="module")
def plans():
    from paper_1507_00687_gb300 import api
    return {"bf16x3": api.Plan(["strassen"], "bf16x3"), "bf16": api.Plan(["strassen"], "bf16"),
            "e4m3": api.Plan(["strassen"], "e4m3b128")}


def test_scale_rejections(L):
    # fmm_scale(steps, A, B, dtype, M, K, N, lda, ldb, eA, d, eB, stream)
    s = lambda *a: L.fmm_scale(*a, None)  # noqa: E731
    assert s(None, FAKE, FAKE, 0, 4, 4, 4, 4, 4, FAKE, FAKE, FAKE) == ARG
    assert s(b"OX", FAKE, FAKE, 0, 4, 4, 4, 4, 4, FAKE, FAKE, FAKE) == ARG
    assert s(b"OI", FAKE, FAKE, 7, 4, 4, 4, 4, 4, FAKE, FAKE, FAKE) == ARG
    assert s(b"", None, None, 0, -1, 4, 4, 4, 4, FAKE, FAKE, FAKE) == ARG
    assert s(b"O", FAKE, FAKE, 0, 4, 4, 4, 4, 4, None, FAKE, FAKE) == ARG
    # an I step alone zero-fills eA and eB first: its operand checks come
    # before those fills
    assert s(b"I", None, FAKE, 0, 4, 4, 4, 4, 4, FAKE, FAKE, FAKE) == ARG
    assert s(b"I", FAKE, FAKE, 0, 4, 4, 4, 3, 4, FAKE, FAKE, FAKE) == SHAPE
    assert s(b"O", FAKE, FAKE, 0, 4, 4, 4, 4, 3, FAKE, FAKE, FAKE) == SHAPE
    # fmm_scale_outside(A, B, dtype, M, K, N, lda, ldb, d_in, eA, eB, stream)
    o = L.fmm_scale_outside
    assert o(FAKE, FAKE, 3, 4, 4, 4, 4, 4, None, FAKE, FAKE, None) == ARG
    assert o(FAKE, FAKE, 0, 4, -4, 4, 4, 4, None, FAKE, FAKE, None) == ARG
    assert o(FAKE, FAKE, 0, 4, 4, 4, 4, 4, None, None, FAKE, None) == ARG
    assert o(FAKE, None, 0, 4, 4, 4, 4, 4, None, FAKE, FAKE, None) == ARG
    assert o(FAKE, FAKE, 0, 4, 4, 4, 2, 4, None, FAKE, FAKE, None) == SHAPE
    # fmm_scale_inside(A, B, dtype, M, K, N, lda, ldb, eA, eB, d, stream)
    i = L.fmm_scale_inside
    assert i(FAKE, FAKE, 0, 4, 4, 4, 4, 4, None, None, None, None) == ARG
    assert i(None, FAKE, 0, 4, 4, 4, 4, 4, None, None, FAKE, None) == ARG
    assert i(FAKE, FAKE, 0, 4, 4, 4, 4, 2, None, None, FAKE, None) == SHAPE


def test_scale_adaptive_rejections(L):
    # fmm_scale_adaptive(A, B, dtype, M, K, N, lda, ldb, tau, max_steps,
    #                    first_inside, eA, d, eB, steps_taken, ws, ws_bytes, stream)
    def a(tau=0.5, max_steps=10, first=0, ws=FAKE, ws_bytes=1 << 20, lda=4):
        return L.fmm_scale_adaptive(FAKE, FAKE, 0, 4, 4, 4, lda, 4, tau, max_steps, first, FAKE, FAKE, FAKE,
                                    None, ws, ws_bytes, None)
    assert a(tau=0.0) == ARG
    assert a(tau=-1.0) == ARG
    assert a(tau=math.nan) == ARG
    assert a(tau=math.inf) == ARG
    assert a(first=2) == ARG
    assert a(max_steps=-1) == ARG
    assert a(lda=3) == SHAPE
    assert a(ws=None) == WORKSPACE
    assert a(ws=C.c_void_p(0x100008)) == WORKSPACE           # not 16-byte aligned
    assert a(ws_bytes=4 * (4 + 4 + 4 + 64) - 1) == WORKSPACE


def test_multiply_rejections(L, plans):
    # fmm_multiply(plan, A, lda, B, ldb, C, ldc, M, K, N, dtype, eA, d, eB, ws, ws_bytes, stream)
    p = plans["bf16x3"]._h

    def m(plan=p, A=FAKE, lda=64, B=FAKE, ldb=64, Cp=FAKE, ldc=64, M=64, K=64, N=64, dt=0):
        return L.fmm_multiply(plan, A, lda, B, ldb, Cp, ldc, M, K, N, dt, None, None, None, None, 0, None)
    assert m(plan=None) == ARG
    assert m(dt=5) == ARG
    assert m(M=-1) == ARG
    assert m(Cp=None) == ARG
    assert m(A=None) == ARG
    assert m(B=None) == ARG
    assert m(lda=63) == SHAPE
    assert m(ldb=63) == SHAPE
    assert m(ldc=63) == SHAPE
    assert m(dt=2) == DTYPE                                  # fp16 data with bf16 hi+lo leaves
    big = (1 << 31) * 2                                      # 2^31 leaf rows: beyond the tile numbering
    assert m(M=big, lda=64) == SHAPE
    # fmm_multiply_backward(plan, dC, lddc, A, lda, B, ldb, dA, ldda, dB, lddb, M, K, N, dtype, ws, ws_bytes, stream)
    bw = L.fmm_multiply_backward
    assert bw(None, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, 64, 64, 64, 0, None, 0, None) == ARG
    assert bw(p, None, 64, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, 64, 64, 64, 0, None, 0, None) == ARG
    assert bw(p, FAKE, 63, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, 64, 64, 64, 0, None, 0, None) == ARG
    assert bw(p, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, FAKE, 64, 64, 64, 64, 2, None, 0, None) == DTYPE
    # fmm_workspace_size(plan, M, K, N, bytes)
    n = C.c_size_t()
    assert L.fmm_workspace_size(None, 4, 4, 4, C.byref(n)) == ARG
    assert L.fmm_workspace_size(p, 4, 4, 4, None) == ARG
    assert L.fmm_workspace_size(p, 4, -4, 4, C.byref(n)) == ARG


def test_plan_setter_rejections(L, plans):
    p = plans["bf16"]._h
    assert L.fmm_plan_set_schedule(None, 0) == ARG
    assert L.fmm_plan_set_schedule(p, -1) == ARG
    assert L.fmm_plan_set_schedule(p, 6) == ARG
    assert L.fmm_plan_set_between_scaling(None, 1) == ARG
    b = C.c_double()
    assert L.fmm_plan_bound(p, -1, 1.0, 1.0, 2.0 ** -24, C.byref(b)) == ARG
    assert L.fmm_plan_bound(p, 64, 1.0, 1.0, 2.0 ** -24, None) == ARG


def test_block_max_rejections(L):
    # fmm_block_max(X, dtype, rows, cols, ld, nrb, ncb, out, stream)
    bm = L.fmm_block_max
    assert bm(FAKE, 4, 8, 8, 8, 2, 2, FAKE, None) == ARG
    assert bm(FAKE, 0, -8, 8, 8, 2, 2, FAKE, None) == ARG
    assert bm(FAKE, 0, 8, 8, 8, 0, 2, FAKE, None) == ARG
    assert bm(FAKE, 0, 8, 8, 8, 2, 65, FAKE, None) == ARG
    assert bm(FAKE, 0, 8, 8, 8, 2, 2, None, None) == ARG
    assert bm(None, 0, 8, 8, 8, 2, 2, FAKE, None) == ARG
    assert bm(FAKE, 0, 8, 8, 7, 2, 2, FAKE, None) == ARG


def test_batch_rejections(L, plans):
    from paper_1507_00687_gb300 import _native as N

    def probs(*specs):
        arr = (N.FmmProblem * len(specs))()
        for i, (plan, M, K, N_) in enumerate(specs):
            arr[i] = N.FmmProblem(plan, FAKE.value, K, FAKE.value, N_, FAKE.value, N_, M, K, N_)
        return arr
    b16, e4 = plans["bf16"]._h.value, plans["e4m3"]._h.value
    x3 = plans["bf16x3"]._h.value
    n = C.c_size_t()
    ws = L.fmm_batch_workspace_size
    assert ws(probs((b16, 256, 256, 256)), 1, 1, b"OI", None) == ARG
    assert ws(None, 1, 1, b"OI", C.byref(n)) == ARG
    assert ws(probs((b16, 256, 256, 256)), 0, 1, b"OI", C.byref(n)) == ARG
    assert ws(probs((b16, 256, 256, 256)), 1, 1, b"OX", C.byref(n)) == ARG
    assert ws(probs((b16, 256, 256, 256)), 1, 9, b"OI", C.byref(n)) == ARG
    assert ws(probs((None, 256, 256, 256)), 1, 1, b"OI", C.byref(n)) == ARG
    assert ws(probs((b16, 0, 256, 256)), 1, 1, b"OI", C.byref(n)) == SHAPE
    bad_ld = probs((b16, 256, 256, 256), (b16, 256, 256, 256))
    bad_ld[1].lda, bad_ld[1].ldb, bad_ld[1].ldc = 256, 256, 255
    assert ws(bad_ld, 2, 1, b"OI", C.byref(n)) == SHAPE                  # ldc < N
    bad_ld[1].ldc, bad_ld[1].ldb = 256, 255
    assert ws(bad_ld, 2, 1, b"OI", C.byref(n)) == SHAPE                  # ldb < N
    bad_ld[1].ldb, bad_ld[1].lda = 256, 255
    assert ws(bad_ld, 2, 1, b"OI", C.byref(n)) == SHAPE                  # lda < K
    assert ws(probs((b16, 256, 256, 256), (x3, 256, 256, 256)), 2, 1, b"OI", C.byref(n)) == ARG  # mixed leaves
    assert ws(probs((x3, 256, 256, 256)), 1, 2, b"OI", C.byref(n)) == DTYPE
    assert ws(probs((e4, 256, 256, 256)), 1, 1, b"OI", C.byref(n)) == UNSUPPORTED
    good = probs((b16, 256, 256, 256), (b16, 512, 128, 384))
    assert ws(good, 2, 1, b"OI", C.byref(n)) == 0 and n.value > 0
    h = C.c_void_p()
    cr = L.fmm_batch_create
    assert cr(None, good, 2, 1, b"OI", FAKE, n.value) == ARG
    assert cr(C.byref(h), good, 2, 1, b"OI", None, n.value) == WORKSPACE
    assert cr(C.byref(h), good, 2, 1, b"OI", C.c_void_p(0x100010), n.value) == WORKSPACE   # not 256-aligned
    assert cr(C.byref(h), good, 2, 1, b"OI", FAKE, n.value - 1) == WORKSPACE
    assert h.value is None
    assert L.fmm_batch_run(None, None) == ARG
    i64 = C.c_int64 * 2
    part = (C.c_int32 * 2)()
    assert L.fmm_batch_partition(i64(4, 4), i64(4, 4), i64(4, 4), 2, 0, part) == ARG
    assert L.fmm_batch_partition(i64(4, -4), i64(4, 4), i64(4, 4), 2, 2, part) == ARG
    assert L.fmm_batch_partition(None, i64(4, 4), i64(4, 4), 2, 2, part) == ARG


def test_host_pipeline_rejections(L, plans):
    # fmm_host_create(out, plan, M, K, N, dtype, steps, depth)
    p = plans["bf16x3"]._h
    h = C.c_void_p()
    hc = L.fmm_host_create
    assert hc(None, p, 64, 64, 64, 0, b"OI", 2) == ARG
    assert hc(C.byref(h), None, 64, 64, 64, 0, b"OI", 2) == ARG
    assert hc(C.byref(h), p, 0, 64, 64, 0, b"OI", 2) == ARG
    assert hc(C.byref(h), p, 64, 64, 64, 6, b"OI", 2) == ARG
    assert hc(C.byref(h), p, 64, 64, 64, 0, b"OQ", 2) == ARG
    assert hc(C.byref(h), p, 64, 64, 64, 0, None, 2) == ARG
    assert hc(C.byref(h), p, 64, 64, 64, 0, b"OI", 0) == ARG
    assert hc(C.byref(h), p, 64, 64, 64, 0, b"OI", 5) == ARG
    assert L.fmm_host_submit(None, FAKE, 64, FAKE, 64, FAKE, 64) == ARG
    assert L.fmm_host_wait(None) == ARG
    assert L.fmm_host_destroy(None) == 0


def test_python_wrappers_check_their_tensors(L):
    # The wrappers reject output and exponent tensors the kernels would
    # write past or misread, before anything reaches the library.
    from paper_1507_00687_gb300 import api
    plan = api.Plan(["strassen"], "bf16x3")
    A, B = torch.zeros((64, 48)), torch.zeros((48, 32))
    i32 = lambda n: torch.zeros(n, dtype=torch.int32)  # noqa: E731
    bad = [
        dict(out=torch.zeros((64, 32), dtype=torch.bfloat16)),      # 2-byte elements
        dict(out=torch.zeros((64, 16))),                             # too few columns
        dict(eA=torch.zeros(64, dtype=torch.int64)),                 # 8-byte exponents
        dict(eA=i32(63)),                                            # one short
        dict(d=i32(64)),                                             # d has length K = 48
        dict(eB=i32(64)[::2]),                                       # strided
        dict(eB=torch.zeros((32, 1), dtype=torch.int32)),            # not 1-D
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            api.multiply(plan, A, B, **kw)
    with pytest.raises(ValueError):
        api.multiply(plan, A, torch.zeros((48, 32), dtype=torch.bfloat16))
    with pytest.raises(ValueError):
        api.multiply_backward(plan, torch.zeros((64, 31)), A, B)
    with pytest.raises(ValueError):
        api.scale_outside(A, B, d=i32(47))
    with pytest.raises(ValueError):
        api.scale_inside(A, B, eA=i32(64), eB=torch.zeros(32, dtype=torch.int16))
    # well-formed tensors get past these checks and stop at the device check
    with pytest.raises(ValueError, match="CUDA"):
        api.multiply(plan, A, B, i32(64), i32(48), i32(32), out=torch.zeros((64, 40))[:, :32])


def test_batch_workspace_covers_every_entry():
    # fmm_batch_workspace_size holds at least every entry's exponent vectors
    # and what its passes write: the combined (or, for a classical entry
    # whose data needs converting, the converted) operands and, with more
    # than one leaf, the FP32 stored products; classical entries with bf16
    # data and bf16 leaves read the caller's matrices and need none.
    import numpy as np
    from paper_1507_00687_gb300 import _native as N
    from paper_1507_00687_gb300 import api
    cdiv = lambda a, b: -(-a // b)  # noqa: E731
    g = np.random.default_rng(23)
    for dt in (N.DT_F32, N.DT_BF16):
        for leaf in ("bf16", "bf16x3"):
            plans = [api.Plan(r, leaf) for r in ([], ["winograd"], ["strassen", "strassen"])]
            specs, need = [], 0
            for i in range(12):
                p = plans[i % 3]
                M, K, N_ = (int(x) for x in g.integers(1, 40, size=3) * 64)
                specs.append((p, M, K, N_))
                inf = p.info()
                R, bm, bk, bn = inf["leaves"], cdiv(M, inf["pm"]), cdiv(K, inf["pk"]), cdiv(N_, inf["pn"])
                need += 4 * (M + K + N_)
                direct = R == 1 and dt == N.DT_BF16 and leaf == "bf16"
                if not direct:
                    need += (2 if leaf == "bf16x3" else 1) * R * (bm + bn) * bk * 2 + (R * bm * bn * 4 if R > 1 else 0)
            arr = (N.FmmProblem * len(specs))()
            for i, (p, M, K, N_) in enumerate(specs):
                arr[i] = N.FmmProblem(p._h.value, FAKE.value, K, FAKE.value, N_, FAKE.value, N_, M, K, N_)
            n = C.c_size_t()
            assert N.lib().fmm_batch_workspace_size(arr, len(specs), dt, b"OI", C.byref(n)) == 0
            assert n.value >= need, (dt, leaf, n.value, need)
