"""fmm_multiply_noalloc: the multiply for callers that cannot allocate device
memory (a caller whose device memory all belongs to a pool or arena it does
not control, a plugin given no scratch buffers, a latency-critical path that
must not risk an allocation).  It works in a static scratch array inside the
library instead of a caller-supplied workspace.

The GPU test calls it through the C ABI twice in a row, on two different
problems, and checks each result against fmm_multiply's on the same inputs
within the parity tolerance of the other GPU tests: the second call must not
be disturbed by what the first left in the shared scratch.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_common import assert_within, dev_values, oracle_reference, require_gpu, to_dev
from oracle import scaling as OS
from paper_1507_00687_gb300 import build as B
from paper_1507_00687_gb300 import inputs


def _noalloc(N, plan, A, Bm, out, eA=None, d=None, eB=None):
    """Call fmm_multiply_noalloc through ctypes; returns the status code."""
    from paper_1507_00687_gb300 import api
    ptr = lambda t: None if t is None else t.data_ptr()
    M, K = A.shape
    Nn = Bm.shape[1]
    stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    return N.lib().fmm_multiply_noalloc(plan.handle, ptr(A), A.stride(0), ptr(Bm), Bm.stride(0), ptr(out),
                                        out.stride(0), M, K, Nn, api.DTYPE[A.dtype], ptr(eA), ptr(d), ptr(eB),
                                        stream)


def test_noalloc_rejects_null_operands():
    # Host-side argument checks: null operands with nonzero sizes are
    # rejected before anything else (no device needed, nothing launched).
    B.build()
    from paper_1507_00687_gb300 import _native as N
    from paper_1507_00687_gb300 import api
    plan = api.Plan(["winograd"], "bf16x3")
    lib = N.lib()
    assert lib.fmm_multiply_noalloc(plan.handle, None, 64, None, 64, None, 64, 64, 64, 64, N.DT_F32,
                                    None, None, None, None) == 1  # FMM_ERR_ARG
    # a shape with nothing to compute needs no operands
    assert lib.fmm_multiply_noalloc(plan.handle, None, 64, None, 64, None, 64, 0, 64, 0, N.DT_F32,
                                    None, None, None, None) == 0


def test_noalloc_rejects_problems_beyond_the_scratch_on_the_host():
    # The size check runs on the host before any device call.  Host buffers
    # stand in for the operands only on a machine without a GPU, where no
    # kernel can be launched whatever the check does.
    if torch.cuda.is_available():
        pytest.skip("host buffers are only passed where no device exists; the GPU test covers this")
    B.build()
    from paper_1507_00687_gb300 import _native as N
    from paper_1507_00687_gb300 import api
    plan = api.Plan(["winograd"], "bf16x3")
    n = 4096  # prepared fp32 operands alone take 128 MiB
    A = torch.empty((n, n), dtype=torch.float32)
    out = torch.empty((n, n), dtype=torch.float32)
    code = _noalloc(N, plan, A, A, out)
    assert code == 6  # FMM_ERR_WORKSPACE
    msg = N.lib().fmm_last_error().decode()
    assert "fmm_multiply_noalloc" in msg and str(N.NOALLOC_SCRATCH_BYTES) in msg


def _need(msg):
    return int(msg.split("needs ")[1].split(" bytes")[0])


@pytest.mark.gpu
def test_noalloc_size_limit_follows_the_path_taken():
    # The scratch must hold the workspace of the path the call takes: the
    # forced pass schedule and E4M3 leaves need the combined operands and the
    # stored products, the automatic schedule the smaller of that and the
    # load-stage schedule's prepared copies.  Beyond the limit the call
    # returns FMM_ERR_WORKSPACE with the byte count and launches nothing (C
    # keeps its contents); below it the result equals fmm_multiply's.
    api = require_gpu()
    from paper_1507_00687_gb300 import _native as N
    lib = N.lib()

    # Winograd, bf16 hi+lo, n = 1536: the pass schedule needs ~50 MB, the
    # prepared copies ~19 MB.
    n = 1536
    A = inputs.uniform((n, n), seed=31, lo=-1.0, hi=1.0)
    Bm = inputs.uniform((n, n), seed=32, lo=-1.0, hi=1.0)
    Ad, Bd = to_dev(A, "f32"), to_dev(Bm, "f32")
    out = torch.full((n, n), 3.0, device="cuda")
    assert _noalloc(N, api.Plan(["winograd"], "bf16x3", "pass"), Ad, Bd, out) == 6
    need = _need(lib.fmm_last_error().decode())
    assert need > N.NOALLOC_SCRATCH_BYTES
    torch.cuda.synchronize()
    assert bool((out == 3.0).all())
    # the same problem under the automatic schedule fits (load-stage copies)
    auto = api.Plan(["winograd"], "bf16x3")
    assert _noalloc(N, auto, Ad, Bd, out) == 0
    ref = api.multiply(api.Plan(["winograd"], "bf16x3", "load_stage"), Ad, Bd)
    api.sync_status()
    A64, B64 = dev_values(Ad), dev_values(Bd)
    C, G = oracle_reference(A64, B64, ["winograd"])
    assert_within(dev_values(out), C, G, ["winograd"], n, "bf16x3", "noalloc, automatic schedule")
    assert_within(dev_values(out), dev_values(ref), G, ["winograd"], n, "bf16x3", "noalloc vs fmm_multiply")

    # forced pass schedule below the limit (n = 1024: ~22 MB)
    m = 1024
    Ad2, Bd2 = Ad[:m, :m].contiguous(), Bd[:m, :m].contiguous()
    plan = api.Plan(["winograd"], "bf16x3", "pass")
    got = torch.full((m, m), float("nan"), device="cuda")
    assert _noalloc(N, plan, Ad2, Bd2, got) == 0
    ref = api.multiply(plan, Ad2, Bd2)
    api.sync_status()
    C, G = oracle_reference(dev_values(Ad2), dev_values(Bd2), ["winograd"])
    assert_within(dev_values(got), dev_values(ref), G, ["winograd"], m, "bf16x3", "noalloc, pass schedule")

    # E4M3 leaves (pass schedule only): Strassen two levels at n = 1536
    # exceeds the scratch, Strassen one level at n = 512 fits
    names = ["strassen", "strassen"]
    assert _noalloc(N, api.Plan(names, "e4m3b128"), Ad, Bd, out) == 6
    assert _need(lib.fmm_last_error().decode()) > N.NOALLOC_SCRATCH_BYTES
    s = 512
    Ad3, Bd3 = Ad[:s, :s].contiguous(), Bd[:s, :s].contiguous()
    plan = api.Plan(["strassen"], "e4m3b128")
    got = torch.full((s, s), float("nan"), device="cuda")
    assert _noalloc(N, plan, Ad3, Bd3, got) == 0
    ref = api.multiply(plan, Ad3, Bd3)
    api.sync_status()
    C, G = oracle_reference(dev_values(Ad3), dev_values(Bd3), ["strassen"])
    assert_within(dev_values(got), dev_values(ref), G, ["strassen"], s, "e4m3b128", "noalloc, E4M3 leaves")


@pytest.mark.gpu
def test_noalloc_matches_fmm_multiply_on_two_calls_in_a_row():
    api = require_gpu()
    from paper_1507_00687_gb300 import _native as N

    # Call 1: Winograd, bf16 hi+lo leaves, fp32 inputs with outside-inside
    # scaling and ragged sizes, so both operands are prepared in the scratch.
    names1 = ["winograd"]
    A1, B1 = inputs.diag_scaled_pair(300, 260, 212, seed=2024)
    Ad1, Bd1 = to_dev(A1, "f32"), to_dev(B1, "f32")
    eA, d, eB = api.scale(Ad1, Bd1, "OI")
    plan1 = api.Plan(names1, "bf16x3")
    ref1 = api.multiply(plan1, Ad1, Bd1, eA, d, eB)
    got1 = torch.full_like(ref1, float("nan"))
    assert _noalloc(N, plan1, Ad1, Bd1, got1, eA, d, eB) == 0

    # Call 2, straight after: a different plan (Strassen then Winograd, plain
    # bf16 leaves), bf16 inputs, no scaling, another shape.
    names2 = ["strassen", "winograd"]
    A2 = inputs.uniform((384, 520), seed=7, lo=-1.0, hi=1.0)
    B2 = inputs.uniform((520, 264), seed=8, lo=-1.0, hi=1.0)
    Ad2, Bd2 = to_dev(A2, "bf16"), to_dev(B2, "bf16")
    plan2 = api.Plan(names2, "bf16")
    ref2 = api.multiply(plan2, Ad2, Bd2)
    got2 = torch.full_like(ref2, float("nan"))
    assert _noalloc(N, plan2, Ad2, Bd2, got2) == 0
    api.sync_status()

    A64, B64 = dev_values(Ad1), dev_values(Bd1)
    st = OS.pow2_repeated(A64, B64, "OI")
    C1, G1 = oracle_reference(A64, B64, names1, st.eA, st.d, st.eB)
    r1, g1 = dev_values(ref1), dev_values(got1)
    assert_within(r1, C1, G1, names1, 260, "bf16x3", "fmm_multiply, call 1")
    assert_within(g1, C1, G1, names1, 260, "bf16x3", "fmm_multiply_noalloc, call 1")
    assert_within(g1, r1, G1, names1, 260, "bf16x3", "noalloc vs fmm_multiply, call 1")

    A64, B64 = dev_values(Ad2), dev_values(Bd2)
    C2, G2 = oracle_reference(A64, B64, names2)
    r2, g2 = dev_values(ref2), dev_values(got2)
    assert_within(g2, C2, G2, names2, 520, "bf16", "fmm_multiply_noalloc, call 2")
    assert_within(g2, r2, G2, names2, 520, "bf16", "noalloc vs fmm_multiply, call 2")
