"""The host-memory pipeline (fmm_host_*): products submitted from host
buffers give exactly what the device entry points give on the same
values, at every pipeline depth, with pinned or pageable memory."""
import numpy as np
import pytest
import torch

from gpu_common import dev_values, require_gpu
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return require_gpu()


def _device_result(api, plan, A, B, steps):
    Ad, Bd = A.cuda(), B.cuda()
    if steps:
        eA, d, eB = api.scale(Ad, Bd, steps)
        return api.multiply(plan, Ad, Bd, eA, d, eB).cpu()
    return api.multiply(plan, Ad, Bd).cpu()


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("steps", ["OI", ""])
def test_host_pipeline_equals_device_path(api, depth, steps):
    M, K, N = 520, 384, 456
    plan = api.Plan(["winograd"], "bf16x3")
    pipe = api.HostPipeline(plan, M, K, N, torch.float32, steps, depth)
    ins = []
    for i in range(5):
        A, B = inputs.diag_scaled_pair(M, K, N, seed=100 + i, span=6.0)
        ins.append((torch.from_numpy(A).float().pin_memory(), torch.from_numpy(B).float().pin_memory(),
                    torch.full((M, N), float("nan")).pin_memory()))
    for A, B, C in ins:
        pipe.submit(A, B, C)
    pipe.wait()
    for A, B, C in ins:
        assert torch.equal(C, _device_result(api, plan, A, B, steps))


def test_host_pipeline_pageable_strided_bf16(api):
    M, K, N = 300, 256, 200
    plan = api.Plan(["strassen", "strassen"], "bf16")
    pipe = api.HostPipeline(plan, M, K, N, torch.bfloat16, "OI", 2)
    Abig = torch.from_numpy(inputs.uniform((M, K + 8), -1, 1, seed=1)).to(torch.bfloat16)
    Bbig = torch.from_numpy(inputs.uniform((K, N + 24), -1, 1, seed=2)).to(torch.bfloat16)
    Cbig = torch.full((M, N + 4), 7.0)
    A, B, C = Abig[:, :K], Bbig[:, :N], Cbig[:, :N]
    pipe.submit(A, B, C)
    pipe.wait()
    assert torch.equal(C, _device_result(api, plan, A.contiguous(), B.contiguous(), "OI"))
    assert torch.all(Cbig[:, N:] == 7.0)
    # integer inputs: exact
    Ai = inputs.integers((M, K), -4, 4, seed=3)
    Bi = inputs.integers((K, N), -4, 4, seed=4)
    Ci = torch.empty((M, N))
    pipe.submit(torch.from_numpy(Ai).to(torch.bfloat16), torch.from_numpy(Bi).to(torch.bfloat16), Ci)
    pipe.wait()
    assert np.array_equal(Ci.double().numpy(), Ai @ Bi)


def test_host_pipeline_rejects_bad_arguments(api):
    from paper_1507_00687_gb300 import _native as N
    import ctypes as C
    plan = api.Plan(["strassen"], "bf16x3")
    L = N.lib()
    h = C.c_void_p()
    arg = 1  # FMM_ERR_ARG
    assert L.fmm_host_create(C.byref(h), plan.handle, 0, 4, 4, N.DT_F32, b"OI", 2) == arg
    assert L.fmm_host_create(C.byref(h), plan.handle, 4, 4, 4, N.DT_F32, b"OX", 2) == arg
    assert L.fmm_host_create(C.byref(h), plan.handle, 4, 4, 4, N.DT_F32, b"OI", 5) == arg
    pipe = api.HostPipeline(plan, 8, 8, 8)
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros(8, 8).cuda(), torch.zeros(8, 8), torch.zeros(8, 8))
    assert L.fmm_host_submit(pipe._h, None, 8, None, 8, None, 8) == arg
