"""Adaptive Alg. 3 with the tau stopping test (Sec. 6.3) on the GPU against
the oracle: exponents and the number of steps bit-exact."""
import numpy as np
import pytest
import torch

from gpu_common import dev_values, oracle_reference, assert_within, require_gpu, to_dev
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return require_gpu()


def _check(api, Ad, Bd, tau, max_steps, first):
    eA, d, eB, steps = api.scale_adaptive(Ad, Bd, tau, max_steps, first)
    api.sync_status()
    st, t = OS.pow2_adaptive(dev_values(Ad), dev_values(Bd), tau, max_steps, first)
    assert int(steps.item()) == t, (tau, max_steps, first)
    assert np.array_equal(eA.cpu().numpy(), st.eA)
    assert np.array_equal(d.cpu().numpy(), st.d)
    assert np.array_equal(eB.cpu().numpy(), st.eB)
    return t


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("first", ["O", "I"])
def test_adaptive_bit_exact(api, kind, dt, first):
    A, B = inputs.paper_distribution(kind, 300, seed=kind)
    A, B = A[:, :260], B[:260, :290]  # M = 300, K = 260, N = 290
    Ad, Bd = to_dev(A, dt), to_dev(B, dt)
    for tau in (1e-3, 0.5, 15.0, 255.0, 1e6):
        for max_steps in (0, 1, 2, 5, 40):
            t = _check(api, Ad, Bd, tau, max_steps, first)
            assert t <= max_steps
        assert t < 40  # the uncapped iteration stops by its test


@pytest.mark.parametrize("L", [4, 8, 16, 64])
def test_adaptive_lemma_d4_stop_step(api, L):
    # the closed-form stopping step of the Lemma D.4 example (v = 6), as
    # pinned for the oracle: 11, 9, 7, 3 for L = 4, 8, 16, 64
    v = 6
    A = np.array([[1.0, 0.0], [1.0, 2.0 ** -(2**v)]])
    B = np.eye(2)
    want = {4: 11, 8: 9, 16: 7, 64: 3}[L]
    _, _, _, steps = api.scale_adaptive(to_dev(A, "f32"), to_dev(B, "f32"), 2.0**L - 1, 40)
    assert int(steps.item()) == want
    assert _check(api, to_dev(A, "f32"), to_dev(B, "f32"), 2.0**L - 1, 40, "O") == want


def test_adaptive_edges(api):
    A = np.array([[0.0, 0.0, 0.0], [1.0, 2.0**20, 3.0]])
    B = np.array([[0.0, 5.0], [0.0, 2.0**-30], [0.0, 1.0]])
    _check(api, to_dev(A, "f32"), to_dev(B, "f32"), 1e-2, 30, "O")
    _check(api, to_dev(A, "f32"), to_dev(B, "f32"), 1e-2, 30, "I")
    for M, K, N in ((0, 5, 4), (4, 0, 3), (3, 5, 0)):
        Ad = to_dev(inputs.uniform((M, K), -1, 1, seed=1), "f32")
        Bd = to_dev(inputs.uniform((K, N), -1, 1, seed=2), "f32")
        _check(api, Ad, Bd, 0.1, 7, "O")
    from paper_1507_00687_gb300 import _native as N
    Ad = to_dev(inputs.uniform((8, 8), -1, 1, seed=1), "f32")
    with pytest.raises(N.FmmError):
        api.scale_adaptive(Ad, Ad, 0.0, 3)


def test_adaptive_steps_after_the_stop_change_nothing(api):
    A, B = inputs.paper_distribution(3, 256, seed=9)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    t = _check(api, Ad, Bd, 1e-3, 100, "O")
    assert t < 100
    a = [x.cpu() for x in api.scale_adaptive(Ad, Bd, 1e-3, t)[:3]]
    b = [x.cpu() for x in api.scale_adaptive(Ad, Bd, 1e-3, 100)[:3]]
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_adaptive_in_a_cuda_graph(api):
    # the stop is decided on the device, so a captured iteration replays on
    # new inputs and stops where the oracle does for them
    M = K = N = 256
    Ad = torch.empty((M, K), device="cuda")
    Bd = torch.empty((K, N), device="cuda")
    A0, B0 = inputs.paper_distribution(1, M, seed=31)
    Ad.copy_(torch.from_numpy(A0).float())
    Bd.copy_(torch.from_numpy(B0).float())
    api.scale_adaptive(Ad, Bd, 1e-3, 24)  # warm up (library init, attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            eA, d, eB, steps = api.scale_adaptive(Ad, Bd, 1e-3, 24, stream=s)
    for kind in (2, 3, 1):
        A, B = inputs.paper_distribution(kind, M, seed=40 + kind)
        Ad.copy_(torch.from_numpy(A).float())
        Bd.copy_(torch.from_numpy(B).float())
        g.replay()
        torch.cuda.synchronize()
        st, t = OS.pow2_adaptive(dev_values(Ad), dev_values(Bd), 1e-3, 24, "O")
        assert int(steps.item()) == t
        assert np.array_equal(eA.cpu().numpy(), st.eA) and np.array_equal(d.cpu().numpy(), st.d)
        assert np.array_equal(eB.cpu().numpy(), st.eB)


@pytest.mark.parametrize("kind", [2, 3])
def test_adaptive_scaled_product_within_tolerance(api, kind):
    names = ["strassen", "strassen"]
    A, B = inputs.paper_distribution(kind, 384, seed=50 + kind)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    eA, d, eB, steps = api.scale_adaptive(Ad, Bd, 1e-3, 30)
    got = dev_values(api.multiply(api.Plan(names, "bf16x3", "pass"), Ad, Bd, eA, d, eB))
    api.sync_status()
    st, _ = OS.pow2_adaptive(A64, B64, 1e-3, 30)
    C, G = oracle_reference(A64, B64, names, st.eA, st.d, st.eB)
    assert_within(got, C, G, names, A.shape[1], "bf16x3", f"adaptive kind {kind}")
