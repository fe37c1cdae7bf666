"""Parity at the full sizes of the workloads the benchmark describes, on
sampled outputs: the precision sweep (n = 8192 square and M = 8192,
K = 16384, N = 4096; Strassen / Winograd composed with classical <1,2,1>,
one to four levels; BF16, FP16 and E4M3 leaves), the fast-matmul linear
layer (X[8192, 4096] W[4096, 4096], Strassen two levels, forward and
backward) and the batch of 512 uneven products.

Each sampled entry is checked against its exact value (a float64 dot
product of the stored inputs) within the elementwise tolerance of
gpu_common, whose growth quantity the oracle evaluates at the sampled
entries only (``growth_entries``); the scaling exponents at full size are
checked bit-exact against the oracle.
"""
import numpy as np
import pytest
import torch

from gpu_common import ORACLE_RULES, U_LEAF, dev_values, require_gpu, to_dev
from oracle import fmm as OF
from oracle import rules as OR
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu

SAMPLES = 48


@pytest.fixture(scope="module")
def api():
    return require_gpu()


def _tol(G, rules, K, leaf):
    pk = int(np.prod([r.k0 for r in rules]))
    kl = -(-K // pk)
    t = 1
    for r in rules:
        p = OR.principal(r)
        t *= int(max(p.alpha.max(), p.beta.max(), (r.W != 0).sum(axis=0).max()))
    return (U_LEAF[leaf] + (kl + 2 * t + 8) * 2.0**-23) * G


def _samples(M, N, seed):
    g = np.random.default_rng(seed)
    rows = np.concatenate([[0, M - 1], g.integers(0, M, size=SAMPLES - 2)])
    cols = np.concatenate([[N - 1, 0], g.integers(0, N, size=SAMPLES - 2)])
    return rows, cols


def _check_entries(got, A64, B64, rules, rows, cols, leaf, K, what, scales=None):
    """got: sampled GPU values; A64, B64: the operands the fast algorithm
    multiplies (scaled when ``scales`` = (eA, eB) is given, C then being
    2^eA_i (A' B')_ij 2^eB_j)."""
    exact = np.einsum("sk,ks->s", A64[rows, :], B64[:, cols])
    G = OF.growth_entries(A64, B64, rules, rows, cols)
    if scales is not None:
        eA, eB = scales
        f = np.exp2((eA[rows] + eB[cols]).astype(np.float64))
        exact, G = exact * f, G * f
    tol = _tol(G, rules, K, leaf)
    err = np.abs(got - exact)
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {len(rows)} sampled entries outside tolerance"
    return float((err / tol).max())


SWEEP_PLANS = {
    1: ["strassen"],
    2: ["winograd", "classical121"],
    3: ["strassen", "classical121", "strassen"],
    4: ["winograd", "classical121", "winograd", "classical121"],
}
SHAPES = [(8192, 8192, 8192), (8192, 16384, 4096)]
_cache = {}


def _operands(shape, dist):
    key = (shape, dist)
    if key not in _cache:
        _cache.clear()
        M, K, N = shape
        if dist == "uniform":
            A = inputs.uniform((M, K), -1, 1, seed=M + K)
            B = inputs.uniform((K, N), -1, 1, seed=K + N)
        else:
            A, B = inputs.diag_scaled_pair(M, K, N, seed=M + 2 * K + 3 * N)
        # the values the device holds (FP32)
        _cache[key] = (A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64))
    return _cache[key]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dist", ["uniform", "scaled"])
def test_precision_sweep_full_size(api, shape, dist):
    M, K, N = shape
    A64, B64 = _operands(shape, dist)
    Ad, Bd = torch.from_numpy(A64).float().cuda(), torch.from_numpy(B64).float().cuda()
    rows, cols = _samples(M, N, seed=M + N)
    ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    scales, Ap, Bp = None, A64, B64
    eA = d = eB = None
    if dist == "scaled":
        # outside-inside scaling: the exponents at full size bit-exact
        eA, d, eB = api.scale(Ad, Bd, "OI")
        st = OS.pow2_repeated(A64, B64, "OI")
        assert np.array_equal(eA.cpu().numpy(), st.eA) and np.array_equal(d.cpu().numpy(), st.d)
        assert np.array_equal(eB.cpu().numpy(), st.eB)
        Ap, Bp = OS.pow2_apply(A64, B64, st.eA, st.d, st.eB)
        scales = (st.eA, st.eB)
    cases = [(L, "bf16") for L in SWEEP_PLANS] + [(2, "fp16"), (4, "fp16"), (2, "e4m3b128"), (4, "e4m3b128")]
    for L, leaf in cases:
        names = SWEEP_PLANS[L]
        plan = api.Plan(names, leaf)
        C = api.multiply(plan, Ad, Bd, eA, d, eB)
        api.sync_status()
        got = C[ri, ci].double().cpu().numpy()
        del C
        rules = [ORACLE_RULES[n]() for n in names]
        _check_entries(got, Ap, Bp, rules, rows, cols, leaf, K, f"{shape} {dist} L={L} {leaf}", scales)
    del Ad, Bd
    torch.cuda.empty_cache()


def test_linear_layer_full_size(api):
    # Y = X W, dX = dY W^T, dW = X^T dY with Strassen two levels, BF16
    # operands and BF16 leaves (the autograd workload).  The gradients are
    # checked in FP32 from the library's backward call; the autograd
    # function returns the same values rounded to the operands' BF16.
    Mx, Kx, Nx = 8192, 4096, 4096
    X = to_dev(inputs.uniform((Mx, Kx), -1, 1, seed=11), "bf16")
    W = to_dev(inputs.uniform((Kx, Nx), -1, 1, seed=12), "bf16")
    dY = to_dev(inputs.uniform((Mx, Nx), -1, 1, seed=13), "f32")
    plan = api.Plan(["strassen", "strassen"], "bf16")
    Y = api.multiply(plan, X, W)
    dX, dW = api.multiply_backward(plan, dY, X, W)
    Xg, Wg = X.clone().requires_grad_(True), W.clone().requires_grad_(True)
    api.FastMatmul.apply(Xg, Wg, plan).backward(dY)
    api.sync_status()
    assert torch.equal(Xg.grad, dX.to(torch.bfloat16)) and torch.equal(Wg.grad, dW.to(torch.bfloat16))
    X64, W64, dY64 = dev_values(X), dev_values(W), dev_values(dY)
    s = OR.strassen()

    def at(T, rows, cols):
        return T[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].double().cpu().numpy()

    rows, cols = _samples(Mx, Nx, seed=5)
    _check_entries(at(Y, rows, cols), X64, W64, [s, s], rows, cols, "bf16", Kx, "forward")
    # dX = dY W^T: an <m0, n0, k0> product by the rule for dA
    rows, cols = _samples(Mx, Kx, seed=6)
    _check_entries(at(dX, rows, cols), dY64, W64.T, [OR.rule_for_dA(s)] * 2, rows, cols, "bf16", Nx, "dX")
    # dW = X^T dY: a <k0, m0, n0> product by the rule for dB
    rows, cols = _samples(Kx, Nx, seed=7)
    _check_entries(at(dW, rows, cols), X64.T, dY64, [OR.rule_for_dB(s)] * 2, rows, cols, "bf16", Mx, "dW")


def test_batch_of_512_full_size(api):
    # 512 products with every dimension log-uniform over the multiples of 128
    # in [512, 4096], BF16 operands U[-1, 1], BF16 leaves, outside-inside
    # scaling, plans from the autotuner, one launch sequence under a CUDA
    # graph; 16 products checked at sampled entries, the tolerance built
    # from the oracle's scaling exponents of each.
    dims = inputs.log_uniform_dims(512, 512, 4096, 128, seed=1507 + 4000)
    tuner = api.Autotuner(leaf="bf16", dtype=torch.bfloat16, sizes=(512, 1024, 2048), reps=2)
    gen = torch.Generator(device="cuda").manual_seed(1507 + 4001)
    probs, names = [], []
    for M, K, N in dims.tolist():
        A = (torch.rand((M, K), generator=gen, device="cuda") * 2 - 1).to(torch.bfloat16)
        B = (torch.rand((K, N), generator=gen, device="cuda") * 2 - 1).to(torch.bfloat16)
        names.append(tuner.choose(M, K, N))
        probs.append((tuner.plan(M, K, N), A, B, torch.full((M, N), float("nan"), device="cuda")))
    batch = api.Batch(probs, "OI")
    batch.run()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run()
    for _, _, _, Cm in probs:
        Cm.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    api.sync_status()
    for i in range(0, 512, 32):
        _, A, B, Cm = probs[i]
        M, K = A.shape
        N = B.shape[1]
        A64, B64 = dev_values(A), dev_values(B)
        st = OS.pow2_repeated(A64, B64, "OI")
        Ap, Bp = OS.pow2_apply(A64, B64, st.eA, st.d, st.eB)
        rows, cols = _samples(M, N, seed=i)
        got = Cm[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].double().cpu().numpy()
        rules = [ORACLE_RULES[n]() for n in names[i]] or [OR.classical(1, 1, 1)]
        _check_entries(got, Ap, Bp, rules, rows, cols, "bf16", K, f"batch product {i} {names[i]}", (st.eA, st.eB))
    del batch, probs, g
    torch.cuda.empty_cache()
