"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer and exponent outputs must match bit for bit; floating-point outputs
must lie within the elementwise tolerance derived in gpu_common.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_common import (assert_within, dev_values, oracle_reference, require_gpu, to_dev)
from oracle import fmm as OF
from oracle import precision as OP
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return require_gpu()


# ---------------------------------------------------------------- scaling

SCALE_CASES = [(257, 300, 129, "f32"), (64, 64, 64, "bf16"), (500, 33, 700, "f32"), (96, 1000, 40, "bf16"),
               (7, 5, 3, "f32")]


@pytest.mark.parametrize("M,K,N,dt", SCALE_CASES)
@pytest.mark.parametrize("steps", ["O", "I", "OI", "IO", "OIOI"])
@pytest.mark.parametrize("kind", [1, 2, 3, 0])
def test_scale_exponents_bit_exact(api, M, K, N, dt, steps, kind):
    if kind == 0:
        A, B = inputs.diag_scaled_pair(M, K, N, seed=M + K + N)
    else:
        A, _ = inputs.paper_distribution(kind, max(M, K), seed=kind)
        _, B = inputs.paper_distribution(kind, max(K, N), seed=kind + 7)
        A, B = A[:M, :K], B[:K, :N]
    Ad, Bd = to_dev(A, dt), to_dev(B, dt)
    A64, B64 = dev_values(Ad), dev_values(Bd)
    eA, d, eB = api.scale(Ad, Bd, steps)
    api.sync_status()
    want = OS.pow2_repeated(A64, B64, steps)
    assert np.array_equal(eA.cpu().numpy(), want.eA)
    assert np.array_equal(d.cpu().numpy(), want.d)
    assert np.array_equal(eB.cpu().numpy(), want.eB)


def test_scale_zero_rows_cols_and_strides(api):
    g = np.random.default_rng(3)
    A = g.uniform(-1, 1, (50, 40))
    B = g.uniform(-1, 1, (40, 30))
    A[[0, 7], :] = 0
    A[:, 5] = 0
    B[:, [2, 29]] = 0
    B[11, :] = 0
    # a leading dimension larger than the row (column slice of a wider buffer)
    Abuf = torch.zeros((50, 48), dtype=torch.float32, device="cuda")
    Abuf[:, :40] = torch.from_numpy(A).float()
    Ad = Abuf[:, :40]
    Bd = to_dev(B, "f32")
    for steps in ("O", "OI", "IOIO"):
        eA, d, eB = api.scale(Ad, Bd, steps)
        want = OS.pow2_repeated(dev_values(Ad), dev_values(Bd), steps)
        assert np.array_equal(eA.cpu().numpy(), want.eA)
        assert np.array_equal(d.cpu().numpy(), want.d)
        assert np.array_equal(eB.cpu().numpy(), want.eB)


def test_scale_nonfinite_flagged(api):
    A = torch.ones((8, 8), device="cuda")
    B = torch.ones((8, 8), device="cuda")
    A[3, 3] = float("inf")
    api.scale(A, B, "O")
    with pytest.raises(Exception) as e:
        api.sync_status()
    assert "NONFINITE" in str(e.value)
    api.sync_status()  # cleared


# ---------------------------------------------------------------- multiply, exact

PLANS = [[], ["strassen"], ["winograd"], ["strassen", "strassen"], ["winograd", "winograd"],
         ["winograd", "classical121"], ["fast323"], ["strassen", "classical121", "strassen"],
         ["strassen", "fast323"]]
SHAPES = [(256, 256, 256), (300, 200, 250), (16, 16, 16), (1000, 520, 776), (1, 3, 2), (129, 65, 257)]

# Where S_r and T_r are formed: in the multiply kernel's load stage, or by
# the combination pass into the workspace -- with the output combination in
# the multiply epilogue or over stored leaf products.  All three are checked
# everywhere the multiply is.
SCHEDULES = ["load_stage", "pass_epilogue", "pass_products", "pass_accumulate"]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("names", PLANS, ids=lambda n: "-".join(n) or "classical")
@pytest.mark.parametrize("M,K,N", SHAPES)
def test_multiply_integer_inputs_bit_exact(api, schedule, names, M, K, N):
    # Entries in [-4, 4]: every S, T entry is an integer small enough to be
    # exact in bf16 and fp16 and every sum stays below 2^24, so the fast
    # algorithm must return exactly the classical product.
    A = inputs.integers((M, K), -4, 4, seed=M)
    B = inputs.integers((K, N), -4, 4, seed=N + 1)
    want = A @ B
    for dt, leaf in (("f32", "bf16x3"), ("bf16", "bf16"), ("f32", "fp16"), ("f16", "fp16"), ("bf16", "bf16x3")):
        plan = api.Plan(names, leaf, schedule)
        got = api.multiply(plan, to_dev(A, dt), to_dev(B, dt))
        api.sync_status()
        assert np.array_equal(dev_values(got), want), (dt, leaf)


# Shapes whose tiling is exact take the streaming producers (every tile
# interior); the last one has more tiles than SMs, so CTAs loop over tiles.
STREAM_CASES = [(["strassen"], 512, 256, 1024), (["winograd", "winograd"], 512, 256, 1024),
                (["strassen", "classical121"], 256, 256, 512), ([], 4096, 128, 4096),
                (["winograd"], 2048, 384, 1024)]


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("names,M,K,N", STREAM_CASES, ids=lambda x: "-".join(x) if isinstance(x, list) else str(x))
def test_streaming_path_integer_exact_and_uniform(api, schedule, names, M, K, N):
    A = inputs.integers((M, K), -4, 4, seed=M + 3)
    B = inputs.integers((K, N), -4, 4, seed=N + 4)
    for dt, leaf in (("f32", "bf16x3"), ("bf16", "bf16"), ("f32", "fp16")):
        got = api.multiply(api.Plan(names, leaf, schedule), to_dev(A, dt), to_dev(B, dt))
        api.sync_status()
        assert np.array_equal(dev_values(got), A @ B), (dt, leaf)
    Ar = inputs.uniform((M, K), -1, 1, seed=7)
    Br = inputs.uniform((K, N), -1, 1, seed=8)
    Ad, Bd = to_dev(Ar, "f32"), to_dev(Br, "f32")
    got = dev_values(api.multiply(api.Plan(names, "bf16x3", schedule), Ad, Bd))
    C, G = oracle_reference(dev_values(Ad), dev_values(Bd), names)
    assert_within(got, C, G, names, K, "bf16x3", "streaming")


def test_multiply_leading_dims_and_k_zero(api):
    A = inputs.integers((70, 90), -3, 3, seed=1)
    B = inputs.integers((90, 50), -3, 3, seed=2)
    Ab = torch.zeros((70, 97), device="cuda")
    Ab[:, :90] = torch.from_numpy(A).float()
    Bb = torch.zeros((90, 61), device="cuda")
    Bb[:, :50] = torch.from_numpy(B).float()
    Cb = torch.full((70, 53), 7.0, device="cuda")
    plan = api.Plan(["strassen"], "bf16x3")
    api.multiply(plan, Ab[:, :90], Bb[:, :50], out=Cb[:, :50])
    api.sync_status()
    assert np.array_equal(dev_values(Cb[:, :50]), A @ B)
    assert torch.all(Cb[:, 50:] == 7.0)
    Z = api.multiply(plan, torch.zeros((5, 0), device="cuda"), torch.zeros((0, 4), device="cuda"))
    assert torch.all(Z == 0)


# ---------------------------------------------------------------- multiply, real inputs

@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("names", [[], ["strassen"], ["winograd"], ["strassen", "strassen"],
                                   ["winograd", "winograd"], ["fast323"]], ids=lambda n: "-".join(n) or "classical")
@pytest.mark.parametrize("leaf", ["bf16x3", "bf16", "fp16"])
def test_multiply_uniform_within_tolerance(api, schedule, names, leaf):
    M, K, N = 700, 520, 650
    A = inputs.uniform((M, K), -1, 1, seed=5)
    B = inputs.uniform((K, N), -1, 1, seed=6)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan(names, leaf, schedule)
    got = dev_values(api.multiply(plan, Ad, Bd))
    api.sync_status()
    C, G = oracle_reference(A64, B64, names)
    assert_within(got, C, G, names, K, leaf, f"{names} {leaf}")


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("names", [["strassen"], ["winograd"], []], ids=lambda n: "-".join(n) or "classical")
@pytest.mark.parametrize("leaf", ["bf16", "fp16", "bf16x3"])
def test_multiply_matches_rounding_emulation(api, schedule, names, leaf):
    # One level: S_r, T_r are formed in FP32 in index order on both sides, so
    # the rounded leaf operands agree exactly; only the FP32 accumulation of
    # the tensor core and of the output sums differ.
    M, K, N = 384, 640, 320
    A = inputs.uniform((M, K), -1, 1, seed=15)
    B = inputs.uniform((K, N), -1, 1, seed=16)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan(names, leaf, schedule)
    got = dev_values(api.multiply(plan, Ad, Bd))
    from gpu_common import oracle_tree
    tree = oracle_tree(names)
    leaf_fn = OF.leaf_bf16x3 if leaf == "bf16x3" else OF.leaf_rounded(leaf)
    emu = OF.fmm(A64, B64, tree, leaf=leaf_fn, dtype=np.float32).astype(np.float64)
    _, G = oracle_reference(A64, B64, names)
    kl = K // (2 if names else 1)
    tol = (kl + 16) * 2.0**-23 * G
    assert np.all(np.abs(got - emu) <= tol)


def test_bf16x3_detects_dropped_correction(api):
    # Sensitivity of the tolerance: bf16 leaves (no hi/lo correction) on the
    # same inputs fall outside the bf16x3 tolerance, so a kernel that dropped
    # a correction product would fail the test above.
    M = K = N = 512
    A = inputs.uniform((M, K), -1, 1, seed=25)
    B = inputs.uniform((K, N), -1, 1, seed=26)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    got = dev_values(api.multiply(api.Plan(["strassen"], "bf16"), Ad, Bd))
    C, G = oracle_reference(dev_values(Ad), dev_values(Bd), ["strassen"])
    with pytest.raises(AssertionError):
        assert_within(got, C, G, ["strassen"], K, "bf16x3")


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("steps", ["", "O", "OI", "IO", "OIOI"])
@pytest.mark.parametrize("names", [["winograd"], ["strassen", "strassen"]], ids=lambda n: "-".join(n))
def test_multiply_scaled_within_tolerance(api, schedule, steps, names):
    M, K, N = 512, 384, 448
    A, B = inputs.diag_scaled_pair(M, K, N, seed=9)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    if steps:
        st = OS.pow2_repeated(A64, B64, steps)
        eA, d, eB = st.eA, st.d, st.eB
        tA = torch.from_numpy(eA.astype(np.int32)).cuda()
        td = torch.from_numpy(d.astype(np.int32)).cuda()
        tB = torch.from_numpy(eB.astype(np.int32)).cuda()
    else:
        eA = d = eB = None
        tA = td = tB = None
    plan = api.Plan(names, "bf16x3", schedule)
    got = dev_values(api.multiply(plan, Ad, Bd, tA, td, tB))
    api.sync_status()
    C, G = oracle_reference(A64, B64, names, eA, d, eB)
    assert_within(got, C, G, names, K, "bf16x3", f"scaled {steps}")


def test_scaling_improves_componentwise_error(api):
    # Sec. 6.5, distribution 2 (inside-scaling adversary), one Winograd level
    # with bf16x3 leaves: outside-inside scaling reduces the componentwise
    # relative error of the GPU result.
    n = 512
    A, B = inputs.paper_distribution(2, n, seed=41)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    exact = A64 @ B64
    plan = api.Plan(["winograd"], "bf16x3")
    plain = dev_values(api.multiply(plan, Ad, Bd))
    eA, d, eB = api.scale(Ad, Bd, "IO")
    scaled = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
    api.sync_status()
    e_plain = OF.err_componentwise(plain, exact)
    e_scaled = OF.err_componentwise(scaled, exact)
    assert e_scaled < e_plain / 4


# ---------------------------------------------------------------- backward

@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("names", [["strassen"], ["winograd"], ["strassen", "strassen"], ["fast323"], []],
                         ids=lambda n: "-".join(n) or "classical")
def test_backward_against_oracle(api, schedule, names):
    from oracle import rules as OR
    from gpu_common import ORACLE_RULES
    M, K, N = 320, 256, 384
    A = inputs.uniform((M, K), -1, 1, seed=51)
    B = inputs.uniform((K, N), -1, 1, seed=52)
    G0 = inputs.uniform((M, N), -1, 1, seed=53)
    Ad, Bd, dC = to_dev(A, "bf16"), to_dev(B, "bf16"), to_dev(G0, "f32")
    A64, B64, dC64 = dev_values(Ad), dev_values(Bd), dev_values(dC)
    plan = api.Plan(names, "bf16x3", schedule)
    dA, dB = api.multiply_backward(plan, dC, Ad, Bd)
    api.sync_status()
    ra = OF.uniform([OR.rule_for_dA(ORACLE_RULES[n]()) for n in names])
    rb = OF.uniform([OR.rule_for_dB(ORACLE_RULES[n]()) for n in names])
    # exact gradients of sum(dC * (A B)) and the growth of the permuted rules
    want_a, want_b = dC64 @ B64.T, A64.T @ dC64
    Ga, Gb = OF.growth(dC64, B64.T, ra), OF.growth(A64.T, dC64, rb)
    kla = -(-N // OF.dims(ra)[1])
    klb = -(-M // OF.dims(rb)[1])
    from gpu_common import U_LEAF, max_terms
    t = max_terms(names)
    assert np.all(np.abs(dev_values(dA) - want_a) <= (U_LEAF["bf16x3"] + (kla + 2 * t + 8) * 2.0**-23) * Ga)
    assert np.all(np.abs(dev_values(dB) - want_b) <= (U_LEAF["bf16x3"] + (klb + 2 * t + 8) * 2.0**-23) * Gb)


def test_autograd_finite_differences(api):
    # loss = sum(G * (A B)) is bilinear, so central differences with any h
    # are exact in exact arithmetic; checked in float64 at M = K = N = 64.
    n = 64
    A = inputs.uniform((n, n), -1, 1, seed=61)
    B = inputs.uniform((n, n), -1, 1, seed=62)
    Gw = inputs.uniform((n, n), -1, 1, seed=63)
    plan = api.Plan(["strassen", "strassen"], "bf16x3")
    At = torch.from_numpy(A).float().cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).float().cuda().requires_grad_(True)
    out = api.fast_matmul(At, Bt, plan)
    (out * torch.from_numpy(Gw).float().cuda()).sum().backward()
    A64 = dev_values(At)
    B64 = dev_values(Bt)
    h = 1.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        i, j = rng.integers(0, n, 2)
        Ap, Am = A64.copy(), A64.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (np.sum(Gw * (Ap @ B64)) - np.sum(Gw * (Am @ B64))) / (2 * h)
        assert abs(dev_values(At.grad)[i, j] - fd) <= 1e-4 * (np.abs(Gw) @ np.abs(B64).T)[i, j]
        Bp, Bm = B64.copy(), B64.copy()
        Bp[i, j] += h
        Bm[i, j] -= h
        fd = (np.sum(Gw * (A64 @ Bp)) - np.sum(Gw * (A64 @ Bm))) / (2 * h)
        assert abs(dev_values(Bt.grad)[i, j] - fd) <= 1e-4 * (np.abs(A64).T @ np.abs(Gw))[i, j]


# ---------------------------------------------------------------- full size

def test_full_size_winograd_bf16x3_scaled(api):
    # The benchmark workload: n = 4096, FP32 A = D1 X D2, B = D3 Y D4,
    # Winograd one level, bf16x3 leaves, outside-inside scaling computed on
    # the GPU (its exponents checked bit-exact), every entry of C checked.
    n = 4096
    A, B = inputs.diag_scaled_pair(n, n, n, seed=1507 + 1000)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    eA, d, eB = api.scale(Ad, Bd, "OI")
    plan = api.Plan(["winograd"], "bf16x3")
    got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
    api.sync_status()
    st = OS.pow2_repeated(A64, B64, "OI")
    assert np.array_equal(eA.cpu().numpy(), st.eA) and np.array_equal(d.cpu().numpy(), st.d)
    assert np.array_equal(eB.cpu().numpy(), st.eB)
    C, G = oracle_reference(A64, B64, ["winograd"], st.eA, st.d, st.eB)
    assert_within(got, C, G, ["winograd"], n, "bf16x3", "full size")


@pytest.mark.parametrize("levels", [2, 3])
@pytest.mark.parametrize("steps", ["", "O", "OI"], ids=["none", "O", "OI"])
def test_full_size_winograd_deep_bf16x3(api, levels, steps):
    # The benchmark's workload at two and three Winograd levels: n = 4096,
    # FP32 A = D1 X D2, B = D3 Y D4, bf16 hi+lo leaves, no scaling, outside
    # scaling or outside-inside scaling computed on the GPU (exponents
    # bit-exact against the oracle), every entry of C within tolerance of
    # the oracle's exact fast product.
    n = 4096
    names = ["winograd"] * levels
    A, B = inputs.diag_scaled_pair(n, n, n, seed=1507 + 1000)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan(names, "bf16x3")
    if steps:
        eA, d, eB = api.scale(Ad, Bd, steps)
        got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
        api.sync_status()
        st = OS.pow2_repeated(A64, B64, steps)
        assert np.array_equal(eA.cpu().numpy(), st.eA) and np.array_equal(eB.cpu().numpy(), st.eB)
        assert np.array_equal(d.cpu().numpy(), st.d)
        C, G = oracle_reference(A64, B64, names, st.eA, st.d, st.eB)
    else:
        got = dev_values(api.multiply(plan, Ad, Bd))
        api.sync_status()
        C, G = oracle_reference(A64, B64, names)
    assert_within(got, C, G, names, n, "bf16x3", f"full size, Winograd L={levels}, scaling {steps or 'none'}")


# ---------------------------------------------------------------- failure path

@pytest.mark.parametrize("pairs", ["1", "0"], ids=["cta_pairs", "one_cta"])
def test_device_timeout_reported_without_fault(api, pairs):
    # FMM_TEST_STALL makes the multiply kernel's epilogue wait on a barrier
    # that nothing arrives at; its bounded wait (0.1 s here) must run out,
    # the kernel must stop every role, wait for its own copies and MMAs,
    # free its TMEM and report FMM_ERR_DEVICE_TIMEOUT through the status
    # word, and the context must stay usable.  Run in a child process so
    # the settings (read once per process) do not leak into other tests.
    code = r"""
import torch, sys, time
sys.path.insert(0, '.')
from paper_1507_00687_gb300 import api, _native
A = torch.ones((1024, 1024), device='cuda'); B = torch.ones((1024, 1024), device='cuda')
p = api.Plan(['strassen'], 'bf16x3')
t0 = time.time()
api.multiply(p, A, B)
try:
    api.sync_status()
    print('NO-TIMEOUT')
except _native.FmmError as e:
    print('CODE', e.code)
print('SECONDS', time.time() - t0)
x = (torch.ones(4, device='cuda') * 2).sum().item()
print('ALIVE', x)
"""
    env = dict(os.environ, FMM_WAIT_TIMEOUT_NS="100000000", FMM_TEST_STALL="1", FMM_TILE_PAIRS=pairs)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert "ALIVE 8.0" in r.stdout, r.stdout + r.stderr
    assert "CODE 8" in r.stdout, r.stdout + r.stderr


def test_cta_pair_kernel_matches_one_cta_kernel(api, tmp_path):
    # The CTA-pair multiply (256 x 256 tiles on two SMs) and the one-CTA
    # multiply (128 x 256 tiles) run the same leaf products with the same
    # K order per element; both must be within tolerance of the oracle and
    # of each other, under stored products and the fused epilogue, for the
    # forward and both gradient layouts.
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, '.'); sys.path.insert(0, 'tests')
from paper_1507_00687_gb300 import api, inputs
M, K, N = 1280, 1024, 1536
A = torch.from_numpy(inputs.uniform((M, K), -1, 1, seed=71)).float().cuda()
B = torch.from_numpy(inputs.uniform((K, N), -1, 1, seed=72)).float().cuda()
G = torch.from_numpy(inputs.uniform((M, N), -1, 1, seed=73)).float().cuda()
out = {}
for sched in ("pass_products", "pass_epilogue"):
    for leaf in ("bf16x3", "bf16"):
        p = api.Plan(["winograd"], leaf, sched)
        out[f"{sched}_{leaf}"] = api.multiply(p, A, B).cpu().numpy()
        dA, dB = api.multiply_backward(p, G, A, B)
        out[f"{sched}_{leaf}_dA"] = dA.cpu().numpy()
        out[f"{sched}_{leaf}_dB"] = dB.cpu().numpy()
api.sync_status()
np.savez(sys.argv[1], **out)
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for key, env in (("1", {"FMM_TILE_PAIRS": "1"}), ("0", {"FMM_TILE_PAIRS": "0"}),
                     ("unstreamed", {"FMM_COMBINE_STREAM": "0"})):
        f = str(tmp_path / f"c{key}.npz")
        r = subprocess.run([sys.executable, "-c", code, f], cwd=root, env=dict(os.environ, **env),
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        res[key] = dict(np.load(f))
    # the streamed combination pass does the arithmetic of the unrolled
    # one: the same values bit for bit
    for key in res["1"]:
        assert np.array_equal(res["1"][key], res["unstreamed"][key]), key
    M, K, N = 1280, 1024, 1536
    A = inputs.uniform((M, K), -1, 1, seed=71).astype(np.float32).astype(np.float64)
    B = inputs.uniform((K, N), -1, 1, seed=72).astype(np.float32).astype(np.float64)
    G = inputs.uniform((M, N), -1, 1, seed=73).astype(np.float32).astype(np.float64)
    C, Gr = oracle_reference(A, B, ["winograd"])
    for key in res["1"]:
        leaf = "bf16x3" if "bf16x3" in key else "bf16"
        if key.endswith("_dA") or key.endswith("_dB"):
            continue
        assert_within(res["1"][key], C, Gr, ["winograd"], K, leaf, "pairs " + key)
        assert_within(res["0"][key], C, Gr, ["winograd"], K, leaf, "one CTA " + key)
    # gradients: against the classical FP64 gradients with a norm-wise bound
    gA, gB = G @ B.T, A.T @ G
    for key in res["1"]:
        if key.endswith("_dA") or key.endswith("_dB"):
            ref = gA if key.endswith("_dA") else gB
            scale = np.abs(ref).max()
            tol = (2e-2 if "_bf16_" in key else 1e-3) * scale
            for pairs in ("1", "0"):
                assert np.abs(res[pairs][key] - ref).max() <= tol, (pairs, key)


@pytest.mark.parametrize("names", [["winograd"], ["strassen", "winograd"], ["winograd", "classical121"]],
                         ids=lambda n: "-".join(n))
@pytest.mark.parametrize("leaf", ["bf16x3", "bf16", "fp16"])
def test_accumulating_epilogue(api, names, leaf):
    # FMM_SCHEDULE_PASS_ACCUMULATE on CTA pairs: every (leaf, tile) unit adds
    # its unscaled W-weighted terms into C by atomic FP32 additions.  Scaled
    # inputs with ragged sizes (leaf blocks of at least 256 rows), two runs:
    # each within tolerance of the oracle's exact fast product (the
    # tolerance counts t_max roundings for the C sums in any order), and
    # integer inputs exact.
    M, K, N = 1290, 1100, 1170
    dt = "f16" if leaf == "fp16" else "f32"
    A, B = inputs.diag_scaled_pair(M, K, N, seed=77, span=4.0 if leaf == "fp16" else 12.0)
    Ad, Bd = to_dev(A, dt), to_dev(B, dt)
    A64, B64 = dev_values(Ad), dev_values(Bd)
    eA, d, eB = api.scale(Ad, Bd, "OI")
    st = OS.pow2_repeated(A64, B64, "OI")
    C, G = oracle_reference(A64, B64, names, st.eA, st.d, st.eB)
    plan = api.Plan(names, leaf, "pass_accumulate")
    runs = []
    for _ in range(2):
        got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
        api.sync_status()
        assert_within(got, C, G, names, K, leaf, f"accumulate {names} {leaf}")
        runs.append(got)
    Ai = inputs.integers((M, K), -4, 4, seed=5)
    Bi = inputs.integers((K, N), -4, 4, seed=6)
    got = dev_values(api.multiply(plan, to_dev(Ai, dt), to_dev(Bi, dt)))
    api.sync_status()
    assert np.array_equal(got, Ai @ Bi)


def test_overlapped_output_pass_bitwise(api, tmp_path):
    # A product large enough for the overlapped form (two multiply launches
    # over tile-row halves, the first half's output pass on a side stream)
    # gives the single launch's values bit for bit, forward and backward.
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, '.')
from paper_1507_00687_gb300 import api, inputs
M, K, N = 8192, 4096, 8192
A = torch.from_numpy(inputs.uniform((M, K), -1, 1, seed=81)).cuda().to(torch.bfloat16)
B = torch.from_numpy(inputs.uniform((K, N), -1, 1, seed=82)).cuda().to(torch.bfloat16)
p = api.Plan(["winograd"], "bf16")
C = api.multiply(p, A, B)
eA, d, eB = api.scale(A, B, "OI")
Cs = api.multiply(p, A, B, eA, d, eB)
api.sync_status()
np.savez(sys.argv[1], C=C.cpu().numpy(), Cs=Cs.cpu().numpy())
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for ov in ("1", "0"):
        f = str(tmp_path / f"o{ov}.npz")
        r = subprocess.run([sys.executable, "-c", code, f], cwd=root, env=dict(os.environ, FMM_OVERLAP=ov),
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        res[ov] = dict(np.load(f))
    for key in ("C", "Cs"):
        assert np.isfinite(res["1"][key]).all()
        assert np.array_equal(res["1"][key], res["0"][key]), key


# ---------------------------------------------------------------- schedules

def test_schedule_workspace_rules(api):
    # The pass schedule needs the combined operands in the workspace; given
    # only the load-stage workspace, a forced pass schedule reports
    # FMM_ERR_WORKSPACE while the automatic one runs the load-stage schedule.
    from paper_1507_00687_gb300 import _native as N
    M, K, N_ = 384, 320, 448
    A = inputs.uniform((M, K), -1, 1, seed=61)
    B = inputs.uniform((K, N_), -1, 1, seed=62)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    small = api.workspace_bytes(api.Plan(["winograd"], "bf16x3", "load_stage"), M, K, N_)
    big = api.workspace_bytes(api.Plan(["winograd"], "bf16x3", "pass"), M, K, N_)
    assert big > small
    ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    with pytest.raises(N.FmmError) as e:
        api.multiply(api.Plan(["winograd"], "bf16x3", "pass"), Ad, Bd, ws=ws)
    assert e.value.code == 6
    got = {s: dev_values(api.multiply(api.Plan(["winograd"], "bf16x3", s), Ad, Bd,
                                      ws=ws if s == "auto" else None)) for s in ("auto", "load_stage", "pass")}
    api.sync_status()
    C, G = oracle_reference(dev_values(Ad), dev_values(Bd), ["winograd"])
    for s, v in got.items():
        assert_within(v, C, G, ["winograd"], K, "bf16x3", s)
