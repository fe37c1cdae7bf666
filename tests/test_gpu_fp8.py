"""E4M3 leaves with power-of-two scales per 128-block along K against the
oracle: exact on small integers, the oracle's block quantization to within
FP32 accumulation, and the parity tolerance on real and scaled inputs."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_common import assert_within, dev_values, oracle_reference, oracle_tree, require_gpu, to_dev
from oracle import fmm as OF
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return require_gpu()


@pytest.mark.parametrize("names", [[], ["strassen"], ["winograd"], ["fast323"]], ids=lambda n: "-".join(n) or "classical")
@pytest.mark.parametrize("M,K,N", [(256, 256, 256), (300, 520, 250), (129, 65, 257)])
@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_e4m3_integers_exact(api, names, M, K, N, dt):
    # Entries in [-2, 2]: |S|, |T| <= 8 at one level, so every operand is an
    # integer of at most 4 significant bits, exact in E4M3 after any
    # power-of-two block scale; every product and sum is exact.
    A = inputs.integers((M, K), -2, 2, seed=M + 1)
    B = inputs.integers((K, N), -2, 2, seed=N + 2)
    got = dev_values(api.multiply(api.Plan(names, "e4m3b128"), to_dev(A, dt), to_dev(B, dt)))
    api.sync_status()
    assert np.array_equal(got, A @ B)


@pytest.mark.parametrize("names", [["winograd", "classical121", "winograd", "classical121"],
                                   ["strassen", "strassen", "strassen"],
                                   ["strassen", "strassen", "classical211", "classical211", "classical112"]],
                         ids=lambda n: "-".join(n))
def test_e4m3_deep_plans_integers_exact(api, names):
    # Many input blocks per operand (64 for B in the first plan): the
    # combination pass stages four rows per CTA; 16 x 8 = 128 C blocks in
    # the last: the output pass gathers per C block.  Entries in [-1, 1]: every
    # S, T entry is an integer of magnitude at most 16, exact in E4M3 after
    # its power-of-two block scale.
    M, K, N = 264, 520, 200
    A = inputs.integers((M, K), -1, 1, seed=3)
    B = inputs.integers((K, N), -1, 1, seed=4)
    for dt in ("f32", "bf16"):
        got = dev_values(api.multiply(api.Plan(names, "e4m3b128"), to_dev(A, dt), to_dev(B, dt)))
        api.sync_status()
        assert np.array_equal(got, A @ B), dt


def test_e4m3_many_input_blocks_integers_exact(api):
    # 16 x 16 input blocks per operand (Strassen, four levels) are more than
    # the E4M3 combination pass stages in shared memory: the unstaged form
    # reads each term's elements directly.  Entries in [-1, 1]: every S, T
    # entry is an integer of magnitude at most 16 (exact in E4M3).
    A = inputs.integers((256, 384), -1, 1, seed=1)
    B = inputs.integers((384, 320), -1, 1, seed=2)
    got = dev_values(api.multiply(api.Plan(["strassen"] * 4, "e4m3b128"), to_dev(A, "f32"), to_dev(B, "f32")))
    api.sync_status()
    assert np.array_equal(got, A @ B)


def test_e4m3_unstaged_combination_and_fold_kernel_match(api, tmp_path):
    # The unstaged combination (forced for every plan) must give the staged
    # kernel's E4M3 operands and scales exactly, so the products are equal
    # bit for bit; the folding multiply kernel (FMM_FP8_FOLD=1) must match
    # the oracle's block quantization as the block-scaled one does.  Child
    # processes: both settings are read once per process.
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, '.'); sys.path.insert(0, 'tests')
from paper_1507_00687_gb300 import api, inputs
A = torch.from_numpy(inputs.uniform((384, 640), -1, 1, seed=31)).float().cuda()
B = torch.from_numpy(inputs.uniform((640, 320), -1, 1, seed=32)).float().cuda()
A[:, :100] *= 2.0 ** -9
B[200:, :] *= 2.0 ** 7
out = {}
for names in (["strassen"], ["winograd", "classical121"]):
    out["-".join(names)] = api.multiply(api.Plan(names, "e4m3b128"), A, B).cpu().numpy()
api.sync_status()
np.savez(sys.argv[1], **out)
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for tag, extra in (("base", {}), ("direct", {"FMM_E4M3_DIRECT": "1"}), ("fold", {"FMM_FP8_FOLD": "1"})):
        path = str(tmp_path / f"{tag}.npz")
        r = subprocess.run([sys.executable, "-c", code, path], cwd=root, env=dict(os.environ, **extra),
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        res[tag] = dict(np.load(path))
    for k in res["base"]:
        assert np.array_equal(res["base"][k], res["direct"][k]), k
    A64 = inputs.uniform((384, 640), -1, 1, seed=31).astype(np.float32).astype(np.float64)
    B64 = inputs.uniform((640, 320), -1, 1, seed=32).astype(np.float32).astype(np.float64)
    A64[:, :100] *= 2.0 ** -9
    B64[200:, :] *= 2.0 ** 7
    emu = OF.fmm(A64, B64, oracle_tree(["strassen"]), leaf=OF.leaf_e4m3_b128, dtype=np.float32).astype(np.float64)
    _, G = oracle_reference(A64, B64, ["strassen"])
    for tag in ("base", "fold"):
        assert np.all(np.abs(res[tag]["strassen"] - emu) <= (320 + 16) * 2.0 ** -23 * G), tag


@pytest.mark.parametrize("names", [["strassen"], ["winograd"], []], ids=lambda n: "-".join(n) or "classical")
def test_e4m3_matches_block_quantization(api, names):
    # One level: S_r, T_r are formed in FP32 in index order on both sides and
    # quantized with the same 128-blocks and exponents, so the E4M3 operands
    # agree exactly; only the FP32 accumulation differs.
    M, K, N = 384, 640, 320
    A = inputs.uniform((M, K), -1, 1, seed=31)
    B = inputs.uniform((K, N), -1, 1, seed=32)
    A[:, :100] *= 2.0 ** -9  # blocks with very different ranges
    B[200:, :] *= 2.0 ** 7
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    got = dev_values(api.multiply(api.Plan(names, "e4m3b128"), Ad, Bd))
    api.sync_status()
    emu = OF.fmm(A64, B64, oracle_tree(names), leaf=OF.leaf_e4m3_b128, dtype=np.float32).astype(np.float64)
    _, G = oracle_reference(A64, B64, names)
    kl = K // (2 if names else 1)
    assert np.all(np.abs(got - emu) <= (kl + 16) * 2.0 ** -23 * G)


@pytest.mark.parametrize("names", [["strassen"], ["winograd"], ["strassen", "strassen"], ["winograd", "classical121"]],
                         ids=lambda n: "-".join(n))
@pytest.mark.parametrize("steps", ["", "OI"])
def test_e4m3_within_tolerance(api, names, steps):
    M, K, N = 512, 384, 448
    A, B = inputs.diag_scaled_pair(M, K, N, seed=41)
    Ad, Bd = to_dev(A, "f32"), to_dev(B, "f32")
    A64, B64 = dev_values(Ad), dev_values(Bd)
    plan = api.Plan(names, "e4m3b128")
    if steps:
        eA, d, eB = api.scale(Ad, Bd, steps)
        got = dev_values(api.multiply(plan, Ad, Bd, eA, d, eB))
        st = OS.pow2_repeated(A64, B64, steps)
        C, G = oracle_reference(A64, B64, names, st.eA, st.d, st.eB)
    else:
        got = dev_values(api.multiply(plan, Ad, Bd))
        C, G = oracle_reference(A64, B64, names)
    api.sync_status()
    assert_within(got, C, G, names, K, "e4m3b128", f"e4m3 {names} {steps}")


def test_e4m3_backward_and_refusals(api):
    from paper_1507_00687_gb300 import _native as N
    M, K, N_ = 256, 384, 320
    A = inputs.integers((M, K), -2, 2, seed=5)
    B = inputs.integers((K, N_), -2, 2, seed=6)
    G0 = inputs.integers((M, N_), -2, 2, seed=7)
    Ad, Bd, dC = to_dev(A, "bf16"), to_dev(B, "bf16"), to_dev(G0, "f32")
    dA, dB = api.multiply_backward(api.Plan(["strassen"], "e4m3b128"), dC, Ad, Bd)
    api.sync_status()
    assert np.array_equal(dev_values(dA), G0 @ B.T) and np.array_equal(dev_values(dB), A.T @ G0)
    with pytest.raises(N.FmmError) as e:
        api.multiply(api.Plan(["strassen"], "e4m3b128", "load_stage"), Ad, Bd)
    assert e.value.code == 10
