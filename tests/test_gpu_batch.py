"""Batched products (fmm_batch_create / fmm_batch_run): mixed shapes and
plans in one launch sequence, each product checked against the oracle within
the parity tolerance; CUDA-graph capture and replay on new inputs; the batch
against the single-product path."""
import numpy as np
import pytest
import torch

from gpu_common import assert_within, dev_values, oracle_reference, require_gpu, to_dev
from oracle import scaling as OS
from paper_1507_00687_gb300 import inputs

pytestmark = pytest.mark.gpu

MIX = [(["strassen"], 384, 256, 512), ([], 128, 640, 256), (["winograd"], 1000, 520, 776),
       (["winograd", "winograd"], 512, 384, 640), (["strassen", "classical121"], 300, 200, 250),
       (["fast323"], 450, 320, 390), (["winograd"], 129, 65, 257), (["strassen", "strassen"], 1024, 512, 768)]


@pytest.fixture(scope="module")
def api():
    return require_gpu()


def _problems(api, leaf, dt, seed):
    probs, host = [], []
    for i, (names, M, K, N) in enumerate(MIX):
        A, B = inputs.diag_scaled_pair(M, K, N, seed=seed + i)
        Ad, Bd = to_dev(A, dt), to_dev(B, dt)
        C = torch.full((M, N), float("nan"), device="cuda")
        probs.append((api.Plan(names, leaf), Ad, Bd, C))
        host.append(names)
    return probs, host


@pytest.mark.parametrize("steps", ["", "OI", "O", "I"])
def test_batch_matches_oracle(api, steps):
    probs, names = _problems(api, "bf16x3", "f32", 300)
    batch = api.Batch(probs, steps)
    batch.run()
    api.sync_status()
    for (plan, Ad, Bd, C), nm in zip(probs, names):
        A64, B64 = dev_values(Ad), dev_values(Bd)
        if steps:
            st = OS.pow2_repeated(A64, B64, steps)
            Cref, G = oracle_reference(A64, B64, nm, st.eA, st.d, st.eB)
        else:
            Cref, G = oracle_reference(A64, B64, nm)
        assert_within(dev_values(C), Cref, G, nm, Ad.shape[1], "bf16x3", f"batch {nm} {steps}")


def test_batch_bf16_leaves_and_integers_exact(api):
    # Integer entries in [-4, 4]: every leaf product is exact, so each batched
    # product equals the classical product bit for bit.
    probs = []
    for i, (names, M, K, N) in enumerate(MIX):
        A = inputs.integers((M, K), -4, 4, seed=40 + i)
        B = inputs.integers((K, N), -4, 4, seed=80 + i)
        probs.append((api.Plan(names, "bf16"), to_dev(A, "bf16"), to_dev(B, "bf16"),
                      torch.empty((M, N), device="cuda"), A @ B))
    batch = api.Batch([p[:4] for p in probs], "")
    batch.run()
    api.sync_status()
    for plan, Ad, Bd, C, want in probs:
        assert np.array_equal(dev_values(C), want)


def test_batch_cuda_graph_replay_on_new_inputs(api):
    probs, names = _problems(api, "bf16x3", "f32", 500)
    batch = api.Batch(probs, "OI")
    batch.run()  # first run outside the capture (library set-up happens here)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run()
    # new inputs into the same buffers, then replay
    for i, (plan, Ad, Bd, C) in enumerate(probs):
        A, B = inputs.diag_scaled_pair(Ad.shape[0], Ad.shape[1], Bd.shape[1], seed=900 + i)
        Ad.copy_(torch.from_numpy(A).float())
        Bd.copy_(torch.from_numpy(B).float())
        C.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    api.sync_status()
    for (plan, Ad, Bd, C), nm in zip(probs, names):
        A64, B64 = dev_values(Ad), dev_values(Bd)
        st = OS.pow2_repeated(A64, B64, "OI")
        Cref, G = oracle_reference(A64, B64, nm, st.eA, st.d, st.eB)
        assert_within(dev_values(C), Cref, G, nm, Ad.shape[1], "bf16x3", f"graph replay {nm}")


def test_batch_agrees_with_single_products(api):
    probs, names = _problems(api, "bf16x3", "f32", 700)
    batch = api.Batch(probs, "OI")
    batch.run()
    api.sync_status()
    for (plan, Ad, Bd, C), nm in zip(probs, names):
        eA, d, eB = api.scale(Ad, Bd, "OI")
        single = api.multiply(plan, Ad, Bd, eA, d, eB)
        _, G = oracle_reference(dev_values(Ad), dev_values(Bd), nm)
        A64, B64 = dev_values(Ad), dev_values(Bd)
        st = OS.pow2_repeated(A64, B64, "OI")
        _, G = oracle_reference(A64, B64, nm, st.eA, st.d, st.eB)
        assert_within(dev_values(C), dev_values(single), G, nm, Ad.shape[1], "bf16x3", f"batch vs single {nm}")


def test_batch_rejects_mixed_leaf_formats(api):
    from paper_1507_00687_gb300 import _native as N
    A = torch.ones((64, 64), device="cuda")
    with pytest.raises(N.FmmError):
        api.Batch([(api.Plan(["strassen"], "bf16"), A, A, torch.empty_like(A)),
                   (api.Plan(["strassen"], "bf16x3"), A, A, torch.empty_like(A))], "")


def test_autotuner_choices_run_and_respect_cutoff(api):
    tuner = api.Autotuner(leaf="bf16", sizes=(512, 1024), reps=2)
    assert tuner.table, "no candidate timed"
    for shape in ((512, 512, 512), (1024, 768, 1536), (384, 4096, 384)):
        names = tuner.choose(*shape)
        plan = tuner.plan(*shape)
        info = plan.info()
        if names:
            assert min(shape[0] // info["pm"], shape[1] // info["pk"], shape[2] // info["pn"]) >= tuner.cutoff
        A = (torch.rand(shape[:2], device="cuda") * 2 - 1).to(torch.bfloat16)
        B = (torch.rand(shape[1:], device="cuda") * 2 - 1).to(torch.bfloat16)
        got = dev_values(api.multiply(plan, A, B))
        C, G = oracle_reference(dev_values(A), dev_values(B), names)
        assert_within(got, C, G, names, shape[1], "bf16", f"autotuned {names}")
    # the accuracy axis: a cap on the relative instability keeps only the
    # candidates whose error bound is within that factor of the classical one
    for cap in (1.0, 3.0, 4.5, 1e9):
        names = tuner.choose(2048, 2048, 2048, max_instability=cap)
        assert not names or api.relative_instability(api.Plan(names, "bf16")) <= cap
    assert tuner.choose(2048, 2048, 2048, max_instability=1.0) == []


def test_batch_many_products_fused_epilogue(api):
    # Enough tiles to fill the GPU: the batch forms C in the multiply
    # epilogue (every tile of every product one unit, all leaves in order).
    # Eight copies of each product: identical results, within tolerance.
    base, names = _problems(api, "bf16x3", "f32", 1100)
    probs = []
    for copy in range(8):
        for plan, Ad, Bd, C in base:
            probs.append((plan, Ad, Bd, torch.full_like(C, float("nan"))))
    batch = api.Batch(probs, "OI")
    batch.run()
    api.sync_status()
    n = len(base)
    for i, ((plan, Ad, Bd, _), nm) in enumerate(zip(base, names)):
        A64, B64 = dev_values(Ad), dev_values(Bd)
        st = OS.pow2_repeated(A64, B64, "OI")
        Cref, G = oracle_reference(A64, B64, nm, st.eA, st.d, st.eB)
        first = dev_values(probs[i][3])
        assert_within(first, Cref, G, nm, Ad.shape[1], "bf16x3", f"fused batch {nm}")
        for copy in range(1, 8):
            assert np.array_equal(dev_values(probs[copy * n + i][3]), first)


def test_batch_with_trees_and_rotations(api):
    # Non-uniform plans and rotated rules in one batch with uniform ones:
    # each product within tolerance against the oracle's tree.
    import tree_cases as TC
    from oracle import fmm as OF
    from gpu_common import U_LEAF
    cases = [(TC.dalberto(), 300, 256, 280), (TC.mixed_rank(), 200, 128, 160), (["F_r1", []], 270, 390, 200),
             (["S", ["S"] * 7], 256, 256, 256)]
    probs, trees = [], []
    for i, (desc, M, K, N) in enumerate(cases):
        if desc[1]:
            lib, orc = TC.two_level(*desc)
            plan = api.Plan.tree(lib, "bf16x3")
        else:
            plan = api.Plan([TC.package_rule(desc[0])], "bf16x3")
            orc = OF.uniform([TC.oracle_rule(desc[0])])
        A, B = inputs.diag_scaled_pair(M, K, N, seed=700 + i, span=6.0)
        probs.append((plan, to_dev(A, "f32"), to_dev(B, "f32"), torch.full((M, N), float("nan"), device="cuda")))
        trees.append(orc)
    batch = api.Batch(probs, "OI")
    batch.run()
    api.sync_status()
    for (plan, Ad, Bd, C), orc in zip(probs, trees):
        A64, B64 = dev_values(Ad), dev_values(Bd)
        st = OS.pow2_repeated(A64, B64, "OI")
        Ap, Bp = OS.pow2_apply(A64, B64, st.eA, st.d, st.eB)
        Cref = OS.pow2_unscale(OF.fmm(Ap, Bp, orc), st.eA, st.eB)
        G = OS.pow2_unscale(OF.growth(Ap, Bp, orc), st.eA, st.eB)
        _, pk, _ = OF.dims(orc)
        kl = -(-Ad.shape[1] // pk)
        tol = (U_LEAF["bf16x3"] + (kl + 2 * TC.max_terms(orc) + 8) * 2.0**-23) * G
        assert np.all(np.abs(dev_values(C) - Cref) <= tol)


@pytest.mark.parametrize("dt,leaf", [("bf16", "bf16")])
def test_batch_classical_entries_read_inputs_directly(api, dt, leaf):
    # Classical entries with bf16 inputs and leaves are multiplied straight
    # from the caller's matrices (no scaling reductions, no conversion):
    # power-of-two scaling cancels exactly for the classical product, so
    # each result equals, bit for bit, the single-product path with the
    # batch's scaling applied (conversion, multiply, unscale) and without
    # it; ragged sizes included, beside a fast entry that is scaled.
    shapes = [(512, 640, 384), (1000, 520, 776), (129, 65, 257), (768, 1024, 512), (300, 2048, 256)]
    probs, refs = [], []
    for i, (M, K, N) in enumerate(shapes):
        A = inputs.uniform((M, K), -1, 1, seed=700 + i)
        B = inputs.uniform((K, N), -1, 1, seed=800 + i)
        Ad, Bd = to_dev(A, dt), to_dev(B, dt)
        probs.append((api.Plan([], leaf), Ad, Bd, torch.full((M, N), float("nan"), device="cuda")))
    # a fast entry alongside (scaled through the reductions and combination)
    A, B = inputs.diag_scaled_pair(640, 512, 768, seed=950, span=4.0)
    probs.append((api.Plan(["winograd"], leaf), to_dev(A, dt), to_dev(B, dt),
                  torch.full((640, 768), float("nan"), device="cuda")))
    batch = api.Batch(probs, "OI")
    batch.run()
    api.sync_status()
    for plan, Ad, Bd, C in probs[:-1]:
        eA, d, eB = api.scale(Ad, Bd, "OI")
        scaled = api.multiply(plan, Ad, Bd, eA, d, eB)
        plain = api.multiply(plan, Ad, Bd)
        api.sync_status()
        assert np.array_equal(dev_values(C), dev_values(scaled)), tuple(Ad.shape)
        assert np.array_equal(dev_values(C), dev_values(plain)), tuple(Ad.shape)
    plan, Ad, Bd, C = probs[-1]
    A64, B64 = dev_values(Ad), dev_values(Bd)
    st = OS.pow2_repeated(A64, B64, "OI")
    Cref, G = oracle_reference(A64, B64, ["winograd"], st.eA, st.d, st.eB)
    assert_within(dev_values(C), Cref, G, ["winograd"], 512, leaf, "fast entry beside direct ones")


def test_batch_direct_entries_write_only_their_c(api):
    # Direct classical entries write C by bulk tensor stores clipped at C's
    # edges: with C a column slice of a wider row-major buffer (ldc > N) and
    # ragged M, N, the columns beyond N and the rows beyond M of the buffer
    # keep their contents, and C equals the single-product result bit for bit.
    shapes = [(1000, 520, 776), (300, 2048, 264), (777, 384, 520)]
    probs, bufs = [], []
    for i, (M, K, N) in enumerate(shapes):
        A = to_dev(inputs.uniform((M, K), -1, 1, seed=900 + i), "bf16")
        B = to_dev(inputs.uniform((K, N), -1, 1, seed=910 + i), "bf16")
        buf = torch.full((M + 40, N + 72), float("nan"), device="cuda")
        probs.append((api.Plan([], "bf16"), A, B, buf[:M, :N]))
        bufs.append(buf)
    batch = api.Batch(probs, "OI")
    batch.run()
    api.sync_status()
    for (plan, A, B, C), buf in zip(probs, bufs):
        M, N = C.shape
        want = api.multiply(plan, A, B)
        api.sync_status()
        assert np.array_equal(dev_values(C), dev_values(want)), (M, N)
        rest = dev_values(buf)
        assert np.isnan(rest[:, N:]).all() and np.isnan(rest[M:, :]).all(), (M, N)
