"""Pins for the oracle's rounding emulation against IEEE / OCP definitions
(hand-computed ties) and independent library conversions, and for the
E4M3 leaf with 128-block power-of-two scales (exactness on small integers,
the per-entry error bound, the UE8M0 scale floor, the quantization axes)."""
import numpy as np
import pytest
import torch

from oracle import precision as P


def test_bf16_ties_to_even():
    x = np.array([1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-8), 1 + 2**-8 + 2**-20, 0.0])
    assert list(P.round_to(x, "bf16")) == [1.0, 1 + 2**-6, -1.0, 1 + 2**-7, 0.0]


def test_fp16_range_and_subnormals():
    x = np.array([65504.0, 65520.0, 2.0**-24, 2.0**-25, 3 * 2.0**-25])
    r = P.round_to(x, "fp16")
    assert r[0] == 65504.0 and np.isinf(r[1])
    assert r[2] == 2.0**-24 and r[3] == 0.0 and r[4] == 2.0**-23


@pytest.mark.parametrize("fmt,tdtype", [("bf16", torch.bfloat16), ("fp16", torch.float16)])
def test_matches_library_conversion(fmt, tdtype):
    g = np.random.default_rng(7)
    x = np.concatenate([g.normal(size=4000) * 10.0 ** g.integers(-6, 6, size=4000),
                        g.uniform(-1, 1, size=1000)]).astype(np.float32).astype(np.float64)
    if fmt == "fp16":
        x = x[np.abs(x) < 60000]
    want = torch.from_numpy(x).to(torch.float32).to(tdtype).to(torch.float64).numpy()
    assert np.array_equal(P.round_to(x, fmt), want)


def test_e4m3_matches_library_in_range():
    g = np.random.default_rng(8)
    x = g.uniform(-440, 440, size=3000) * 2.0 ** g.integers(-10, 0, size=3000)
    want = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(P.round_to(x, "e4m3"), want)
    assert P.round_to(np.array([1000.0]), "e4m3")[0] == 448.0


def test_split_bf16():
    g = np.random.default_rng(9)
    x = g.uniform(-1, 1, size=10000).astype(np.float32).astype(np.float64)
    hi, lo = P.split_bf16(x)
    assert np.array_equal(hi, P.round_to(hi, "bf16")) and np.array_equal(lo, P.round_to(lo, "bf16"))
    assert np.all(np.abs(x - hi - lo) <= 2.0**-16 * np.abs(x))
    assert np.all(np.abs(lo) <= 2.0**-8 * np.abs(x))


# ---------------------------------------------------------------- E4M3 with 128-blocks

def test_e4m3_blocks_exact_on_small_integers_and_scale_invariant():
    from oracle import fmm as F
    rng = np.random.default_rng(11)
    X = rng.integers(-15, 16, size=(7, 300)).astype(np.float64)
    q, s = F.quantize_e4m3_blocks(X, axis=1)
    assert np.array_equal(q, X)  # every integer of magnitude <= 15 has 4 significant bits
    # scaling a block by a power of two scales its representation exactly
    Y = X.copy()
    Y[:, 128:256] *= 2.0 ** 37
    qy, sy = F.quantize_e4m3_blocks(Y, axis=1)
    assert np.array_equal(qy[:, 128:256], q[:, 128:256] * 2.0 ** 37)
    assert np.array_equal(sy[:, 1] - s[:, 1], np.full(7, 37)) or np.all(X[:, 128:256] == 0)
    # columns (axis 0) are the transpose
    qc, sc = F.quantize_e4m3_blocks(X.T, axis=0)
    assert np.array_equal(qc, X.T) and np.array_equal(sc, s.T)


def test_e4m3_blocks_error_bound():
    # Relative error <= 2^-4 for entries within 2^-6 of... every entry whose
    # scaled magnitude is a normal E4M3 number (>= 2^-6); smaller entries have
    # absolute error <= 2^-10 times the block scale (half the subnormal step).
    from oracle import fmm as F
    rng = np.random.default_rng(12)
    X = rng.standard_normal((5, 384)) * np.exp2(rng.integers(-30, 30, size=(5, 1)))
    X[:, 7] *= 2.0 ** -20  # a tiny entry inside a block
    q, s = F.quantize_e4m3_blocks(X, axis=1)
    f = np.repeat(np.exp2(s.astype(np.float64)), 128, axis=1)[:, :384]
    scaled = np.abs(X) / f
    assert np.all(scaled < 256)
    normal = scaled >= 2.0 ** -6
    assert np.all(np.abs(q - X)[normal] <= 2.0 ** -4 * np.abs(X)[normal])
    assert np.all((np.abs(q - X) / f)[~normal] <= 2.0 ** -10)
    # each block's largest magnitude scales into [128, 256)
    for b in range(3):
        m = (np.abs(X[:, b * 128:(b + 1) * 128]) / f[:, b * 128:b * 128 + 1]).max(axis=1)
        assert np.all((m >= 128) & (m < 256))


def test_e4m3_block_scale_floor_is_the_ue8m0_minimum():
    # Block scales are UE8M0 numbers, 2^-127 at the least: a block whose
    # largest magnitude is 2^-125 (frexp exponent -124, so s would be -132)
    # takes s = -127 and is held as 4 = 2^-125 * 2^127; its entry 2^-137
    # scales to 2^-10, half the smallest E4M3 subnormal (2^-9), and rounds to
    # zero (ties to even), where s = -132 would have kept it exactly (2^-5).
    # A block just above the floor (largest magnitude 2^-119, s = -126) is
    # unaffected.
    from oracle import fmm as F
    X = np.zeros((2, 128))
    X[0, 0], X[0, 1], X[0, 2] = 2.0 ** -125, 2.0 ** -137, 3 * 2.0 ** -131
    X[1, 0], X[1, 1] = 2.0 ** -119, 2.0 ** -126
    q, s = F.quantize_e4m3_blocks(X, axis=1)
    assert s[0, 0] == -127 and s[1, 0] == -126
    assert q[0, 0] == 2.0 ** -125 and q[0, 1] == 0.0 and q[0, 2] == 3 * 2.0 ** -131
    assert q[1, 0] == 2.0 ** -119 and q[1, 1] == 2.0 ** -126


def test_e4m3_leaf_scales_rows_of_s_and_columns_of_t():
    # The E4M3 leaf quantizes S (rows x K) in 128-blocks along K per row and
    # T (K x cols) per column.  Rows and columns at very different scales
    # then keep their relative accuracy: each scaled entry is a normal E4M3
    # number, so |fl(s) fl(t) - s t| <= (2 * 2^-4 + 2^-8) |s t| entrywise.
    # Had S been quantized along its columns (T along its rows), the rows at
    # 2^-30 and 2^-50 would share a scale with the row at 2^10 and vanish.
    from oracle import fmm as F
    g = np.random.default_rng(13)
    S = g.uniform(1, 2, (4, 256)) * np.exp2(np.array([0.0, -30.0, 10.0, -50.0]))[:, None]
    T = g.uniform(1, 2, (256, 3)) * np.exp2(np.array([0.0, -40.0, 20.0]))[None, :]
    C = F.leaf_e4m3_b128(S, T)
    exact = S @ T
    assert np.all(np.abs(C - exact) <= (2 * 2.0 ** -4 + 2.0 ** -8) * exact)
    # the same leaf inside one Strassen level on small integers is exact
    A = g.integers(-3, 4, (256, 512)).astype(np.float64)
    B = g.integers(-3, 4, (512, 128)).astype(np.float64)
    from oracle import rules as R
    assert np.array_equal(F.fmm(A, B, F.uniform([R.strassen()]), leaf=F.leaf_e4m3_b128), A @ B)


def test_e4m3_block_quantization_by_hand():
    # One block [200, 1.25 * 2^-9]: its max 200 has frexp exponent 8, so
    # s = 0 and the entries are rounded on the E4M3 grid itself: 200 lies
    # midway between 192 and 208 and goes to the even significand (192);
    # 1.25 * 2^-9 is a subnormal multiple of 2^-9 and goes to 2^-9.
    from oracle import fmm as F
    q, s = F.quantize_e4m3_blocks(np.array([[200.0, 1.25 * 2.0 ** -9]]), axis=1)
    assert s.tolist() == [[0]] and q.tolist() == [[192.0, 2.0 ** -9]]


def test_non_finite_values_pass_through():
    x = np.array([np.inf, -np.inf, np.nan, 1.0])
    for fmt in ("bf16", "fp16", "fp32"):
        r = P.round_to(x, fmt)
        assert r[0] == np.inf and r[1] == -np.inf and np.isnan(r[2]) and r[3] == 1.0


def test_e4m3_block_max_is_by_magnitude_and_saturation():
    # The block scale follows the largest magnitude, here a negative entry:
    # -200 gives s = 0 and rounds to -192 (a tie, even significand).
    from oracle import fmm as F
    q, s = F.quantize_e4m3_blocks(np.array([[-200.0, 1.0]]), axis=1)
    assert s.tolist() == [[0]] and q.tolist() == [[-192.0, 1.0]]
    # overflow: infinity by default, the largest finite value when saturating
    big = float.fromhex("0x1.fep127")
    assert P.round_to(np.array([1e39]), "bf16")[0] == np.inf
    assert P.round_to(np.array([1e39, -1e39]), "bf16", saturate=True).tolist() == [big, -big]
    assert P.round_to(np.array([7e4]), "fp16", saturate=True)[0] == 65504.0
