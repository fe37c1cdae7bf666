"""The seeded input generators follow the input definitions they state.

Pinned against: the three test distributions of Sec. 6.5 (which blocks of
A and B are shrunk or grown, by n^-2 or n^2, with the 1-based index
conditions read on 0-based arrays), the benchmark pair A = D1 X D2,
B = D3 Y D4 (the diagonal factors cancel in every cross ratio, lie in
[2^-span, 2^span) and are exact powers of two with integer exponents), and
the log-uniform batch dimensions.
"""
import numpy as np
import pytest

from paper_1507_00687_gb300 import inputs


@pytest.mark.parametrize("n", [64, 65])
def test_paper_distributions_follow_sec_6_5(n):
    one = 1.0 / n**2
    A1, B1 = inputs.paper_distribution(1, n, seed=5)
    assert A1.min() >= 0 and A1.max() < 1 and B1.min() >= 0 and B1.max() < 1
    # 1-based i < n/2 is rows 0 .. ceil(n/2) - 2; j > n/2 is columns floor(n/2) .. n-1
    lo = [i for i in range(n) if i + 1 < n / 2]
    hi = [j for j in range(n) if j + 1 > n / 2]
    rest_lo = [i for i in range(n) if i not in lo]
    rest_hi = [j for j in range(n) if j not in hi]
    A2, B2 = inputs.paper_distribution(2, n, seed=5)
    # the same uniform draws, shrunk where the definition says
    assert np.array_equal(A2[:, rest_hi], A1[:, rest_hi]) and np.allclose(A2[:, hi], A1[:, hi] * one)
    assert np.array_equal(B2[rest_lo, :], B1[rest_lo, :]) and np.allclose(B2[lo, :], B1[lo, :] * one)
    assert A2[:, hi].max() < one and B2[lo, :].max() < one
    A3, B3 = inputs.paper_distribution(3, n, seed=5)
    grown = np.zeros((n, n), bool)
    grown[np.ix_(lo, hi)] = True
    assert np.allclose(A3[grown], A1[grown] * n**2) and np.array_equal(A3[~grown], A1[~grown])
    assert np.allclose(B3[:, lo], B1[:, lo] * one) and np.array_equal(B3[:, rest_lo], B1[:, rest_lo])
    # the index reading: with n even, row n/2 - 1 (1-based n/2) is not "< n/2"
    if n % 2 == 0:
        assert n // 2 - 1 not in lo and n // 2 in hi and n // 2 - 1 not in hi
    with pytest.raises(ValueError):
        inputs.paper_distribution(4, n, seed=5)


def test_benchmark_pair_is_diagonally_scaled():
    M, K, N = 48, 40, 56
    X, Y = inputs.diag_scaled_pair(M, K, N, seed=11, span=0.0)   # D = I: the uniform factors
    assert X.min() >= 0 and X.max() < 1 and Y.min() >= 0 and Y.max() < 1
    for integer in (False, True):
        A, B = inputs.diag_scaled_pair(M, K, N, seed=11, integer_exponents=integer)
        for P, Q in ((A, X), (B, Y)):
            # P = D Q D': the ratio P / Q is the outer product d_i d'_j
            R = np.log2(P / Q)
            assert np.allclose(R - R[:, :1] - R[:1, :] + R[0, 0], 0, atol=1e-9)
            # each factor lies in [2^-12, 2^12), so their product in [2^-24, 2^24)
            assert R.min() >= -24 - 1e-9 and R.max() < 24
            if integer:
                assert np.allclose(R, np.round(R), atol=1e-9)   # exact powers of two
            else:
                assert np.abs(R - np.round(R)).max() > 1e-3     # not powers of two


def test_log_uniform_dims():
    d = inputs.log_uniform_dims(4000, 512, 4096, 128, seed=3)
    assert d.shape == (4000, 3) and d.dtype == np.int64
    assert np.all(d % 128 == 0) and d.min() >= 512 and d.max() <= 4096
    # log-uniform: the median is near the geometric mean of the range
    med = float(np.median(d))
    assert abs(np.log(med) - 0.5 * (np.log(512) + np.log(4096))) < 0.1
    # the same seed draws the same batch
    assert np.array_equal(d, inputs.log_uniform_dims(4000, 512, 4096, 128, seed=3))
