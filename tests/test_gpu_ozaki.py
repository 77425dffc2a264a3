"""FP64 products on the tensor cores by error-free splitting (the fitting net's first layer).

Against the FP64 host product: integer matrices (exact products, sums
below 2^53) must come out exactly; random matrices within a few units of
FP64 rounding of K max|a| max|b|; rows spanning many orders of magnitude
keep their relative accuracy against their own scale.  A wrong digit
weight, a dropped diagonal or a mis-staged K chunk fails by many orders
of magnitude.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2005_00223_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def model(dp):
    import dpsynth
    return dp.Model(dpsynth.copper_student_config(), 0)


def _run(dp, model, A, Bt):
    import torch
    dA = torch.tensor(A, device="cuda")
    dB = torch.tensor(Bt, device="cuda")
    dC = torch.empty((A.shape[0], Bt.shape[0]), dtype=torch.float64, device="cuda")
    dp.dp_ozaki_dgemm_dev(model.h, dA, dB, dC)
    return dC.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(300, 240, 1600), (129, 1600, 240), (128, 64, 48), (5, 48, 320), (131, 48, 1808)])
def test_integer_matrices_exact(dp, model, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-3000, 3001, size=(M, K)).astype(np.float64)
    Bt = rng.integers(-3000, 3001, size=(N, K)).astype(np.float64)
    C = _run(dp, model, A, Bt)
    ref = (A.astype(np.int64) @ Bt.astype(np.int64).T).astype(np.float64)
    np.testing.assert_array_equal(C, ref)


@pytest.mark.parametrize("M,N,K", [(300, 240, 1600), (257, 1600, 240)])
def test_random_matrices_fp64_accuracy(dp, model, M, N, K):
    rng = np.random.default_rng(7)
    A = rng.normal(size=(M, K))
    Bt = rng.normal(size=(N, K))
    C = _run(dp, model, A, Bt)
    ref = A @ Bt.T
    scale = K * np.abs(A).max(1)[:, None] * np.abs(Bt).max(1)[None, :]
    err = np.abs(C - ref) / scale
    assert err.max() < 4 * 2.0 ** -53, err.max()
    # and against the exact product of a few entries (rational arithmetic)
    from fractions import Fraction
    for (r, c) in [(0, 0), (M - 1, N - 1), (M // 2, N // 3)]:
        ex = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[r], Bt[c]))
        assert abs(Fraction(float(C[r, c])) - ex) <= Fraction(2.0 ** -50) * Fraction(float(scale[r, c]))


def test_rows_of_different_magnitudes(dp, model):
    rng = np.random.default_rng(3)
    M, N, K = 256, 240, 1600
    A = rng.normal(size=(M, K)) * 10.0 ** rng.uniform(-30, 30, size=(M, 1))
    Bt = rng.normal(size=(N, K)) * 10.0 ** rng.uniform(-30, 30, size=(N, 1))
    A[7] = 0.0                       # an all-zero row
    C = _run(dp, model, A, Bt)
    ref = A @ Bt.T
    scale = K * np.abs(A).max(1)[:, None] * np.abs(Bt).max(1)[None, :]
    scale[7] = 1.0
    assert (np.abs(C - ref) / scale).max() < 4 * 2.0 ** -53
    assert (C[7] == 0).all()
