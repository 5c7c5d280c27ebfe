"""The batched complex product on the tcgen05 tensor cores (qmc_cgemm,
digits > 0) against numpy's FP64 product.

The digit split is error-free per digit and the FP32 accumulation exact
while partial sums stay below 2^24, so with 7 digits the error is bounded by
the dropped digit pairs and the 55-bit fixed point: a few 1e-14 of
(|op A| |d| |op B|)_ij (tolerance 2e-13 here); with 3 digits it is FP32
class (tolerance 2e-6).  Matrices of small integers are reproduced exactly,
which pins the exact accumulation.  The CUDA-core path (digits = 0) is
checked at the same time.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _run(qmc, A, B, d, opA, opB, digits, negate=0, addI=0):
    import torch
    batch = A.shape[0]
    M = A.shape[1] if opA == 0 else A.shape[2]
    K = A.shape[2] if opA == 0 else A.shape[1]
    N = B.shape[2] if opB == 0 else B.shape[1]
    At = torch.tensor(A, dtype=torch.complex128, device="cuda")
    Bt = torch.tensor(B, dtype=torch.complex128, device="cuda")
    dt = torch.tensor(d, dtype=torch.complex128, device="cuda") if d is not None else None
    Ct = torch.full((batch, M, N), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    qmc.qmc_cgemm(M, N, K, batch, At.data_ptr(), opA, Bt.data_ptr(), opB,
                  dt.data_ptr() if dt is not None else 0, Ct.data_ptr(), negate, addI, digits)
    return Ct.cpu().numpy()


def _ref(A, B, d, opA, opB, negate=0, addI=0):
    oA = A if opA == 0 else np.conj(np.swapaxes(A, 1, 2))
    oB = B if opB == 0 else np.conj(np.swapaxes(B, 1, 2))
    dB = oB * d[:, :, None] if d is not None else oB
    C = oA @ dB
    bound = np.abs(oA) @ np.abs(dB)
    if negate:
        C = -C
    if addI:
        C = C + np.eye(C.shape[1])
    return C, bound


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("M,N,K,batch", [(72, 72, 72, 3), (36, 36, 36, 5), (5, 7, 9, 2),
                                         (120, 120, 120, 2), (130, 40, 72, 2), (280, 56, 16, 1),
                                         (72, 72, 72, 720)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (2, 0), (0, 2)])
def test_products_match_fp64(qmc, M, N, K, batch, opA, opB):
    rng = np.random.default_rng(M * 1000 + N * 10 + K + 7 * opA + 3 * opB)
    A = _rand(rng, batch, M, K) if opA == 0 else _rand(rng, batch, K, M)
    B = _rand(rng, batch, K, N) if opB == 0 else _rand(rng, batch, N, K)
    d = np.exp(1j * rng.uniform(0, 6.3, size=(batch, K))) * rng.uniform(0.5, 2, size=(batch, K))
    for dd in (None, d):
        ref, bound = _ref(A, B, dd, opA, opB)
        for digits, tol in ((7, 2e-13), (3, 2e-6), (0, 1e-13)):
            C = _run(qmc, A, B, dd, opA, opB, digits)
            err = np.abs(C - ref) / bound
            assert np.all(np.isfinite(C)), digits
            assert err.max() < tol, (digits, err.max())


def test_negate_and_identity(qmc):
    rng = np.random.default_rng(3)
    A, B = _rand(rng, 2, 72, 72), _rand(rng, 2, 72, 72)
    for neg, addI in ((1, 0), (0, 1), (1, 1)):
        ref, bound = _ref(A, B, None, 0, 0, neg, addI)
        C = _run(qmc, A, B, None, 0, 0, 7, neg, addI)
        assert (np.abs(C - ref) / (bound + 1)).max() < 2e-13


def test_small_integer_matrices_exact(qmc):
    """Entries are integers below 2^7 in modulus: every digit but the
    leading one is zero and all partial sums are exact in FP32, so the
    product is exact."""
    rng = np.random.default_rng(11)
    for (M, N, K) in ((72, 72, 72), (120, 120, 120), (33, 17, 65)):
        A = rng.integers(-127, 128, size=(2, M, K)) + 1j * rng.integers(-127, 128, size=(2, M, K))
        B = rng.integers(-127, 128, size=(2, K, N)) + 1j * rng.integers(-127, 128, size=(2, K, N))
        C = _run(qmc, A, B, None, 0, 0, 7)
        assert np.array_equal(C, A @ B)


def test_graded_rows_and_columns(qmc):
    """Row scales of A and column scales of B spanning 2^-250 .. 2^250 (the
    products stay inside the FP64 range): each output stays within the error
    bound of its own row and column."""
    rng = np.random.default_rng(5)
    M = N = K = 72
    A = _rand(rng, 1, M, K) * np.exp2(rng.integers(-250, 250, size=(1, M, 1)))
    B = _rand(rng, 1, K, N) * np.exp2(rng.integers(-250, 250, size=(1, 1, N)))
    ref, bound = _ref(A, B, None, 0, 0)
    C = _run(qmc, A, B, None, 0, 0, 7)
    assert (np.abs(C - ref) / bound).max() < 2e-13


def test_nan_rows_and_columns_propagate(qmc):
    rng = np.random.default_rng(9)
    A, B = _rand(rng, 1, 40, 40), _rand(rng, 1, 40, 40)
    A[0, 3, 5] = np.nan
    B[0, 7, 11] = np.inf
    C = _run(qmc, A, B, None, 0, 0, 7)
    assert np.all(np.isnan(C[0, 3, :])) and np.all(np.isnan(C[0, :, 11]))
    ok = np.ones((40, 40), bool)
    ok[3, :] = False
    ok[:, 11] = False
    ref, bound = _ref(np.nan_to_num(A), np.nan_to_num(B), None, 0, 0)
    assert (np.abs(C[0][ok] - ref[0][ok]) / bound[0][ok]).max() < 2e-13
