"""The stabilisation stacks' decomposition X diag(e^c) = Q diag(e^d) V
(qmc_udv) against its definition, on random matrices, on column-graded ones
(scales e^-120 .. e^120 in X itself) and with column log scales passed as
log_scale, shifted far beyond FP64's exponent range (the stacks carry their D
this way, since the slice products' singular values grow like
e^{c beta u} and leave FP64's range at large beta times coupling).

For n <= 128 the columns are ordered by log |x_j| + c_j once and factored by
blocked Householder QR over a cluster of CTAs; the column-pivoted one-CTA
kernel (QMC_QR_CS=1, run in a fresh process) must satisfy the same
definition.  Each column of X is reproduced to FP64 rounding relative to
that column, Q is unitary to rounding, and V = D^-1 R P^T stays bounded.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _udv(qmc, X, lsc=None):
    import torch
    b, n, _ = X.shape
    Xt = torch.tensor(np.ascontiguousarray(X), dtype=torch.complex128, device="cuda").contiguous()
    Qt = torch.full((b, n, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    Vt = torch.full((b, n, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    Dt = torch.full((b, n), np.nan, dtype=torch.float64, device="cuda")
    Lt = None if lsc is None else torch.tensor(np.ascontiguousarray(lsc), dtype=torch.float64,
                                                device="cuda").contiguous()
    qmc.qmc_udv(n, b, Xt.data_ptr(), Qt.data_ptr(), Dt.data_ptr(), Vt.data_ptr(),
                0 if Lt is None else Lt.data_ptr())
    return Qt.cpu().numpy(), Dt.cpu().numpy(), Vt.cpu().numpy()


def _inputs(n, b, graded, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(b, n, n)) + 1j * rng.normal(size=(b, n, n))
    if graded:
        X = X * np.exp(rng.uniform(-120, 120, size=(b, 1, n)))
    return X


def _check(X, Q, d, V, c=None):
    b, n, _ = X.shape
    c = np.zeros((b, n)) if c is None else c
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(V)) and np.all(np.isfinite(d))
    un = np.abs(np.conj(np.swapaxes(Q, 1, 2)) @ Q - np.eye(n)).max()
    assert un < 1e-13, un
    assert np.abs(V).max() < 1e3  # bounded by the ordering
    # X_j = sum_i Q_i V_ij e^{d_i - c_j}, each factor formed in log space
    with np.errstate(divide="ignore"):
        lv = np.log(np.abs(V))
    W = np.where(V != 0, np.exp(np.minimum(lv + d[:, :, None] - c[:, None, :], 700.0)) *
                 np.exp(1j * np.angle(V)), 0)
    Y = Q @ W
    colerr = (np.abs(Y - X).max(1) / np.abs(X).max(1)).max()
    assert colerr < 1e-12, colerr


@pytest.mark.parametrize("n", [2, 10, 36, 72, 120, 280])
@pytest.mark.parametrize("graded", [False, True])
def test_udv_reproduces_x(qmc, n, graded):
    X = _inputs(n, 8 if n <= 120 else 2, graded, n + 7 * graded)
    _check(X, *_udv(qmc, X))


@pytest.mark.parametrize("n", [10, 72, 120, 280])
def test_udv_with_log_scales_beyond_fp64(qmc, n):
    """Column log scales c (spread over e^-300 .. e^300, where X diag(e^c)
    is still representable) reproduce the scaled columns; shifting every c
    by 2500 (far beyond FP64's range) leaves Q bit for bit and V to rounding, and shifts
    log D by exactly the same amount: the decomposition never forms the
    scaled matrix.  V's entries carry e^{c_j - c_i} formed from the shifted
    scales, so they move by the rounding of that difference (2500 * 2^-52
    absolute in the exponent): 1e-11 relative."""
    b = 4 if n <= 120 else 2
    X = _inputs(n, b, False, 100 + n)
    c = np.random.default_rng(n).uniform(-300, 300, size=(b, n))
    Q, d, V = _udv(qmc, X, c)
    _check(X, Q, d, V, c)
    Q2, d2, V2 = _udv(qmc, X, c + 2500.0)
    assert np.array_equal(Q2, Q)
    assert np.all(np.abs(V2 - V) <= 1e-11 * np.abs(V) + 1e-300)
    assert np.abs(d2 - d - 2500.0).max() < 1e-9


RUN = """
import sys, numpy as np, torch
sys.path.insert(0, '.')
from paper_2605_03700_gb300 import build
build.build()
import paper_2605_03700_gb300 as P
from tests.test_gpu_udv import _inputs, _udv
X = _inputs(int(sys.argv[1]), 8, True, 3)
c = np.random.default_rng(5).uniform(-180, 180, size=(8, int(sys.argv[1])))
Q, D, V = _udv(P, X, c)
np.savez(sys.argv[2], Q=Q, D=D, V=V, c=c)
"""


def test_blocked_and_pivoted_kernels_agree(tmp_path):
    """Both kernels factor the same graded, log-scaled matrices to the
    definition.  The column scales log |x_j| + c_j span e^-300 .. e^300 here:
    V = D^-1 R holds ratios of column scales, so once their spread passes
    FP64's range (e^~744) entries of V underflow and the smallest columns are
    reproduced only relative to the largest ones, not to themselves."""
    for cs in (1, 4):
        path = str(tmp_path / f"udv{cs}.npz")
        r = subprocess.run([sys.executable, "-c", RUN, "72", path], cwd=ROOT, capture_output=True,
                           text=True, timeout=600, env=dict(os.environ, QMC_QR_CS=str(cs)))
        assert r.returncode == 0, r.stderr[-3000:]
        out = np.load(path)
        X = _inputs(72, 8, True, 3)
        _check(X, out["Q"], out["D"], out["V"], out["c"])
