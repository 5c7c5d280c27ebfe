"""The stabilisation stacks' decomposition X = Q diag(D) V (qmc_udv) against
its definition, on random and on column-graded matrices (the graded products
of the UDV chain: column scales spanning e^-120 .. e^120).

For n <= 128 the columns are ordered by 2-norm once and factored by blocked
Householder QR over a cluster of CTAs; the column-pivoted one-CTA kernel
(QMC_QR_CS=1, run in a fresh process) must agree with it on X and Q^H Q.
Each column of X is reproduced to FP64 rounding relative to that column.
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


def _udv(qmc, X):
    import torch
    b, n, _ = X.shape
    Xt = torch.tensor(np.ascontiguousarray(X), dtype=torch.complex128, device="cuda").contiguous()
    Qt = torch.full((b, n, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    Vt = torch.full((b, n, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    Dt = torch.full((b, n), np.nan, dtype=torch.float64, device="cuda")
    qmc.qmc_udv(n, b, Xt.data_ptr(), Qt.data_ptr(), Dt.data_ptr(), Vt.data_ptr())
    return Qt.cpu().numpy(), Dt.cpu().numpy(), Vt.cpu().numpy()


def _inputs(n, b, graded, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(b, n, n)) + 1j * rng.normal(size=(b, n, n))
    if graded:
        X = X * np.exp(rng.uniform(-120, 120, size=(b, 1, n)))
    return X


def _check(X, Q, D, V):
    n = X.shape[1]
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(V)) and np.all(D > 0)
    un = np.abs(np.conj(np.swapaxes(Q, 1, 2)) @ Q - np.eye(n)).max()
    assert un < 1e-13, un
    Y = Q @ (D[:, :, None] * V)
    colerr = (np.abs(Y - X).max(1) / np.abs(X).max(1)).max()
    assert colerr < 1e-12, colerr
    # V's rows have unit-modulus pivots: |V| entries of each row at most ~1
    # where the ordering is by norm (row i of R is dominated by R_ii)
    return un, colerr


@pytest.mark.parametrize("n", [2, 10, 36, 72, 120, 280])
@pytest.mark.parametrize("graded", [False, True])
def test_udv_reproduces_x(qmc, n, graded):
    X = _inputs(n, 8 if n <= 120 else 2, graded, n + 7 * graded)
    _check(X, *_udv(qmc, X))


RUN = """
import sys, numpy as np, torch
sys.path.insert(0, '.')
from paper_2605_03700_gb300 import build
build.build()
import paper_2605_03700_gb300 as P
from tests.test_gpu_udv import _inputs, _udv
X = _inputs(int(sys.argv[1]), 8, True, 3)
Q, D, V = _udv(P, X)
np.savez(sys.argv[2], Q=Q, D=D, V=V)
"""


def test_blocked_and_pivoted_kernels_agree(tmp_path):
    """Both kernels factor the same graded matrices; the products agree
    column by column, and so do the Gram matrices V^H D^2 V = X^H X."""
    out = {}
    for cs in (1, 4):
        path = str(tmp_path / f"udv{cs}.npz")
        r = subprocess.run([sys.executable, "-c", RUN, "72", path], cwd=ROOT, capture_output=True,
                           text=True, timeout=600, env=dict(os.environ, QMC_QR_CS=str(cs)))
        assert r.returncode == 0, r.stderr[-3000:]
        out[cs] = np.load(path)
    X = _inputs(72, 8, True, 3)
    for cs in (1, 4):
        Q, D, V = out[cs]["Q"], out[cs]["D"], out[cs]["V"]
        _check(X, Q, D, V)
