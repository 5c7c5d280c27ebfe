"""The blocked cluster LU (panels of 8 columns spread over a cluster of CTAs
per matrix) against the one-CTA LU, and both against the oracle.

Per element the blocked factorisation performs the unblocked algorithm's
operations in the same order (the rows of U by forward substitution in panel
order, the trailing update with k in panel order, the same pivot rule), so a
chain run with any cluster size must be bit-identical to one run with the
one-CTA kernel.  The cluster size is read once per process
(QMC_LU_CS=1, 2, 4, 8), so each size runs in a fresh process; the traces,
fields, G and records are compared bit for bit, and the FP64 ratios against
the oracle's brute-force values.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one chain batch per case: (N_phi, beta, precision, sweeps); N = 2 N_phi is
# 10 (ragged last panel, 2 panels on a 4-CTA cluster), 72 (9 panels) and
# 120 (15 panels)
CASES = [(5, 1.0, 0, 3), (36, 0.4, 0, 2), (36, 0.4, 1, 2), (60, 0.2, 1, 1)]

RUN = """
import sys, numpy as np
from paper_2605_03700_gb300 import build
build.build()
import paper_2605_03700_gb300 as P
nphi, beta, prec, nsw, out = int(sys.argv[1]), float(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), sys.argv[5]
L = int(round(beta / 0.1))
ch = P.Chain(P.QMC_TORUS, nphi, beta, 0.1, 1.2, 0.05, 0, n_chains=3, seeds=[7, 8, 9], n_stab=2,
             precision=prec, trace_capacity=2 * nsw * L)
ch.sweep(nsw)
ch.sweep_prior(nsw, 0.0)
ch.sync()
np.savez(out, trace=np.stack([ch.trace(c) for c in range(3)]), phi=np.stack([ch.fields(c) for c in range(3)]),
         green=np.stack([ch.green(c) for c in range(3)]), series=ch.series())
"""


def _run(cs, case, tmp_path):
    out = str(tmp_path / f"lu_{cs}_{case[0]}_{case[2]}.npz")
    env = dict(os.environ, QMC_LU_CS=str(cs))
    r = subprocess.run([sys.executable, "-c", RUN] + [str(x) for x in case] + [out], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


@pytest.mark.parametrize("case", CASES)
def test_cluster_lu_bit_identical_to_one_cta(case, tmp_path):
    ref = _run(1, case, tmp_path)
    assert 0 < ref["trace"][:, :, 6].sum() < ref["trace"][:, :, 6].size
    for cs in (2, 4, 8):
        got = _run(cs, case, tmp_path)
        for key in ("trace", "phi", "green", "series"):
            assert np.array_equal(got[key], ref[key]), (cs, key)


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


@pytest.mark.parametrize("N", [2, 10, 72, 120])
def test_ratio_update_log_det_against_numpy(qmc, N):
    """log det M and G M^-1 of the ratio update (blocked LU + right
    division) against numpy's FP64 results on random well-conditioned
    inputs."""
    import ctypes as C
    import torch
    rng = np.random.default_rng(N)
    b = 3
    G = 0.5 * np.eye(N) + 0.1 * (rng.normal(size=(b, N, N)) + 1j * rng.normal(size=(b, N, N)))
    D = np.eye(N) + 0.1 * (rng.normal(size=(b, N, N)) + 1j * rng.normal(size=(b, N, N)))
    Gt = torch.tensor(G, dtype=torch.complex128, device="cuda")
    Dt = torch.tensor(D, dtype=torch.complex128, device="cuda")
    Gp = torch.empty_like(Gt)
    ld = torch.empty(b, dtype=torch.complex128, device="cuda")
    c = qmc.lib().qmc_ratio_update(N, b, C.c_void_p(Gt.data_ptr()), C.c_void_p(Dt.data_ptr()),
                                   C.c_void_p(Gp.data_ptr()), C.c_void_p(ld.data_ptr()),
                                   C.c_void_p(0))
    torch.cuda.synchronize()
    assert c == 0
    M = np.eye(N) + (D - np.eye(N)) @ (np.eye(N) - G)
    sign, logabs = np.linalg.slogdet(M)
    ref = logabs + 1j * np.angle(sign)
    got = ld.cpu().numpy()
    assert np.abs(got.real - ref.real).max() < 1e-11
    assert np.abs(np.angle(np.exp(1j * (got.imag - ref.imag)))).max() < 1e-11
    X = G @ np.linalg.inv(M)
    assert np.abs(Gp.cpu().numpy() - X).max() < 1e-11 * np.abs(X).max()
