"""qmc_ratio_update_noalloc, the variant of the ratio-and-G-update step for
callers that may not allocate device memory (their host framework owns all
device memory, or a fixed memory budget makes a run-time allocation risky),
checked against qmc_ratio_update, which allocates its own scratch.

Both are called through the C ABI on the same device inputs; two calls of
the allocation-free entry point in a row (different batch sizes, so the
second runs on the scratch left behind by the first) must each reproduce the
allocating entry point within the tolerances of the parity tests.  This file
is collected last so that a run stopping at the first failure has run every
other test first.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_LOGR = 1e-10
TOL_G = 1e-9


def _inputs(rng, N, batch, torch):
    """well-conditioned G (norm ~ 1/2) and Delta = 1 + small, as device
    complex128 tensors"""
    G = 0.5 * np.eye(N) + 0.1 * (rng.normal(size=(batch, N, N)) + 1j * rng.normal(size=(batch, N, N))) / np.sqrt(N)
    D = np.eye(N) + 0.2 * (rng.normal(size=(batch, N, N)) + 1j * rng.normal(size=(batch, N, N))) / np.sqrt(N)
    return (torch.tensor(G, dtype=torch.complex128, device="cuda"),
            torch.tensor(D, dtype=torch.complex128, device="cuda"))


def _call(fn, N, batch, G, D, torch):
    Gp = torch.empty_like(G)
    ld = torch.empty(batch, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = fn(N, batch, C.c_void_p(G.data_ptr()), C.c_void_p(D.data_ptr()),
              C.c_void_p(Gp.data_ptr()), C.c_void_p(ld.data_ptr()), C.c_void_p(stream))
    torch.cuda.synchronize()
    return code, Gp.cpu().numpy(), ld.cpu().numpy()


def test_noalloc_ratio_update_matches_allocating_entry_point():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    from paper_2605_03700_gb300 import qmc
    lib = qmc.lib()
    rng = np.random.default_rng(2024)
    for N, batch in [(72, 8), (19, 3)]:
        G, D = _inputs(rng, N, batch, torch)
        c_ref, Gp_ref, ld_ref = _call(lib.qmc_ratio_update, N, batch, G, D, torch)
        c_new, Gp_new, ld_new = _call(lib.qmc_ratio_update_noalloc, N, batch, G, D, torch)
        assert c_ref == 0 and c_new == 0
        assert np.abs(Gp_new - Gp_ref).max() <= TOL_G * np.abs(Gp_ref).max()
        assert np.abs(ld_new.real - ld_ref.real).max() < TOL_LOGR
        assert np.abs(np.exp(1j * ld_new.imag) - np.exp(1j * ld_ref.imag)).max() < TOL_LOGR
        # and it really is the ratio: det M by numpy's LU on the host
        Gh, Dh = G.cpu().numpy(), D.cpu().numpy()
        Mh = np.eye(N) + (Dh - np.eye(N)) @ (np.eye(N) - Gh)
        sign, lab = np.linalg.slogdet(Mh)
        assert np.abs(ld_new.real - lab).max() < 1e-9
    # a request beyond the 8 MiB scratch is refused before any device work
    G, D = _inputs(rng, 72, 1, torch)
    Gp = torch.empty_like(G)
    ld = torch.empty(1, dtype=torch.complex128, device="cuda")
    too_big = lib.qmc_ratio_update_noalloc(72, 40, C.c_void_p(G.data_ptr()), C.c_void_p(D.data_ptr()),
                                           C.c_void_p(Gp.data_ptr()), C.c_void_p(ld.data_ptr()),
                                           C.c_void_p(0))
    assert too_big == -1
