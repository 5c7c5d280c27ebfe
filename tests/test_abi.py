"""The C-ABI library builds, loads and exports every symbol include/qmc.h
declares; argument validation happens before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_03700_gb300 import build
    build.build()
    from paper_2605_03700_gb300 import qmc
    return qmc.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "qmc_create" in names and "qmc_sweep" in names and "qmc_get_green" in names
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_before_device_work(lib):
    from paper_2605_03700_gb300 import qmc
    h = C.c_void_p()
    o = qmc.qmc_default_opts()
    # beta / dtau not an integer
    assert lib.qmc_create(C.byref(h), 0, 4, 1.05, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert not h.value
    # coupling outside the sign-free region: U_N < 0
    assert lib.qmc_create(C.byref(h), 0, 4, 1.0, 0.1, -1.0, 0.0, 0, C.byref(o)) != 0
    # unsupported geometry code / size
    assert lib.qmc_create(C.byref(h), 7, 4, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert lib.qmc_create(C.byref(h), 0, 1, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert lib.qmc_strerror(-1) == b"invalid argument or unsupported size"


def test_tau_int_host_function(lib):
    import numpy as np
    from paper_2605_03700_gb300 import qmc
    from oracle import analysis as A
    rng = np.random.default_rng(1)
    x = np.zeros(20000)
    for i in range(1, len(x)):
        x[i] = 0.7 * x[i - 1] + rng.normal()
    assert abs(qmc.qmc_tau_int(x) - A.tau_int(x)) < 1e-9
    exact = (1 + 0.7) / (2 * (1 - 0.7))
    assert abs(qmc.qmc_tau_int(x) - exact) < 0.15 * exact
