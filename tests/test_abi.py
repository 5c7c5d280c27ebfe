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


def test_new_entry_points_reject_invalid_arguments_before_device_work(lib):
    """The learned-proposal, graph, group and standalone ratio entry points
    check their arguments before touching the device (runs without a GPU)."""
    from paper_2605_03700_gb300 import qmc
    L = qmc.lib()
    h = C.c_void_p()
    # network: null out, empty field count, oversized width, zero capacity
    assert L.qmc_net_create(None, 10, 8, 4, 0) == -1
    assert L.qmc_net_create(C.byref(h), 0, 8, 4, 0) == -1 and not h.value
    assert L.qmc_net_create(C.byref(h), 10, 5000, 4, 0) == -1
    assert L.qmc_net_create(C.byref(h), 10, 8, 0, 0) == -1
    assert L.qmc_net_destroy(None) == 0
    assert L.qmc_net_num_params(None) == -1 and L.qmc_net_dataset_size(None) == -1
    assert L.qmc_net_train(None, 1, 1, 1e-3, 0.0, None) == -1
    assert L.qmc_net_collect(None, None) == -1
    # sweeps without a context
    assert L.qmc_sweep_learned(None, None, 1, 0.0) == -1
    assert L.qmc_sweep_graph(None, 1) == -1
    # groups: null out, no members, a null member
    arr = (C.c_void_p * 2)(None, None)
    assert L.qmc_group_create(None, arr, 2) == -1
    assert L.qmc_group_create(C.byref(h), arr, 0) == -1
    assert L.qmc_group_create(C.byref(h), arr, 2) == -1
    assert L.qmc_group_sweep(None, 1) == -1 and L.qmc_group_sync(None) == -1
    assert L.qmc_group_destroy(None) == 0
    # standalone ratio updates: sizes beyond what the kernels hold
    assert L.qmc_ratio_update(121, 1, None, None, None, None, None) == -1
    assert L.qmc_ratio_update_noalloc(72, 1, None, None, None, None, None) == -1
    # eigensolver: null buffers, n beyond 140, FP64 beyond 64, unknown precision
    assert L.qmc_eigh(36, 1, None, None, None, 1, None) == -1
    one = C.c_void_p(1)
    assert L.qmc_eigh(141, 1, one, one, one, 1, None) == -1
    assert L.qmc_eigh(65, 1, one, one, one, 0, None) == -1
    assert L.qmc_eigh(36, 1, one, one, one, 3, None) == -1
    # UDV: null buffers, n beyond 280
    assert L.qmc_udv(72, 1, None, None, None, None, None, None) == -1
    assert L.qmc_udv(281, 1, one, None, one, one, one, None) == -1
    # sphere beyond 60 orbitals; torus beyond 140, or beyond 60 in FP64
    o = qmc.qmc_default_opts()
    assert L.qmc_create(C.byref(h), 1, 60, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert L.qmc_create(C.byref(h), 0, 61, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    o.precision = 1
    assert L.qmc_create(C.byref(h), 0, 141, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    o.precision = 3
    assert L.qmc_create(C.byref(h), 0, 4, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    # slice kinds: shared (0) and a set per factor (2); the single exponential
    # (1) is oracle-only
    o = qmc.qmc_default_opts()
    assert o.slice_kind == qmc.QMC_SLICE_SHARED
    o.slice_kind = 1
    assert L.qmc_create(C.byref(h), 0, 4, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert not h.value


def test_opts_struct_matches_the_library(lib):
    """qmc_default_opts writes exactly the binding's qmc_opts: nothing past
    its end (a larger C struct would overrun the caller's buffer), and its
    last field holds the default."""
    from paper_2605_03700_gb300 import qmc
    n = C.sizeof(qmc.qmc_opts)
    buf = (C.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    assert lib.qmc_default_opts(C.cast(buf, C.POINTER(qmc.qmc_opts))) == 0
    assert all(b == 0xA5 for b in bytes(buf)[n:])
    o = qmc.qmc_opts.from_buffer(buf)
    assert o.n_stab == 10 and o.sign_tol == 1e-6 and o.drift == qmc.QMC_DRIFT_EXACT
    assert qmc.qmc_opts.drift.offset + C.sizeof(C.c_int) <= n


def test_unknown_drift_is_rejected(lib):
    from paper_2605_03700_gb300 import qmc
    h = C.c_void_p()
    o = qmc.qmc_default_opts()
    o.drift = 2
    assert lib.qmc_create(C.byref(h), 0, 4, 1.0, 0.1, 1.0, 0.0, 0, C.byref(o)) == -1
    assert not h.value


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with libqmc.so absent the binding raises instead of
    computing anything."""
    from paper_2605_03700_gb300 import qmc
    monkeypatch.setattr(qmc, "LIB", str(tmp_path / "libqmc.so"))
    monkeypatch.setattr(qmc, "_lib", None)
    with pytest.raises(qmc.QMCError, match="missing"):
        qmc.lib()
    with pytest.raises(qmc.QMCError):
        qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 1.0)
