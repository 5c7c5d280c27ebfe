"""Checkpoint files (host code of libqmc, no GPU): round trip, atomic
replacement, and rejection of corrupted, truncated, overlong and foreign
files."""
import ctypes as C
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def qmc():
    from paper_2605_03700_gb300 import build
    build.build()
    from paper_2605_03700_gb300 import qmc as Q
    return Q


def _header(Q, n):
    h = Q.qmc_checkpoint_header()
    h.magic, h.version = Q.QMC_CKPT_MAGIC, Q.QMC_CKPT_VERSION
    h.geometry, h.n_orb, h.L, h.n_q, h.n_chains = 0, 4, 20, 37, 3
    h.precision, h.drift, h.n_stab = 1, 0, 5
    h.beta, h.dtau, h.params_hash, h.n_doubles = 2.0, 0.1, 0x1234_5678_9ABC_DEF0, n
    return h


def test_layout_and_round_trip(qmc, tmp_path):
    assert C.sizeof(qmc.qmc_checkpoint_header) == 72
    state = np.random.default_rng(1).normal(size=3 * 20 * 148 + 4)
    h = _header(qmc, state.size)
    p = tmp_path / "run.ckpt"
    qmc.checkpoint_write(p, h, state)
    assert os.path.getsize(p) == 72 + 8 * state.size + 8
    assert [f for f in os.listdir(tmp_path)] == ["run.ckpt"]     # no temporary left
    h2 = qmc.checkpoint_read_header(p)
    assert bytes(h2) == bytes(h)
    assert np.array_equal(qmc.checkpoint_read(p, h), state)
    # a second write replaces the file whole
    qmc.checkpoint_write(p, h, 2 * state)
    assert np.array_equal(qmc.checkpoint_read(p), 2 * state)


def test_damaged_or_foreign_files_are_rejected(qmc, tmp_path):
    state = np.arange(50, dtype=float)
    h = _header(qmc, state.size)
    p = tmp_path / "a.ckpt"
    qmc.checkpoint_write(p, h, state)
    raw = p.read_bytes()
    cases = {
        "flipped bit in the state": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
        "truncated": raw[:-9],
        "trailing byte": raw + bytes(1),
        "bad magic": b"XXXX" + raw[4:],
    }
    for name, data in cases.items():
        q = tmp_path / "bad.ckpt"
        q.write_bytes(data)
        with pytest.raises(qmc.QMCError, match="checkpoint file"):
            qmc.checkpoint_read(q)
    # a file of another run (different couplings hash): an argument error
    other = _header(qmc, state.size)
    other.params_hash ^= 1
    with pytest.raises(qmc.QMCError, match="invalid argument"):
        qmc.checkpoint_read(p, other)
    with pytest.raises(qmc.QMCError, match="checkpoint file"):
        qmc.checkpoint_read_header(tmp_path / "missing.ckpt")
    # a short destination and a state of the wrong length
    L = qmc.lib()
    buf = np.zeros(10)
    assert L.qmc_checkpoint_read(os.fsencode(p), None, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                 10) == -1
    with pytest.raises(qmc.QMCError):
        qmc.checkpoint_write(tmp_path / "x.ckpt", h, state[:-1])
    # an unwritable location fails cleanly
    with pytest.raises(qmc.QMCError, match="checkpoint file"):
        qmc.checkpoint_write(tmp_path / "no" / "such" / "dir.ckpt", h, state)
