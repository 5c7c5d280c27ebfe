"""Checkpoint and resume on the GPU (qmc_get_state / qmc_set_state): a
context rebuilt from a checkpoint continues as the uninterrupted one, in
step with the oracle resumed from the same state."""
import numpy as np
import pytest

from oracle import model as M
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _chain(qmc, **kw):
    return qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=[0.5, 1.2, 2.0],
                     anisotropies=[0.0, 0.1, -0.15], seeds=[3, 11, 42], n_stab=5, n_adapt=8,
                     **kw)


def test_resumed_context_continues_the_chain(qmc):
    a = _chain(qmc)
    a.sweep(5)
    st = a.get_state()
    nf = 4 * a.n_q
    assert st.shape == (3 * a.L * nf + 3 + 1,)
    assert st[-1] == 5
    a.sweep(6)
    a.sync()
    ref = a.series()
    b = _chain(qmc)
    b.set_state(st)
    b.sweep(6)
    b.sync()
    got = b.series()
    assert got.shape == (3, 6, qmc.QMC_NOBS)
    assert np.array_equal(got[:, :, 17], ref[:, -6:, 17])        # same decisions
    assert np.allclose(got, ref[:, -6:], rtol=1e-10, atol=1e-13)
    for c in range(3):
        assert np.abs(a.fields(c) - b.fields(c)).max() < 1e-10
    # and in step with the oracle resumed from the same fields and steps
    o = O.Chain(M.TORUS, 4, 1.0, 0.1, 1.2, 0.1, 11, n_stab=5, n_adapt=8)
    L = o.L
    ost = np.concatenate([st[L * nf:2 * L * nf], [st[3 * L * nf + 1], st[-1]]])
    o.set_state(ost)
    obs = o.sweep(6)
    assert np.array_equal(obs[:, 17], got[1, :, 17])
    with pytest.raises(qmc.QMCError):
        b.set_state(st[:-1])
    bad = st.copy()
    bad[-1] = -1
    with pytest.raises(qmc.QMCError):
        b.set_state(bad)
    # a non-finite field or step is refused before it reaches the device
    for k in (7, 3 * L * nf):
        bad = st.copy()
        bad[k] = np.nan
        with pytest.raises(qmc.QMCError):
            b.set_state(bad)


def test_checkpoint_file_round_trip(qmc, tmp_path):
    a = _chain(qmc)
    a.sweep(3)
    p = tmp_path / "batch.ckpt"
    a.save(p)
    a.sweep(4)
    a.sync()
    ref = a.series()[:, -4:]
    b = _chain(qmc)
    b.load(p)
    b.sweep(4)
    b.sync()
    assert np.array_equal(b.series()[:, :, 17], ref[:, :, 17])
    # a context with other couplings refuses the file
    c = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=[0.5, 1.2, 2.1],
                  anisotropies=[0.0, 0.1, -0.15], seeds=[3, 11, 42], n_stab=5, n_adapt=8)
    with pytest.raises(qmc.QMCError):
        c.load(p)
