"""The seeded generators at the sizes of the five workload configurations (CPU only).

They are shared by the oracle and the CUDA path, so their structural promises are
checked here: a sorted, structurally symmetric CSR pattern with every diagonal
stored, symmetric values, the analytic kernel basis (K-bar V = 0), the configuration
sizes, determinism under the seed, and the row-sign form of the Stokes matrix.
"""
import numpy as np
import pytest

from workloads import (adjoint_diffusion2d, batched_systems, config_system, consistent_rhs, stokes3d,
                       stokes3d_ldu)


def _structure_ok(s):
    rp, col = s.rowptr, s.col
    assert rp[0] == 0 and rp[-1] == col.shape[0] and (np.diff(rp) >= 1).all()
    rows = np.repeat(np.arange(s.L), np.diff(rp))
    assert ((col[1:] > col[:-1]) | (rows[1:] != rows[:-1])).all()          # sorted per row
    key = rows.astype(np.int64) * s.L + col                                # ascending (sorted rows)
    dkey = np.arange(s.L, dtype=np.int64) * (s.L + 1)
    pos = np.minimum(np.searchsorted(key, dkey), key.shape[0] - 1)
    assert (key[pos] == dkey).all()                                        # diagonal stored
    tkey = np.sort(col.astype(np.int64) * s.L + rows)
    np.testing.assert_array_equal(tkey, key)                               # symmetric pattern
    return rows


@pytest.mark.parametrize("cfg,L,kdim", [(1, 2304, 1), (2, 128095, 3), (3, 192000, 6), (5, 65536, 0)])
def test_configuration_systems(cfg, L, kdim):
    s = config_system(cfg)
    assert s.L == L
    _structure_ok(s)
    K = s.to_scipy()
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()                     # symmetric to assembly rounding
    if kdim:
        V = s.kernel
        assert V.shape == (L, kdim)
        assert np.abs(K @ V).max() <= 1e-10 * abs(K).max()                 # analytic kernel
        assert np.linalg.matrix_rank(V) == kdim
    else:
        assert s.kernel is None
    b = consistent_rhs(s, cfg, 2)
    if kdim:
        assert np.abs(s.kernel.T @ b).max() <= 1e-10 * np.abs(b).max()
    t = config_system(cfg)
    np.testing.assert_array_equal(s.val, t.val)                             # seeded


def test_stokes_nnz_and_paper_sign_form():
    s = config_system(2)
    assert s.nnz == 2129455
    u = stokes3d_ldu(6, delta=0.01)
    S = stokes3d(6, delta=0.01)
    J = u.meta["row_sign"].astype(np.float64)
    nv = S.meta["n_velocity"]
    assert (J[:nv] == 1).all() and (J[nv:] == -1).all()
    rows = _structure_ok(u)
    np.testing.assert_array_equal(u.val, J[rows] * S.val)
    Ku = u.to_scipy()
    assert (Ku.diagonal()[nv:] > 0).all()                                  # +delta D on the diagonal
    assert abs(Ku - Ku.T).max() > 0
    assert np.abs(Ku @ u.kernel).max() <= 1e-10 * abs(Ku).max()


def test_batched_and_adjoint_generators():
    sy = batched_systems(count=6, Lmin=2000, Lmax=6000, seed=4)
    assert len(sy) == 6 and all(2000 <= s.L <= 6000 * 1.1 for s in sy)
    for s in sy:
        _structure_ok(s)
        K = s.to_scipy()
        assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    s, theta = adjoint_diffusion2d(32, seed=5)[:2]
    assert s.L == 32 * 32 and theta.shape == (s.L,)
