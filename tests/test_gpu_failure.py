"""Failure detection on the GPU without a fault: a bounded wait that runs out.

The dataflow triangular sweeps (one launch per tree level) let a block wait for a
diagonal block that another block solves.  Every such wait polls a flag a bounded
number of times (hf_opts.spin_limit); a wait that gives up sets an abort word, every
later wait of the launch gives up at once, and the host reports HF_ERR_TIMEOUT after
the sweep.  With a limit of one poll, a block that reaches its first wait before the
block it reads has been published gives up, which happens on any front with more than
one diagonal block.  No kernel traps, faults or spins without a bound; the context
stays usable and the next factorization clears the state.
"""
import numpy as np
import pytest

from workloads import stokes3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sweep_wait_timeout_is_reported_and_cleared_by_refactorization():
    import paper_2208_01907_gb300 as hf
    s = stokes3d(10, seed=2)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    vals = torch.tensor(s.val, device="cuda")
    H.factorize(vals, 1e-2)
    _, lam2 = H.split()
    rng = np.random.default_rng(5)
    X = rng.standard_normal((s.L, 64))
    X[lam2] = 0
    R = torch.tensor(X, device="cuda")
    W_ref = torch.zeros_like(R)
    H.precond(R, W_ref)                              # built-in limit: completes
    H.set_spin_limit(1)
    W = torch.zeros_like(R)
    with pytest.raises(hf.HFError) as e:
        H.precond(R, W)
    assert e.value.code == hf.hf.HF_ERR_TIMEOUT
    # the solves of this factor stay void until the next factorization
    H.set_spin_limit(0)
    with pytest.raises(hf.HFError) as e:
        H.precond(R, W)
    assert e.value.code == hf.hf.HF_ERR_TIMEOUT
    H.factorize(vals, 1e-2)
    W2 = torch.zeros_like(R)
    H.precond(R, W2)
    assert torch.equal(W2, W_ref)                    # same factor, same deterministic sweeps
    H.schur()
    assert H.info()["kernel_dim"] == 3


def test_spin_limit_rejects_negative():
    import paper_2208_01907_gb300 as hf
    s = stokes3d(4, seed=2)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    with pytest.raises(hf.HFError) as e:
        H.set_spin_limit(-1)
    assert e.value.code == hf.hf.HF_ERR_ARG
