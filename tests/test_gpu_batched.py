"""Batched form: many independent systems through hf_*_batched (run concurrently on
worker streams) give exactly the results of the same calls made one system at a time,
and every system meets the method's accuracy gates."""
import numpy as np
import pytest

import oracle as O
from workloads import batched_systems, consistent_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(systems):
    import paper_2208_01907_gb300 as hf
    # the saddle-point (Darcy) systems take the null-pivot test: with the ratio test alone
    # FP32 noise pivots of their singular zero-block structure can stay in K11
    Hs = [hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, nd_leaf=128,
                          null_test=int(bool(s.meta.get("saddle_point")))) for s in systems]
    vals = [torch.tensor(s.val, device="cuda", dtype=torch.float64) for s in systems]
    return Hs, vals


def test_batched_equals_one_by_one():
    import paper_2208_01907_gb300 as hf
    systems = batched_systems(count=12, Lmin=600, Lmax=4000, seed=7)
    nrhs = 8
    bs = [consistent_rhs(s, 20 + i, nrhs, "uniform") for i, s in enumerate(systems)]
    # one system at a time
    Hs1, vals1 = _setup(systems)
    ref = []
    for H, v, s, b in zip(Hs1, vals1, systems, bs):
        H.factorize(v, 1e-2)
        H.schur()
        bt = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
        xt = torch.zeros_like(bt)
        H.solve(bt, xt)
        ref.append((H.split()[1].copy(), H.s22(torch).cpu().numpy(), xt.cpu().numpy()))
    # batched
    Hs2, vals2 = _setup(systems)
    st = hf.factorize_batched(Hs2, vals2, 1e-2)
    assert all(v == 0 for v in st)
    hf.schur_batched(Hs2)
    bts = [torch.tensor(np.ascontiguousarray(b.T), device="cuda") for b in bs]
    xts = [torch.zeros_like(bt) for bt in bts]
    hf.solve_batched(Hs2, bts, xts)
    for i, (H, s, b) in enumerate(zip(Hs2, systems, bs)):
        lam2, S22, X = ref[i]
        assert H.split()[1].tolist() == lam2.tolist()
        np.testing.assert_array_equal(H.s22(torch).cpu().numpy(), S22)
        x = xts[i].cpu().numpy()
        np.testing.assert_array_equal(x, X)
        assert O.backward_error(s.to_scipy(), x.T, b) <= 1e-12


def test_batched_rejects_repeated_contexts():
    import paper_2208_01907_gb300 as hf
    systems = batched_systems(count=2, Lmin=600, Lmax=800, seed=3)
    Hs, vals = _setup(systems)
    with pytest.raises(hf.HFError):
        hf.factorize_batched([Hs[0], Hs[0]], [vals[0], vals[0]], 1e-2)
