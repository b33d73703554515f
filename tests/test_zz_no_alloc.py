"""hf_precond_noalloc: the lower-precision solve Q^-1 with no device allocation.

Some callers cannot allocate device memory while they run (another allocator owns
the memory, or cudaMalloc's implicit synchronisation is not acceptable).  The
no-allocation entry point keeps its scratch in a fixed device array of the
library; this test checks, through the C ABI, that it returns what hf_precond
returns, on two calls in a row with different inputs (the array keeps the first
call's contents), and that it rejects a request larger than the array.
Collected last so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

from workloads import diffusion2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# both scratch layouts: the FP32 factor (FP32 sweep vectors and cast copies) and the FP64
# factor of the plain double form (FP64 sweep vectors)
FORMS = {"fp32_factor": 0, "fp64_factor": 1}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_precond_noalloc_matches_precond_on_two_calls(form):
    import paper_2208_01907_gb300 as hf
    s = diffusion2d(48, 48, n_islands=6, island=4, contrast=1e8, seed=1)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, precision=FORMS[form])
    H.factorize(torch.tensor(s.val, device="cuda"), 1e-2)
    rng = np.random.default_rng(7)
    for m in (3, 5):
        R = torch.tensor(rng.standard_normal((s.L, m)), device="cuda")
        W_ref = torch.full_like(R, np.nan)
        W_new = torch.full_like(R, np.nan)
        H.precond(R, W_ref)
        H.precond_noalloc(R, W_new)
        ref, new = W_ref.cpu().numpy(), W_new.cpu().numpy()
        assert np.isfinite(new).all()
        assert np.linalg.norm(new - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_precond_noalloc_rejects_scratch_above_limit(form):
    import paper_2208_01907_gb300 as hf
    s = diffusion2d(48, 48, n_islands=6, island=4, contrast=1e8, seed=1)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, precision=FORMS[form])
    H.factorize(torch.tensor(s.val, device="cuda"), 1e-2)
    m = 2000                                   # (rows of all fronts + L) * m * (4 or 8) B > 64 MiB
    R = torch.zeros((s.L, m), dtype=torch.float64, device="cuda")
    W = torch.zeros_like(R)
    with pytest.raises(hf.HFError) as e:
        H.precond_noalloc(R, W)
    assert e.value.code == hf.hf.HF_ERR_ARG
