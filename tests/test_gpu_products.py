"""The dense products of the block GCR (Sec. 3.5, Alg. 5) through hf_gram_fp64 and
hf_update_fp64: G = A^T B and Y = Yinit + sgn A C, by default products of BF16 slices
on the tensor cores.  Each row of the left operand and column of the right one is
scaled by its largest power of two and cut into 8 digits of 7 bits, so every product
term carries an error of about 2^-53 relative to the row and column maxima: the normwise
FP64 level.  Checked element by element against the exact products (numpy extended
precision) for |err_ij| <= 4 K u max|a_i| max|b_j| (a dropped slice diagonal s + t = 6
would exceed it more than tenfold), with entries spanning a wide exponent range, exact
zeros, ragged sizes (not multiples of the 128 x 64 tiles nor of the 8-row slice groups)
and K split into chunks."""
import numpy as np
import pytest

from workloads import diffusion2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
C_BOUND = 4.0           # |err_ij| <= C_BOUND * u * (K max|a_i| max|b_j| + |Yinit_ij|)


def _ctx(**opts):
    import paper_2208_01907_gb300 as hf
    s = diffusion2d(12, 12, n_islands=0, seed=3)
    return hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, **opts)


def _operand(rng, L, m, spread):
    x = rng.standard_normal((L, m))
    x *= 2.0 ** rng.integers(-spread, spread + 1, size=(L, m))
    x[rng.random((L, m)) < 0.05] = 0.0          # exact zeros
    return x


def _exact_gram(A, B):
    return (A.astype(np.longdouble).T @ B.astype(np.longdouble))


def _check(got, ref, amax, bmax, K, what, extra=None):
    """amax[i] = max|a_i| (row i of the left factor), bmax[j] = max|b_j|, K terms per entry."""
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    scale = np.outer(amax, bmax)
    tol = C_BOUND * U * (K * scale + (0.0 if extra is None else extra))
    sc = np.where(scale > 0, scale, np.inf)
    print(f"{what}: max |err| / (max|a| max|b|) = {np.max(err / sc) / U:.2f} u "
          f"= {np.max(err / sc) / U / np.sqrt(K):.2f} sqrt(K) u = {np.max(err / sc) / U / K:.3f} K u")
    assert (err <= tol).all(), f"{what}: {int((err > tol).sum())} entries above the bound"


@pytest.mark.parametrize("L,ma,mb,spread", [(3001, 37, 70, 20), (8009, 70, 65, 8), (257, 1, 1, 30)])
def test_gram_matches_exact(L, ma, mb, spread):
    H = _ctx()
    rng = np.random.default_rng(L + ma)
    A, B = _operand(rng, L, ma, spread), _operand(rng, L, mb, spread)
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    G = torch.zeros((ma, mb), dtype=torch.float64, device="cuda")
    H.gram_fp64(At, Bt, G, 1.0)
    _check(G.cpu().numpy(), _exact_gram(A, B), np.abs(A).max(0), np.abs(B).max(0), L, f"gram L={L} {ma}x{mb}")


def test_gram_symmetric_and_scaled():
    H = _ctx()
    rng = np.random.default_rng(5)
    A = _operand(rng, 4099, 96, 12)
    At = torch.tensor(A, device="cuda")
    G = torch.zeros((96, 96), dtype=torch.float64, device="cuda")
    H.gram_fp64(At, At, G, -0.5)
    g = G.cpu().numpy()
    assert (g == g.T).all()                     # A^T A: one product, mirrored
    am = np.abs(A).max(0)
    _check(g, -0.5 * _exact_gram(A, A), 0.5 * am, am, 4099, "gram A^T A")


@pytest.mark.parametrize("L,m,spread,with_init", [(5003, 41, 20, True), (1000, 130, 6, False)])
def test_update_matches_exact(L, m, spread, with_init):
    H = _ctx()
    rng = np.random.default_rng(m)
    A, C = _operand(rng, L, m, spread), _operand(rng, m, m, spread)
    Y0 = _operand(rng, L, m, spread)
    At, Ct = torch.tensor(A, device="cuda"), torch.tensor(C, device="cuda")
    if with_init:
        Yi = torch.tensor(Y0, device="cuda")
        Y = torch.full((L, m), np.nan, dtype=torch.float64, device="cuda")   # overwritten, never read
        H.update_fp64(At, Ct, Y, Yi, -1.0)
    else:
        Y = torch.tensor(Y0, device="cuda")
        H.update_fp64(At, Ct, Y, None, -1.0)
    ref = Y0.astype(np.longdouble) - A.astype(np.longdouble) @ C.astype(np.longdouble)
    _check(Y.cpu().numpy(), ref, np.abs(A).max(1), np.abs(C).max(0), m, f"update L={L} m={m}", extra=np.abs(Y0))


def test_native_fp64_products_agree():
    """The same entry points with hf_opts.fp64_gemm = 1 (native FP64 kernels)."""
    H = _ctx(fp64_gemm=1)
    rng = np.random.default_rng(9)
    A, B = _operand(rng, 2003, 33, 10), _operand(rng, 2003, 17, 10)
    G = torch.zeros((33, 17), dtype=torch.float64, device="cuda")
    H.gram_fp64(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), G, 1.0)
    absref = np.abs(A).T.astype(np.longdouble) @ np.abs(B).astype(np.longdouble)
    err = np.abs(G.cpu().numpy().astype(np.longdouble) - _exact_gram(A, B))
    assert (err <= 2003 * U * absref).all()     # a plain FP64 dot product's bound (gamma_K |A|^T |B|)
