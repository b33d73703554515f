"""Seeded synthetic sparse systems standing in for the paper's FEM matrices.

The paper measures on phb1HYS, a FreeFEM Stokes matrix and a drift-diffusion
matrix (Sec. 4.1-4.3); none of them is available here.  These generators build
matrices with the same structure: 2D/3D stencils, high coefficient contrast,
singular Neumann / traction-free kernels and saddle-point zero blocks.

Every function returns a :class:`CsrSystem` whose CSR pattern is structurally
symmetric, sorted by column within each row, and holds the diagonal entry of
every row (possibly an explicit zero), which is what the library's analysis
step requires.  Randomness comes only from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp


@dataclass
class CsrSystem:
    """A symmetric sparse matrix K-bar in CSR form plus the geometry of its unknowns."""

    name: str
    rowptr: np.ndarray          # int64, L+1
    col: np.ndarray             # int32, nnz
    val: np.ndarray             # float64, nnz
    coords: np.ndarray          # float64, L x dim (node / cell / face centres)
    kernel: np.ndarray | None   # float64, L x r basis of ker(K-bar) when known analytically
    meta: dict = field(default_factory=dict)   # generator parameters; "saddle_point": True marks
                                               # a zero diagonal block ([A B^T; B 0] forms)

    @property
    def L(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col.astype(np.int64), self.rowptr), shape=(self.L, self.L))


def _finish(name, A: sp.spmatrix, coords, kernel=None, **meta) -> CsrSystem:
    """Symmetrise the pattern, force a stored diagonal and sort columns."""
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    L = A.shape[0]
    # symmetric pattern with every diagonal stored; values placed by (row, col) key so
    # that explicit zeros (e.g. a zero pressure block diagonal) survive
    P = (abs(A) + abs(A.T) + sp.identity(L, format="csr")).tocsr()
    P.sort_indices()
    prow = np.repeat(np.arange(L, dtype=np.int64), np.diff(P.indptr))
    pkey = prow * L + P.indices.astype(np.int64)
    C = A.tocoo()
    akey = C.row.astype(np.int64) * L + C.col.astype(np.int64)
    data = np.zeros(P.nnz)
    data[np.searchsorted(pkey, akey)] = C.data
    A = sp.csr_matrix((data, P.indices, P.indptr), shape=(L, L))
    return CsrSystem(
        name=name,
        rowptr=A.indptr.astype(np.int64),
        col=A.indices.astype(np.int32),
        val=A.data.astype(np.float64),
        coords=np.ascontiguousarray(coords, dtype=np.float64),
        kernel=None if kernel is None else np.ascontiguousarray(kernel, dtype=np.float64),
        meta=meta,
    )


# --------------------------------------------------------------------------
# 2D cell-centred diffusion (phb1HYS-like SPD / Neumann-singular matrices)
# --------------------------------------------------------------------------
def _place_islands(rng, nx, ny, n_islands, size, gap):
    """Non-overlapping size x size squares, >= gap cells from each other and the boundary."""
    placed = []
    tries = 0
    while len(placed) < n_islands:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place islands")
        x0 = int(rng.integers(gap, nx - gap - size + 1))
        y0 = int(rng.integers(gap, ny - gap - size + 1))
        ok = all(abs(x0 - x1) >= size + gap or abs(y0 - y1) >= size + gap for x1, y1 in placed)
        if ok:
            placed.append((x0, y0))
    return placed


def diffusion2d(nx=48, ny=48, n_islands=6, island=4, contrast=1e8, seed=1, gap=2,
                dirichlet_x=False, kcell=None, name=None) -> CsrSystem:
    """Cell-centred finite volumes for -div(k grad u) on an nx x ny grid of unit cells.

    Face transmissibility is the harmonic mean 2 k_a k_b / (k_a + k_b).  The
    boundary is no-flux, except that ``dirichlet_x`` adds a ghost
    transmissibility 2 k_c on the x = 0 and x = 1 sides.  ``n_islands`` square
    islands of ``island`` x ``island`` cells get coefficient ``contrast``
    (a scalar or one value per island).
    """
    rng = np.random.default_rng(seed)
    if kcell is None:
        k = np.ones((ny, nx))
        islands = _place_islands(rng, nx, ny, n_islands, island, gap) if n_islands else []
        cvals = np.broadcast_to(np.asarray(contrast, dtype=np.float64), (max(len(islands), 1),))
        for (x0, y0), c in zip(islands, cvals):
            k[y0:y0 + island, x0:x0 + island] = c
    else:
        k = np.asarray(kcell, dtype=np.float64).reshape(ny, nx)
        islands = []
    idx = np.arange(nx * ny).reshape(ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros(nx * ny)
    # x faces
    ka, kb = k[:, :-1], k[:, 1:]
    t = 2.0 * ka * kb / (ka + kb)
    a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    rows += [a, b]; cols += [b, a]; vals += [-t.ravel(), -t.ravel()]
    np.add.at(diag, a, t.ravel()); np.add.at(diag, b, t.ravel())
    # y faces
    ka, kb = k[:-1, :], k[1:, :]
    t = 2.0 * ka * kb / (ka + kb)
    a, b = idx[:-1, :].ravel(), idx[1:, :].ravel()
    rows += [a, b]; cols += [b, a]; vals += [-t.ravel(), -t.ravel()]
    np.add.at(diag, a, t.ravel()); np.add.at(diag, b, t.ravel())
    if dirichlet_x:
        np.add.at(diag, idx[:, 0], 2.0 * k[:, 0])
        np.add.at(diag, idx[:, -1], 2.0 * k[:, -1])
    rows.append(np.arange(nx * ny)); cols.append(np.arange(nx * ny)); vals.append(diag)
    L = nx * ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(L, L))
    xs, ys = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    coords = np.stack([xs.ravel(), ys.ravel()], axis=1)
    kernel = None if dirichlet_x else np.ones((L, 1)) / math.sqrt(L)
    return _finish(name or f"diffusion2d_{nx}x{ny}", A, coords, kernel,
                   nx=nx, ny=ny, islands=islands, kcell=k, dirichlet_x=dirichlet_x)


# --------------------------------------------------------------------------
# 3D Stokes-like saddle point (Q1 velocity nodes, P0 cell pressures)
# --------------------------------------------------------------------------
def stokes3d(n=32, seed=2, mu_log10=(-3.0, 3.0), p_scale=None, name=None, delta=0.0) -> CsrSystem:
    """[A B^T; B -delta D] on an n^3 node grid, h = 1/(n-1).

    A: 7-point nodal Laplacian for each of the 3 velocity components; the
    weight of an edge is h times the mean viscosity of the (up to 4) cells that
    share it; natural boundary.  B: Q1-P0 divergence, the integral of
    d(phi_node)/dx_d over a cell, +-h^2/4 for its 8 corners, times ``p_scale``.
    Viscosity is 10^U(mu_log10) per cell.  The pressure block is zero, or with
    ``delta`` > 0 the stabilisation -delta D: D is the face-neighbour graph
    Laplacian of the cells times p_scale^2 h^3 (the order of B A^-1 B^T).

    ``p_scale`` nondimensionalises the pressure unknowns.  The default
    h^(-3/2) makes the pressure Schur complement B A^-1 B^T of the same order
    as the unit-scaled velocity block at unit viscosity.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    nc = n - 1
    if p_scale is None:
        p_scale = h ** -1.5
    mu = 10.0 ** rng.uniform(mu_log10[0], mu_log10[1], size=(nc, nc, nc))   # [c, b, a] = (z, y, x)
    mpad = np.full((n + 1, n + 1, n + 1), np.nan)
    mpad[1:n, 1:n, 1:n] = mu
    node = np.arange(n ** 3).reshape(n, n, n)   # [k, j, i]
    nv = 3 * n ** 3
    rows, cols, vals = [], [], []
    diag = np.zeros(nv)

    def edges(axis):
        # weight of edges along `axis` (0 = x, 1 = y, 2 = z in [k, j, i] = (z, y, x) indexing)
        if axis == 0:   # between (k, j, i) and (k, j, i+1); cells (k-1..k, j-1..j, i)
            s = np.stack([mpad[dk:dk + n, dj:dj + n, 1:n] for dk in (0, 1) for dj in (0, 1)])
            a, b = node[:, :, :-1], node[:, :, 1:]
        elif axis == 1:  # (k, j, i)-(k, j+1, i); cells (k-1..k, j, i-1..i)
            s = np.stack([mpad[dk:dk + n, 1:n, di:di + n] for dk in (0, 1) for di in (0, 1)])
            a, b = node[:, :-1, :], node[:, 1:, :]
        else:            # (k, j, i)-(k+1, j, i); cells (k, j-1..j, i-1..i)
            s = np.stack([mpad[1:n, dj:dj + n, di:di + n] for dj in (0, 1) for di in (0, 1)])
            a, b = node[:-1, :, :], node[1:, :, :]
        w = h * np.nanmean(s, axis=0)
        return a.ravel(), b.ravel(), w.ravel()

    for axis in range(3):
        a, b, w = edges(axis)
        for d in range(3):
            ra, rb = 3 * a + d, 3 * b + d
            rows += [ra, rb]; cols += [rb, ra]; vals += [-w, -w]
            np.add.at(diag, ra, w); np.add.at(diag, rb, w)
    rows.append(np.arange(nv)); cols.append(np.arange(nv)); vals.append(diag)
    # divergence
    cell = np.arange(nc ** 3).reshape(nc, nc, nc)
    q = p_scale * h * h / 4.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                nd = node[dz:dz + nc, dy:dy + nc, dx:dx + nc].ravel()
                pc = nv + cell.ravel()
                for d, dd in enumerate((dx, dy, dz)):
                    v = np.full(pc.shape, q if dd == 1 else -q)
                    rows += [pc, 3 * nd + d]; cols += [3 * nd + d, pc]; vals += [v, v]
    L = nv + nc ** 3
    if delta:
        w = delta * p_scale * p_scale * h ** 3
        pdiag = np.zeros(nc ** 3)
        for ax in range(3):
            a = np.take(cell, np.arange(nc - 1), axis=ax).ravel()
            b = np.take(cell, np.arange(1, nc), axis=ax).ravel()
            rows += [nv + a, nv + b]; cols += [nv + b, nv + a]; vals += [np.full(a.shape, w)] * 2
            np.add.at(pdiag, a, -w); np.add.at(pdiag, b, -w)
        rows.append(nv + np.arange(nc ** 3)); cols.append(nv + np.arange(nc ** 3)); vals.append(pdiag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(L, L))
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodec = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    gc = (np.arange(nc) + 0.5) * h
    Zc, Yc, Xc = np.meshgrid(gc, gc, gc, indexing="ij")
    cellc = np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], axis=1)
    coords = np.concatenate([np.repeat(nodec, 3, axis=0), cellc], axis=0)
    kern = np.zeros((L, 3))
    for d in range(3):
        kern[d:nv:3, d] = 1.0 / math.sqrt(n ** 3)
    return _finish(name or f"stokes3d_{n}", A, coords, kern, n=n, h=h, p_scale=p_scale, delta=delta,
                   n_velocity=nv, saddle_point=True)


def row_sign_form(system: CsrSystem, sign: np.ndarray, name: str | None = None) -> CsrSystem:
    """The matrix J K-bar, J = diag(sign), sign_i in {+1, -1}: every row i scaled by sign_i.

    For the saddle point [A B^T; B -delta D] and J = diag(I, -I) this is the
    unsymmetric form [A B^T; -B delta D] of Sec. 4.2.  Same pattern and kernel;
    the signs are kept in meta["row_sign"] (int8).
    """
    sign = np.asarray(sign)
    assert sign.shape == (system.L,) and np.all(np.abs(sign) == 1)
    rows = np.repeat(np.arange(system.L), np.diff(system.rowptr))
    return CsrSystem(
        name=name or f"{system.name}_signed",
        rowptr=system.rowptr.copy(),
        col=system.col.copy(),
        val=system.val * sign[rows],
        coords=system.coords.copy(),
        kernel=None if system.kernel is None else system.kernel.copy(),
        meta={**system.meta, "row_sign": sign.astype(np.int8)},
    )


def stokes3d_ldu(n=8, seed=2, delta=0.01, **kw) -> CsrSystem:
    """[A B^T; -B delta D]: the unsymmetric Stokes form of Sec. 4.2 (velocity rows +1, pressure rows -1)."""
    s = stokes3d(n, seed=seed, delta=delta, **kw)
    sign = np.ones(s.L, dtype=np.int8)
    sign[s.meta["n_velocity"]:] = -1
    return row_sign_form(s, sign, name=f"stokes3d_ldu_{n}")


# --------------------------------------------------------------------------
# 3D linear elasticity with Q1 hexahedra (traction free: 6 rigid modes)
# --------------------------------------------------------------------------
def _q1_elasticity_ref(nu: float) -> np.ndarray:
    """24 x 24 stiffness of the unit-modulus Q1 cube of side 1 by 2x2x2 Gauss quadrature.

    Scaling: the element matrix of a cube of side h and modulus E is E * h * K_ref.
    Local node a = ix + 2 iy + 4 iz, dof 3 a + d.
    """
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(3) * mu
    corners = np.array([[ix, iy, iz] for iz in (0, 1) for iy in (0, 1) for ix in (0, 1)], dtype=float)
    sgn = 2 * corners - 1
    g = 1.0 / math.sqrt(3.0)
    K = np.zeros((24, 24))
    for gx in (-g, g):
        for gy in (-g, g):
            for gz in (-g, g):
                xi = np.array([gx, gy, gz])
                # dN/dxi for the 8 shape functions (1+s0 xi)(1+s1 eta)(1+s2 zeta)/8
                f = 1 + sgn * xi            # 8 x 3
                dN = np.empty((8, 3))
                dN[:, 0] = sgn[:, 0] * f[:, 1] * f[:, 2] / 8
                dN[:, 1] = sgn[:, 1] * f[:, 0] * f[:, 2] / 8
                dN[:, 2] = sgn[:, 2] * f[:, 0] * f[:, 1] / 8
                dNx = dN * 2.0                  # d xi / dx = 2 for a unit cube
                B = np.zeros((6, 24))
                for a in range(8):
                    B[0, 3 * a] = dNx[a, 0]
                    B[1, 3 * a + 1] = dNx[a, 1]
                    B[2, 3 * a + 2] = dNx[a, 2]
                    B[3, 3 * a] = dNx[a, 1]; B[3, 3 * a + 1] = dNx[a, 0]
                    B[4, 3 * a + 1] = dNx[a, 2]; B[4, 3 * a + 2] = dNx[a, 1]
                    B[5, 3 * a] = dNx[a, 2]; B[5, 3 * a + 2] = dNx[a, 0]
                K += B.T @ D @ B * 0.125        # det J = (1/2)^3, unit weights
    return K


def elasticity3d(n=40, seed=3, E_in=1e6, n_incl=8, incl=4, nu=0.3, name=None) -> CsrSystem:
    """Q1 linear elasticity on an n^3 node grid (unit cube), traction free.

    Background modulus 1; ``n_incl`` cubic inclusions of ``incl``^3 elements
    with modulus ``E_in``, non-overlapping, placed by the seed.
    """
    rng = np.random.default_rng(seed)
    ne = n - 1
    h = 1.0 / ne
    E = np.ones((ne, ne, ne))
    placed = []
    tries = 0
    while len(placed) < n_incl:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place inclusions")
        c = rng.integers(1, ne - incl, size=3)
        if all(np.any(np.abs(c - p) >= incl + 1) for p in placed):
            placed.append(c)
            E[c[2]:c[2] + incl, c[1]:c[1] + incl, c[0]:c[0] + incl] = E_in
    Kref = _q1_elasticity_ref(nu)
    node = np.arange(n ** 3).reshape(n, n, n)
    enodes = np.stack([node[dz:dz + ne, dy:dy + ne, dx:dx + ne].ravel()
                       for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], axis=1)   # nel x 8
    edofs = (3 * enodes[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    r = np.repeat(edofs, 24, axis=1).ravel()
    c = np.tile(edofs, (1, 24)).ravel()
    v = (E.ravel()[:, None] * h * Kref.ravel()[None, :]).ravel()
    L = 3 * n ** 3
    A = sp.coo_matrix((v, (r, c)), shape=(L, L)).tocsr()
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodec = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    coords = np.repeat(nodec, 3, axis=0)
    # rigid body modes: 3 translations, 3 rotations about the centre
    xc = nodec - 0.5
    R = np.zeros((L, 6))
    for d in range(3):
        R[d::3, d] = 1.0
    R[0::3, 3] = -xc[:, 1]; R[1::3, 3] = xc[:, 0]
    R[1::3, 4] = -xc[:, 2]; R[2::3, 4] = xc[:, 1]
    R[2::3, 5] = -xc[:, 0]; R[0::3, 5] = xc[:, 2]
    Qr, _ = np.linalg.qr(R)
    return _finish(name or f"elasticity3d_{n}", A, coords, Qr, n=n, h=h, inclusions=[p.tolist() for p in placed])


# --------------------------------------------------------------------------
# 2D mixed Darcy (face fluxes + cell pressures, zero block): dd-hole-like
# --------------------------------------------------------------------------
def darcy2d(nx=32, ny=32, seed=4, n_islands=2, island=4, contrast=1e6, gap=2, name=None) -> CsrSystem:
    """[A B^T; B 0] with lumped face mass A_ff = h^2 * mean resistivity and B = +-h.

    Unknowns: interior x-faces, interior y-faces (no-flux boundary: boundary
    faces carry no unknown), then one pressure per cell.  Islands have
    resistivity 1/contrast.  ker = constant pressure (1-dim), as in Sec. 4.3.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / max(nx, ny)
    r = np.ones((ny, nx))
    islands = _place_islands(rng, nx, ny, n_islands, island, gap) if n_islands else []
    cv = np.broadcast_to(np.asarray(contrast, dtype=np.float64), (max(len(islands), 1),))
    for (x0, y0), c in zip(islands, cv):
        r[y0:y0 + island, x0:x0 + island] = 1.0 / c
    cell = np.arange(nx * ny).reshape(ny, nx)
    nfx = (nx - 1) * ny
    nfy = nx * (ny - 1)
    nf = nfx + nfy
    rows, cols, vals = [], [], []
    # x faces between (y, x) and (y, x+1)
    fx = np.arange(nfx).reshape(ny, nx - 1)
    ax = h * h * 0.5 * (r[:, :-1] + r[:, 1:])
    fy = nfx + np.arange(nfy).reshape(ny - 1, nx)
    ay = h * h * 0.5 * (r[:-1, :] + r[1:, :])
    rows += [fx.ravel(), fy.ravel()]; cols += [fx.ravel(), fy.ravel()]; vals += [ax.ravel(), ay.ravel()]
    for f, cl, cr in ((fx, cell[:, :-1], cell[:, 1:]), (fy, cell[:-1, :], cell[1:, :])):
        pl, pr = nf + cl.ravel(), nf + cr.ravel()
        ff = f.ravel()
        one = np.full(ff.shape, h)
        rows += [pl, ff, pr, ff]; cols += [ff, pl, ff, pr]; vals += [one, one, -one, -one]
    L = nf + nx * ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(L, L))
    xs, ys = np.meshgrid(np.arange(nx - 1) + 1.0, np.arange(ny) + 0.5)
    cfx = np.stack([xs.ravel(), ys.ravel()], axis=1)
    xs, ys = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny - 1) + 1.0)
    cfy = np.stack([xs.ravel(), ys.ravel()], axis=1)
    xs, ys = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    cc = np.stack([xs.ravel(), ys.ravel()], axis=1)
    coords = np.concatenate([cfx, cfy, cc], axis=0)
    kern = np.zeros((L, 1))
    kern[nf:, 0] = 1.0 / math.sqrt(nx * ny)
    return _finish(name or f"darcy2d_{nx}x{ny}", A, coords, kern, nx=nx, ny=ny, saddle_point=True)


# --------------------------------------------------------------------------
# batched mix and adjoint field
# --------------------------------------------------------------------------
def batched_systems(count=96, Lmin=2000, Lmax=60000, seed=4):
    """Independent systems with L ~ U[Lmin, Lmax]: even = diffusion with islands, odd = mixed Darcy."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        Lt = int(rng.integers(Lmin, Lmax + 1))
        s = int(rng.integers(0, 2 ** 31))
        if i % 2 == 0:
            m = max(8, int(round(math.sqrt(Lt))))
            ni = max(1, math.ceil(Lt / 400))
            ni = min(ni, (m // 6) ** 2)
            c = 10.0 ** np.random.default_rng(s).uniform(4, 8, size=ni)
            out.append(diffusion2d(m, m, n_islands=ni, island=2, contrast=c, seed=s, gap=2,
                                   name=f"batch{i}_diffusion_{m}"))
        else:
            m = max(8, int(round(math.sqrt(Lt / 3.0))))
            c = 10.0 ** np.random.default_rng(s).uniform(4, 8, size=2)
            out.append(darcy2d(m, m, seed=s, n_islands=2, island=3, contrast=c, name=f"batch{i}_darcy_{m}"))
    return out


def adjoint_diffusion2d(n=256, seed=5, theta=None):
    """cfg-5 field: theta = 3 N(0,1) per cell, k = exp(theta); Dirichlet on x sides, Neumann on y.

    Returns (system, theta, b, x_star, directions) with b, x* ~ U(-1,1) and 32
    unit directions d ~ N(0, I)/|.|.
    """
    rng = np.random.default_rng(seed)
    if theta is None:
        theta = 3.0 * rng.standard_normal(n * n)
    b = rng.uniform(-1, 1, n * n)
    xs = rng.uniform(-1, 1, n * n)
    dirs = rng.standard_normal((32, n * n))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    sys_ = diffusion2d(n, n, n_islands=0, dirichlet_x=True, kcell=np.exp(theta), name=f"adjoint2d_{n}")
    return sys_, theta, b, xs, dirs


def diffusion2d_structure(system: CsrSystem) -> dict:
    """CSR positions of each face's four entries for a ``diffusion2d`` system.

    Returns index arrays: cells a, b of every interior face; positions of (a,a), (b,b),
    (a,b), (b,a) in the CSR value array; Dirichlet ghost cells and their diagonal
    positions.  With them any (differentiable) cell-coefficient model can assemble the
    values: t_f on the diagonals, -t_f off them, 2 k_c on ghost diagonals.
    """
    nx, ny = system.meta["nx"], system.meta["ny"]
    idx = np.arange(nx * ny).reshape(ny, nx)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    L = system.L
    prow = np.repeat(np.arange(L, dtype=np.int64), np.diff(system.rowptr))
    key = prow * L + system.col.astype(np.int64)

    def pos(r, c):
        return np.searchsorted(key, r.astype(np.int64) * L + c.astype(np.int64))
    out = dict(a=a, b=b, p_aa=pos(a, a), p_bb=pos(b, b), p_ab=pos(a, b), p_ba=pos(b, a))
    if system.meta.get("dirichlet_x"):
        g = np.concatenate([idx[:, 0], idx[:, -1]])
        out.update(ghost=g, p_gg=pos(g, g))
    else:
        out.update(ghost=np.zeros(0, np.int64), p_gg=np.zeros(0, np.int64))
    return out


def consistent_rhs(system: CsrSystem, seed: int, nrhs: int = 1, mode: str = "uniform") -> np.ndarray:
    """Right-hand sides (L x nrhs, float64) orthogonal to the known kernel.

    mode="uniform": b ~ U(-1,1) projected onto ker^perp (cfg 1);
    mode="solution": b = K-bar x_true, x_true ~ U(-1,1) projected onto ker^perp.
    """
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=(system.L, nrhs))
    V = system.kernel
    if V is not None:
        v = v - V @ np.linalg.lstsq(V, v, rcond=None)[0]
    if mode == "solution":
        v = system.to_scipy() @ v
    return np.ascontiguousarray(v)


def config_system(cfg: int, scale: str = "full") -> CsrSystem:
    """The systems named by the five workload configurations ("full") or a small variant ("small")."""
    small = scale == "small"
    if cfg == 1:
        return diffusion2d(48, 48, n_islands=6, island=4, contrast=1e8, seed=1)
    if cfg == 2:
        return stokes3d(8 if small else 32, seed=2)
    if cfg == 3:
        return elasticity3d(10 if small else 40, seed=3, n_incl=2 if small else 8, incl=2 if small else 4)
    if cfg == 5:
        return adjoint_diffusion2d(32 if small else 256, seed=5)[0]
    raise ValueError(cfg)
