"""Seeded synthetic problems for the energy-minimisation prolongation path.

Each generator returns a :class:`Problem`: a symmetric operator ``A`` in CSR
form, the fixed sparsity pattern of ``P`` (the structural pattern of
``A @ P0``, grown by one application of ``A``, Eq. (enlPatt) with k = 1 and
S = pattern(A)), the tentative prolongation ``P0`` stored on that pattern,
the fine near-kernel block ``B`` (V_f, n x k) and the coarse block ``B_c``
(V_c, n_c x k), Section 3 and Eq. (TSP).

The operators stand in for the paper's workloads (Section 5): scalar
diffusion / porous-media flow with heterogeneous coefficients, and 3D linear
elasticity with about 80 entries per row.  The datasets of the paper are not
available, so these seeded synthetic operators replace them.

This module holds none of the method's arithmetic (no Gram factorisation,
no projection, no masked product, no conjugate gradients); both the CUDA
library and the CPU oracle receive the arrays it returns.  Random numbers
come from a counter-based SplitMix64 stream (Steele, Lea and Flood, 2014)
turned into normals by the Box-Muller transform, so every machine draws the
same coefficients for a given seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "splitmix64", "uniform01", "normal",
    "poisson2d", "diffusion3d_fv", "ring1d", "aniso3d", "elasticity3d",
    "random_problem", "strength", "cf_split", "classical", "config", "CONFIG_NAMES",
]

# ---------------------------------------------------------------------------
# counter-based random numbers
# ---------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 sequence for ``seed``.

    Output i is mix(seed + (i + 1) * GAMMA) with the published SplitMix64
    finaliser; all arithmetic wraps modulo 2**64.
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
    th = 2.0 * np.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:count]


# ---------------------------------------------------------------------------
# problem container
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    n: int
    nc: int
    k: int
    A_rowptr: np.ndarray  # int32 [n+1]
    A_col: np.ndarray     # int32 [nnz(A)], sorted and unique per row
    A_val: np.ndarray     # float64 [nnz(A)]
    P_rowptr: np.ndarray  # int32 [n+1]
    P_col: np.ndarray     # int32 [nnz(P)], sorted and unique per row
    P0_val: np.ndarray    # float64 [nnz(P)], P0 on P's pattern
    B: np.ndarray         # float64 [n, k] row-major (V_f)
    Bc: np.ndarray        # float64 [nc, k] row-major (V_c)
    iters: int = 10
    meta: dict = field(default_factory=dict)

    @property
    def nnz_a(self) -> int:
        return int(self.A_rowptr[-1])

    @property
    def nnz_p(self) -> int:
        return int(self.P_rowptr[-1])

    def arrays(self):
        """The arrays in the order of the library's create call."""
        return (self.A_rowptr, self.A_col, self.A_val, self.P_rowptr,
                self.P_col, self.P0_val, self.B, self.Bc)


def _csr_from_dense_slots(cols: np.ndarray, vals: np.ndarray | None,
                          valid: np.ndarray):
    """Pack row-slot arrays (n x s) into CSR, keeping slots where ``valid``.

    The slot order must already be the ascending column order of each row.
    """
    counts = valid.sum(axis=1)
    rowptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[valid].astype(np.int32)
    val = None if vals is None else np.ascontiguousarray(vals[valid], dtype=np.float64)
    return rowptr.astype(np.int32), col, val


def _agg_index(x: np.ndarray, a: int, npts: int) -> np.ndarray:
    """Aggregate index along one axis; the remainder joins the last aggregate."""
    return np.minimum(x // a, npts // a - 1)


def _grid_coords(dims):
    """Lexicographic (x fastest) grid coordinates of every point."""
    nx, ny, nz = dims
    idx = np.arange(nx * ny * nz, dtype=np.int64)
    return idx % nx, (idx // nx) % ny, idx // (nx * ny)


def _stencil_offsets(ndim: int):
    """Neighbour offsets of a 5-point (2D) or 7-point (3D) stencil, sorted so
    that the neighbour's lexicographic index increases."""
    if ndim == 2:
        return [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    return [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0),
            (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def _neighbour_table(dims, offsets):
    """(n, s) neighbour indices and validity for a list of grid offsets."""
    nx, ny, nz = dims
    x, y, z = _grid_coords(dims)
    n = nx * ny * nz
    nb = np.empty((n, len(offsets)), dtype=np.int64)
    ok = np.empty((n, len(offsets)), dtype=bool)
    for s, (dx, dy, dz) in enumerate(offsets):
        xx, yy, zz = x + dx, y + dy, z + dz
        ok[:, s] = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        nb[:, s] = xx + nx * (yy + ny * zz)
    nb[~ok] = 0
    return nb, ok


def _scalar_aggregates(dims, a):
    x, y, z = _grid_coords(dims)
    nx, ny, nz = dims
    ax, ay, az = (_agg_index(x, a, nx), _agg_index(y, a, ny),
                  _agg_index(z, a, nz) if nz > 1 else np.zeros_like(z))
    gx, gy = nx // a, ny // a
    gz = nz // a if nz > 1 else 1
    return ax + gx * (ay + gy * az), gx * gy * gz


def _pattern_from_neighbours(nb, ok, node_agg):
    """Node-level aggregate sets: sorted unique aggregate ids of all
    neighbours (the structural pattern of A @ P0 at node level)."""
    big = np.iinfo(np.int64).max
    g = np.where(ok, node_agg[nb], big)
    g.sort(axis=1)
    keep = g != big
    keep[:, 1:] &= g[:, 1:] != g[:, :-1]
    return g, keep


def _scalar_problem(name, dims, nb, ok, vals, agg, iters, meta):
    """Assemble A from stencil slots and build the k = 1 aggregation data."""
    n = int(np.prod(dims))
    A_rowptr, A_col, A_val = _csr_from_dense_slots(nb, vals, ok)
    node_agg, nc = _scalar_aggregates(dims, agg)
    size = np.bincount(node_agg, minlength=nc).astype(np.float64)
    g, keep = _pattern_from_neighbours(nb, ok, node_agg)
    P_rowptr, P_col, _ = _csr_from_dense_slots(g, None, keep)
    rows = np.repeat(np.arange(n), np.diff(P_rowptr))
    P0_val = np.where(P_col == node_agg[rows], 1.0 / np.sqrt(size[P_col]), 0.0)
    B = np.ones((n, 1))
    Bc = np.sqrt(size)[:, None].copy()
    return Problem(name, n, int(nc), 1, A_rowptr, A_col, A_val, P_rowptr, P_col,
                   P0_val, B, Bc, iters, meta)


# ---------------------------------------------------------------------------
# scalar operators
# ---------------------------------------------------------------------------
def poisson2d(N: int = 64, agg: int = 2, iters: int = 10) -> Problem:
    """2D 5-point Poisson, homogeneous Dirichlet boundary eliminated
    (diagonal 4, off-diagonal -1), lexicographic order; k = 1 constant
    near kernel, agg x agg aggregates, P0 the normalised aggregate indicator."""
    dims = (N, N, 1)
    offs = _stencil_offsets(2)
    nb, ok = _neighbour_table(dims, offs)
    vals = np.where(np.array([o == (0, 0, 0) for o in offs])[None, :], 4.0, -1.0)
    vals = np.broadcast_to(vals, nb.shape)
    return _scalar_problem(f"poisson2d_{N}", dims, nb, ok, vals, agg, iters,
                           {"kind": "poisson2d", "N": N, "agg": agg})


def diffusion3d_fv(N: int = 128, agg: int = 3, sigma: float = 2.0, seed: int = 2,
                   iters: int = 20) -> Problem:
    """3D 7-point finite-volume diffusion with log-normal cell coefficients
    kappa = exp(sigma * xi), xi i.i.d. N(0, 1); harmonic transmissibilities
    T = 2 k k' / (k + k') with unit spacing; no-flux (Neumann) boundary, so
    every row sums to zero."""
    dims = (N, N, N)
    offs = _stencil_offsets(3)
    nb, ok = _neighbour_table(dims, offs)
    kappa = np.exp(sigma * normal(seed, N ** 3))
    kn = kappa[nb]
    kc = kappa[:, None]
    T = np.where(ok, 2.0 * kc * kn / (kc + kn), 0.0)
    centre = offs.index((0, 0, 0))
    T[:, centre] = 0.0
    vals = -T
    vals[:, centre] = T.sum(axis=1)
    return _scalar_problem(f"fv3d_{N}", dims, nb, ok, vals, agg, iters,
                           {"kind": "fv3d", "N": N, "agg": agg, "sigma": sigma,
                            "seed": seed})


def ring1d(n: int = 1000, agg: int = 2, sigma: float = 0.5, seed: int = 3,
           iters: int = 12) -> Problem:
    """Periodic 1D chain (a ring): transmissibility T_i = exp(sigma xi_i)
    between rows i and i + 1 mod n, diagonal T_(i-1) + T_i, so A 1 = 0.  The
    wrap-around coupling joins the first and the last row, the widest
    possible distance between coupled rows in this ordering.  k = 1,
    aggregates of ``agg`` consecutive rows (the remainder joins the last)."""
    T = np.exp(sigma * normal(seed, n))
    i = np.arange(n, dtype=np.int64)
    nb = np.stack([(i - 1) % n, i, (i + 1) % n], axis=1)
    vals = np.stack([-T[(i - 1) % n], T[(i - 1) % n] + T, -T], axis=1)
    order = np.argsort(nb, axis=1, kind="stable")  # ascending columns per row
    nb = np.take_along_axis(nb, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    ok = np.ones(nb.shape, dtype=bool)
    A_rowptr, A_col, A_val = _csr_from_dense_slots(nb, vals, ok)
    nc = n // agg
    node_agg = _agg_index(i, agg, n)
    size = np.bincount(node_agg, minlength=nc).astype(np.float64)
    g, keep = _pattern_from_neighbours(nb, ok, node_agg)
    P_rowptr, P_col, _ = _csr_from_dense_slots(g, None, keep)
    rows = np.repeat(i, np.diff(P_rowptr))
    P0_val = np.where(P_col == node_agg[rows], 1.0 / np.sqrt(size[P_col]), 0.0)
    return Problem(f"ring1d_{n}", n, int(nc), 1, A_rowptr, A_col, A_val, P_rowptr, P_col,
                   P0_val, np.ones((n, 1)), np.sqrt(size)[:, None].copy(), iters,
                   {"kind": "ring1d", "n": n, "agg": agg, "sigma": sigma, "seed": seed})


def aniso3d(N: int = 160, eps: float = 1e-3, agg: int = 2, iters: int = 15) -> Problem:
    """3D 7-point anisotropic Poisson (coupling eps in z), homogeneous
    Dirichlet boundary eliminated: diagonal 4 + 2 eps, off-diagonals -1 in
    x and y and -eps in z."""
    dims = (N, N, N)
    offs = _stencil_offsets(3)
    nb, ok = _neighbour_table(dims, offs)
    row = np.array([-eps if o[2] != 0 else (4.0 + 2.0 * eps if o == (0, 0, 0) else -1.0)
                    for o in offs])
    vals = np.broadcast_to(row[None, :], nb.shape)
    return _scalar_problem(f"aniso3d_{N}", dims, nb, ok, vals, agg, iters,
                           {"kind": "aniso3d", "N": N, "agg": agg, "eps": eps})


# ---------------------------------------------------------------------------
# 3D linear elasticity, trilinear hexahedra
# ---------------------------------------------------------------------------
def _hex8_stiffness(nu: float, h: float) -> np.ndarray:
    """24 x 24 stiffness of a cube of side h (E = 1), 2x2x2 Gauss rule.

    Local node L = lx + 2 ly + 4 lz, local dof 3 L + component."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(3) * mu
    xi_n = np.array([[2 * (L & 1) - 1, 2 * ((L >> 1) & 1) - 1, 2 * ((L >> 2) & 1) - 1]
                     for L in range(8)], dtype=np.float64)
    gp = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for a in gp:
        for b in gp:
            for c in gp:
                q = np.array([a, b, c])
                dN = np.empty((8, 3))
                for L in range(8):
                    f = 1 + xi_n[L] * q
                    dN[L, 0] = xi_n[L, 0] * f[1] * f[2] / 8
                    dN[L, 1] = xi_n[L, 1] * f[0] * f[2] / 8
                    dN[L, 2] = xi_n[L, 2] * f[0] * f[1] / 8
                dN *= 2.0 / h          # d(xi)/dx = 2 / h
                Bm = np.zeros((6, 24))
                for L in range(8):
                    dx, dy, dz = dN[L]
                    Bm[0, 3 * L] = dx
                    Bm[1, 3 * L + 1] = dy
                    Bm[2, 3 * L + 2] = dz
                    Bm[3, 3 * L + 1], Bm[3, 3 * L + 2] = dz, dy
                    Bm[4, 3 * L], Bm[4, 3 * L + 2] = dz, dx
                    Bm[5, 3 * L], Bm[5, 3 * L + 1] = dy, dx
                K += Bm.T @ D @ Bm * (h / 2) ** 3
    return K


def elasticity3d(N: int = 64, nu: float = 0.3, agg: int = 3, sigma: float = 0.0,
                 seed: int = 5, iters: int = 20) -> Problem:
    """Q1 linear elasticity on an N^3 node grid of the unit cube, pure
    Neumann boundary (no dof eliminated), node-interleaved dofs
    (3 * node + component).  Young's modulus is 1, or exp(sigma * xi_e) per
    element when sigma > 0.  The near kernel is the 6 rigid-body modes
    [tx, ty, tz, (-y, x, 0), (0, -z, y), (z, 0, -x)] at centred coordinates in
    [-1/2, 1/2]; aggregates are agg^3 node blocks with the remainder merged
    into the last one; P0 and B_c come from a thin QR of B on each aggregate
    (B(dofs_a, :) = Q_a R_a, diag(R_a) > 0; P0 block = Q_a, B_c rows = R_a)."""
    h = 1.0 / (N - 1)
    Kref = _hex8_stiffness(nu, h)
    ne = N - 1
    if sigma > 0:
        Ee = np.exp(sigma * normal(seed, ne ** 3)).reshape(ne, ne, ne)  # [ez, ey, ex]
    else:
        Ee = np.ones((ne, ne, ne))
    Epad = np.zeros((N + 1, N + 1, N + 1))
    Epad[1:N, 1:N, 1:N] = Ee
    nn = N ** 3
    # block values vals[node, d, i, j]; d runs over the 27 offsets with dx fastest
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    vals = np.zeros((N, N, N, 27, 3, 3))  # axes [z, y, x, d, i, j]
    for di, (dx, dy, dz) in enumerate(offs):
        for lz in (0, 1):
            for ly in (0, 1):
                for lx in (0, 1):
                    mx, my, mz = lx + dx, ly + dy, lz + dz
                    if not (0 <= mx <= 1 and 0 <= my <= 1 and 0 <= mz <= 1):
                        continue
                    La = lx + 2 * ly + 4 * lz
                    Lb = mx + 2 * my + 4 * mz
                    blk = Kref[3 * La:3 * La + 3, 3 * Lb:3 * Lb + 3]
                    # element e = node - (lx, ly, lz); Epad is shifted by one
                    Ew = Epad[1 - lz:N + 1 - lz, 1 - ly:N + 1 - ly, 1 - lx:N + 1 - lx]
                    vals[:, :, :, di] += Ew[..., None, None] * blk
    vals = vals.reshape(nn, 27, 3, 3)
    nb, ok = _neighbour_table((N, N, N), offs)
    # rows (node, i), entries (d, j): reorder to [node, i, d, j]
    V = np.ascontiguousarray(vals.transpose(0, 2, 1, 3))
    colmat = (3 * nb)[:, None, :, None] + np.arange(3)[None, None, None, :]
    colmat = np.broadcast_to(colmat, V.shape)
    valid = np.broadcast_to(ok[:, None, :, None], V.shape)
    cnt = ok.sum(axis=1) * 3
    A_rowptr = np.zeros(3 * nn + 1, dtype=np.int64)
    np.cumsum(np.repeat(cnt, 3), out=A_rowptr[1:])
    A_col = colmat[valid].astype(np.int32)
    A_val = np.ascontiguousarray(V[valid])
    del V, colmat, valid, vals

    # rigid-body modes at centred, unit-scaled coordinates
    x, y, z = _grid_coords((N, N, N))
    xs, ys, zs = x * h - 0.5, y * h - 0.5, z * h - 0.5
    n = 3 * nn
    B = np.zeros((n, 6))
    B[0::3, 0] = 1.0
    B[1::3, 1] = 1.0
    B[2::3, 2] = 1.0
    B[0::3, 3], B[1::3, 3] = -ys, xs
    B[1::3, 4], B[2::3, 4] = -zs, ys
    B[0::3, 5], B[2::3, 5] = zs, -xs

    # aggregates of agg^3 nodes
    node_agg, nagg = _scalar_aggregates((N, N, N), agg)
    nc = 6 * nagg
    order = np.argsort(node_agg, kind="stable")  # nodes grouped by aggregate, ascending id
    sizes = np.bincount(node_agg, minlength=nagg)
    starts = np.zeros(nagg + 1, dtype=np.int64)
    np.cumsum(sizes, out=starts[1:])
    local = np.empty(nn, dtype=np.int64)
    local[order] = np.arange(nn) - starts[node_agg[order]]
    P0_rows = np.empty((n, 6))
    Bc = np.empty((nc, 6))
    for s in np.unique(sizes):
        aggs = np.nonzero(sizes == s)[0]
        nodes = order[(starts[aggs][:, None] + np.arange(s)[None, :])]  # [na, s]
        dofs = (3 * nodes[:, :, None] + np.arange(3)).reshape(len(aggs), 3 * s)
        Q, R = np.linalg.qr(B[dofs])
        sg = np.sign(np.diagonal(R, axis1=1, axis2=2))
        sg[sg == 0] = 1.0
        Q = Q * sg[:, None, :]
        R = R * sg[:, :, None]
        P0_rows[dofs.reshape(-1)] = Q.reshape(-1, 6)
        Bc[(6 * aggs[:, None] + np.arange(6)).reshape(-1)] = R.reshape(-1, 6)

    # pattern of A @ P0: aggregates of all 27 neighbours, 6 columns each
    g, keep = _pattern_from_neighbours(nb, ok, node_agg)
    node_cnt = keep.sum(axis=1)
    P_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.repeat(6 * node_cnt, 3), out=P_rowptr[1:])
    node_cols = (6 * g[:, :, None] + np.arange(6)).reshape(nn, -1)
    node_keep = np.repeat(keep, 6, axis=1)
    cols3 = np.broadcast_to(node_cols[:, None, :], (nn, 3, node_cols.shape[1]))
    keep3 = np.broadcast_to(node_keep[:, None, :], cols3.shape)
    P_col = cols3[keep3].astype(np.int32)
    rows = np.repeat(np.arange(n), np.diff(P_rowptr))
    own = node_agg[rows // 3]
    inblk = (P_col // 6) == own
    P0_val = np.where(inblk, P0_rows[rows, P_col % 6], 0.0)
    return Problem(f"elast3d_{N}", n, int(nc), 6, A_rowptr.astype(np.int32), A_col, A_val,
                   P_rowptr.astype(np.int32), P_col, P0_val, B, Bc, iters,
                   {"kind": "elasticity", "N": N, "agg": agg, "nu": nu, "sigma": sigma,
                    "seed": seed})


# ---------------------------------------------------------------------------
# random small problems for edge cases
# ---------------------------------------------------------------------------
def random_problem(n: int = 40, nc: int = 12, k: int = 1, a_per_row: int = 4,
                   p_per_row: int = 5, seed: int = 0, empty_p_rows=(),
                   wide_rows=(), wide: int = 40) -> Problem:
    """Random symmetric, strictly diagonally dominant A and a random sorted
    pattern for P with at least k entries per row (apart from
    ``empty_p_rows``), rows in ``wide_rows`` get ``wide`` entries (capped at
    nc).  P0 and B are random; P0 does not satisfy the constraint, so the
    set-up correction has work to do."""
    u = uniform01(seed, 8 * n * (a_per_row + p_per_row + wide + k + 8) + 64)
    pos = 0

    def take(m):
        nonlocal pos
        out = u[pos:pos + m]
        pos += m
        return out

    rows, cols = [], []
    for i in range(n):
        c = np.unique((take(a_per_row) * n).astype(np.int64))
        c = c[c != i]
        rows += [i] * len(c)
        cols += list(c)
    r = np.array(rows + cols, dtype=np.int64)
    c = np.array(cols + rows, dtype=np.int64)
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    # symmetric values: both entries of a (min, max) pair share one draw
    pair = np.minimum(r, c) * n + np.maximum(r, c)
    _, inv = np.unique(pair, return_inverse=True)
    pv = -(0.1 + take(int(inv.max()) + 1 if len(inv) else 0))
    off = pv[inv]
    diag = np.zeros(n)
    np.add.at(diag, r, -off)
    diag += 0.5 + take(n)
    allr = np.concatenate([r, np.arange(n)])
    allc = np.concatenate([c, np.arange(n)])
    allv = np.concatenate([off, diag])
    o = np.lexsort((allc, allr))
    allr, allc, allv = allr[o], allc[o], allv[o]
    A_rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(allr, minlength=n), out=A_rowptr[1:])
    prow = []
    for i in range(n):
        if i in empty_p_rows:
            prow.append(np.zeros(0, dtype=np.int64))
            continue
        m = min(nc, wide if i in wide_rows else p_per_row)
        m = max(m, min(k, nc))
        perm = np.argsort(take(nc))[:m]
        prow.append(np.sort(perm))
    P_rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum([len(p) for p in prow], out=P_rowptr[1:])
    P_col = np.concatenate(prow).astype(np.int32)
    P0_val = take(len(P_col)) - 0.5
    B = take(n * k).reshape(n, k) + 0.5
    Bc = take(nc * k).reshape(nc, k) - 0.5
    return Problem(f"random_{n}_{nc}_{k}_{seed}", n, nc, k, A_rowptr, allc.astype(np.int32),
                   allv.astype(np.float64), P_rowptr, P_col, P0_val, B, Bc, 10,
                   {"kind": "random", "seed": seed})


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# classical form P = [W; I] (Section 2): C/F splitting, strength of
# connection, pattern growth S^k P0 (Eq. (enlPatt))
# ---------------------------------------------------------------------------
def strength(prob: Problem, theta: float = 0.25):
    """Classical strength of connection of an M-matrix-like A: j is a strong
    dependency of i if -a_ij >= theta max_(l != i) (-a_il).  Returns S as a
    boolean CSR (rowptr, col) without the diagonal, columns sorted."""
    n = prob.n
    rows = np.repeat(np.arange(n), np.diff(prob.A_rowptr))
    off = prob.A_col != rows
    neg = np.where(off, -prob.A_val, -np.inf)
    mx = np.full(n, -np.inf)
    np.maximum.at(mx, rows, neg)
    strong = off & (neg >= theta * mx[rows]) & (neg > 0)
    cnt = np.bincount(rows[strong], minlength=n)
    Sp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=Sp[1:])
    return Sp, prob.A_col[strong].astype(np.int64)


def cf_split(prob: Problem, Sp, Sj, seed: int = 7):
    """C/F splitting: a maximal independent set of the symmetrised strength
    graph, chosen in rounds (a point joins C when its priority beats every
    undecided neighbour; its neighbours become F), with priorities = number
    of points that depend strongly on it plus a seeded fraction.  Returns a
    boolean C mask."""
    n = prob.n
    rows = np.repeat(np.arange(n), np.diff(Sp))
    ei = np.concatenate([rows, Sj])
    ej = np.concatenate([Sj, rows])
    pri = np.bincount(Sj, minlength=n).astype(np.float64) + uniform01(seed, n)
    state = np.zeros(n, dtype=np.int8)  # 0 undecided, 1 C, 2 F
    state[np.bincount(ei, minlength=n) == 0] = 1  # isolated points are C
    while (state == 0).any():
        und = state == 0
        live = und[ei] & und[ej]
        best = np.full(n, -1.0)
        np.maximum.at(best, ei[live], pri[ej[live]])
        newc = und & (pri > best)
        state[newc] = 1
        nb = ej[newc[ei]]
        state[nb[state[nb] == 0]] = 2
    return state == 1


def classical(base: Problem, theta: float = 0.25, grow: int = 1, seed: int = 7,
              iters: int = 10) -> Problem:
    """The classical form P = [W; I] on the operator of ``base`` (k = 1,
    near kernel B = 1): C/F splitting from the strength of connection S,
    tentative pattern P0 = identity on C rows and the strong C dependencies
    on F rows, grown to P = S^grow P0 on the F rows (Eq. (enlPatt)), C rows
    kept as identity rows.  P0 values: 1 on C rows, equal weights summing to
    1 on an F row's strong C dependencies, so that P0 B_c = B with B_c = B(C)
    = 1.  A C row has one entry, so its constraint fixes it: only W moves,
    and mask_P(A P0) carries f = -A_fc of Eq. (11blk) into the residual."""
    n = base.n
    Sp, Sj = strength(base, theta)
    isC = cf_split(base, Sp, Sj, seed)
    cidx = np.full(n, -1, dtype=np.int64)
    cidx[isC] = np.arange(int(isC.sum()))
    nc = int(isC.sum())
    rows = np.repeat(np.arange(n), np.diff(Sp))
    # P0 pattern: C rows {own}, F rows {strong C dependencies}
    sc = isC[Sj]
    p0_rows = np.concatenate([np.nonzero(isC)[0], rows[sc]])
    p0_cols = np.concatenate([cidx[isC], cidx[Sj[sc]]])
    f_nc = np.bincount(rows[sc], minlength=n)
    lone = (~isC) & (f_nc == 0)  # F points with no strong C dependency: any C neighbour
    if lone.any():
        arow = np.repeat(np.arange(n), np.diff(base.A_rowptr))
        m = lone[arow] & isC[base.A_col] & (base.A_col != arow)
        p0_rows = np.concatenate([p0_rows, arow[m]])
        p0_cols = np.concatenate([p0_cols, cidx[base.A_col[m]]])
    key = np.unique(p0_rows * nc + p0_cols)
    p0_rows, p0_cols = key // nc, key % nc
    # growth on F rows: row i gathers the P0 columns of its strong dependencies
    pat_r, pat_c = p0_rows, p0_cols
    for _ in range(grow):
        ptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(np.bincount(pat_r, minlength=n), out=ptr[1:])
        fr = ~isC[rows]
        src_i, src_l = rows[fr], Sj[fr]
        cnt = ptr[src_l + 1] - ptr[src_l]
        rep_i = np.repeat(src_i, cnt)
        starts = np.repeat(ptr[src_l], cnt)
        offs = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        new_c = pat_c[starts + offs]
        key = np.unique(np.concatenate([pat_r * nc + pat_c, rep_i * nc + new_c]))
        pat_r, pat_c = key // nc, key % nc
    P_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(pat_r, minlength=n), out=P_rowptr[1:])
    P_col = pat_c.astype(np.int32)
    # P0 values on the grown pattern
    own = np.zeros(len(pat_r))
    in0 = np.isin(pat_r * nc + pat_c, p0_rows * nc + p0_cols)
    cnt0 = np.bincount(p0_rows, minlength=n).astype(np.float64)
    own[in0] = 1.0 / cnt0[pat_r[in0]]
    return Problem(f"classical_{base.name}", n, nc, 1, base.A_rowptr, base.A_col, base.A_val,
                   P_rowptr.astype(np.int32), P_col, own, np.ones((n, 1)), np.ones((nc, 1)),
                   iters, {"kind": "classical", "base": base.name, "theta": theta,
                           "grow": grow, "seed": seed, "cpoints": np.nonzero(isC)[0]})


CONFIG_NAMES = {
    1: "2D 5-point Poisson 64x64, k=1, 2x2 aggregates, 10 iterations, FP64",
    2: "3D 7-point FV diffusion 128^3, log-normal kappa (sigma=2, seed 2), k=1, "
       "3x3x3 aggregates, 20 iterations, FP64 vs mixed",
    3: "3D Q1 elasticity 64^3 nodes, E=1, nu=0.3, 6 RBMs, 3^3-node aggregates, 20 iterations",
    4: "3D anisotropic 7-point Poisson 160^3 (eps=1e-3 in z), k=1, 2x2x2 aggregates, "
       "15 iterations + backward",
    5: "3D heterogeneous Q1 elasticity 96^3 nodes (E log-normal sigma=1.5, seed 5), "
       "nu=0.25, 6 RBMs, 3^3-node aggregates, 30 iterations + backward",
}


def config(cfg: int, scale: float = 1.0) -> Problem:
    """Workload ``cfg`` (1-5).  ``scale`` < 1 shrinks the grid (same recipe)
    for tests that the oracle must finish in seconds."""
    def sz(n, lo):
        return max(lo, int(round(n * scale)))
    if cfg == 1:
        return poisson2d(sz(64, 4), 2, 10)
    if cfg == 2:
        return diffusion3d_fv(sz(128, 6), 3, 2.0, 2, 20)
    if cfg == 3:
        return elasticity3d(sz(64, 6), 0.3, 3, 0.0, 5, 20)
    if cfg == 4:
        return aniso3d(sz(160, 4), 1e-3, 2, 15)
    if cfg == 5:
        return elasticity3d(sz(96, 6), 0.25, 3, 1.5, 5, 30)
    raise ValueError(f"unknown workload {cfg}")
