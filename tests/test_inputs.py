"""The seeded synthetic inputs: sizes, symmetry, boundary conditions, and the
near-kernel constraint satisfied by the tentative prolongation."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2208_02995_gb300 import inputs as I


def _A(p):
    return sp.csr_matrix((p.A_val, p.A_col, p.A_rowptr), shape=(p.n, p.n))


def _P(p, vals=None):
    v = p.P0_val if vals is None else vals
    return sp.csr_matrix((v, p.P_col, p.P_rowptr), shape=(p.n, p.nc))


def _check_csr(rowptr, col, ncols):
    assert rowptr[0] == 0 and np.all(np.diff(rowptr) >= 0)
    for i in range(len(rowptr) - 1):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0), f"row {i} not sorted/unique"
    assert col.min(initial=0) >= 0 and col.max(initial=0) < ncols


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    z = I.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_moments():
    x = I.normal(7, 200001)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    assert np.array_equal(I.normal(7, 11), I.normal(7, 11))


# exact sizes of the five workloads (n, nnz(A), n_c, nnz(P), max row of P)
SIZES = {
    1: (4096, 20224, 1024, 12032, 3),
    2: (2097152, 14581760, 74088, 6127616, 4),
    4: (4096000, 28518400, 512000, 16230400, 4),
    3: (786432, 61731000, 55566, 20247552, 48),
}


@pytest.mark.parametrize("cfg", [1, 2, 4, 3])
def test_config_sizes(cfg):
    p = I.config(cfg)
    n, nnza, nc, nnzp, mmax = SIZES[cfg]
    assert (p.n, p.nnz_a, p.nc, p.nnz_p) == (n, nnza, nc, nnzp)
    assert int(np.diff(p.P_rowptr).max()) == mmax


@pytest.mark.parametrize("prob", [
    I.poisson2d(12, 2), I.diffusion3d_fv(8, 3), I.aniso3d(6, 1e-3, 2),
    I.elasticity3d(5, 0.3, 2), I.elasticity3d(6, 0.25, 3, 1.5, 5),
    I.random_problem(40, 12, 2, seed=3), I.ring1d(41, 2),
], ids=lambda p: p.name)
def test_structure(prob):
    A = _A(prob)
    _check_csr(prob.A_rowptr, prob.A_col, prob.n)
    _check_csr(prob.P_rowptr, prob.P_col, prob.nc)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    assert np.all(A.diagonal() > 0)
    # the pattern of P contains the pattern of P0
    nz0 = prob.P0_val != 0
    assert nz0.any()
    if prob.meta["kind"] != "random":
        # pattern of P = structural pattern of A @ P0
        A1 = sp.csr_matrix((np.ones_like(prob.A_val), prob.A_col, prob.A_rowptr), shape=A.shape)
        rows = np.repeat(np.arange(prob.n), np.diff(prob.P_rowptr))
        struct0 = sp.csr_matrix((np.ones(nz0.sum()), (rows[nz0], prob.P_col[nz0])),
                                shape=(prob.n, prob.nc))
        if prob.k > 1:  # P0 blocks are structurally dense Q_a blocks
            own = rows // 3
            struct0 = None
        if struct0 is not None:
            S = (A1 @ struct0).tocsr()
            S.sort_indices()
            assert np.array_equal(S.indptr, prob.P_rowptr)
            assert np.array_equal(S.indices, prob.P_col)
        # P0 B_c = B
        err = np.abs(_P(prob) @ prob.Bc - prob.B).max()
        assert err < 1e-13


def test_neumann_kernels():
    fv = I.diffusion3d_fv(10, 3)
    assert np.abs(_A(fv) @ np.ones(fv.n)).max() < 1e-10 * np.abs(fv.A_val).max()
    el = I.elasticity3d(6, 0.3, 3)
    AB = _A(el) @ el.B
    assert np.abs(AB).max() < 1e-12 * np.abs(el.A_val).max()
    het = I.elasticity3d(6, 0.25, 3, 1.5, 5)
    assert np.abs(_A(het) @ het.B).max() < 1e-12 * np.abs(het.A_val).max()
    ring = I.ring1d(41, 2)
    assert np.abs(_A(ring) @ np.ones(ring.n)).max() < 1e-14 * np.abs(ring.A_val).max()
    assert _A(ring)[0, ring.n - 1] != 0  # the wrap-around coupling


def test_elasticity_blocks():
    el = I.elasticity3d(7, 0.3, 3)
    # rows of one node share a pattern in A and in P; P's columns come in
    # whole 6-column aggregate blocks
    for v in range(el.n // 3):
        a = [el.A_col[el.A_rowptr[3 * v + i]:el.A_rowptr[3 * v + i + 1]] for i in range(3)]
        p = [el.P_col[el.P_rowptr[3 * v + i]:el.P_rowptr[3 * v + i + 1]] for i in range(3)]
        assert np.array_equal(a[0], a[1]) and np.array_equal(a[0], a[2])
        assert np.array_equal(p[0], p[1]) and np.array_equal(p[0], p[2])
        assert len(p[0]) % 6 == 0 and np.all(p[0][::6] % 6 == 0)
    # P0 block of an aggregate has orthonormal columns (thin QR)
    P = _P(el).toarray()
    G = P.T @ P
    assert np.abs(G - np.eye(el.nc)).max() < 1e-12


@pytest.mark.parametrize("base", [I.poisson2d(12, 2), I.aniso3d(7, 1e-3, 2),
                                  I.diffusion3d_fv(9, 3)], ids=lambda p: p.name)
def test_classical_form(base):
    """P = [W; I]: C rows are identity rows (one entry, the point's own
    coarse index, value 1), every F row of P0 sums to 1 (P0 B_c = B with
    B = B_c = 1), and the F rows' pattern is the boolean product S P0_bar
    of the strength matrix with the tentative pattern (Eq. (enlPatt))."""
    p = I.classical(base, theta=0.25, grow=1)
    n, nc = p.n, p.nc
    C = p.meta["cpoints"]
    isC = np.zeros(n, dtype=bool)
    isC[C] = True
    m = np.diff(p.P_rowptr)
    assert np.all(m[isC] == 1)
    assert np.array_equal(p.P_col[p.P_rowptr[C]], np.arange(nc))
    assert np.all(p.P0_val[p.P_rowptr[C]] == 1.0)
    assert np.all(m[~isC] >= 1)
    rows = np.repeat(np.arange(n), m)
    assert np.allclose(np.bincount(rows, weights=p.P0_val, minlength=n), 1.0)
    # strength: -a_ij >= theta max_l -a_il (dense re-computation)
    A = _A(p).toarray()
    Sp, Sj = I.strength(p, 0.25)
    S = np.zeros((n, n), dtype=bool)
    S[np.repeat(np.arange(n), np.diff(Sp)), Sj] = True
    for i in range(n):
        off = -A[i].copy()
        off[i] = -np.inf
        mx = off.max()
        ref = (off >= 0.25 * mx) & (off > 0)
        assert np.array_equal(S[i], ref)
    # pattern of the F rows = S P0_bar (dense boolean) united with P0_bar
    P0bar = np.zeros((n, nc), dtype=bool)
    P0bar[rows[p.P0_val != 0], p.P_col[p.P0_val != 0]] = True
    grown = (S.astype(int) @ P0bar.astype(int) > 0) | P0bar
    Pbar = np.zeros((n, nc), dtype=bool)
    Pbar[rows, p.P_col] = True
    assert np.array_equal(Pbar[~isC], grown[~isC])
