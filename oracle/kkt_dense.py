"""Dense brute force of the constrained energy minimisation, for tiny inputs.

TEST INFRASTRUCTURE (see ``oracle.py``).  Everything here is written out
densely with NumPy so that it can be compared with the sparse oracle:

* ``dense_K``      K over the nnz(P) unknowns in CSR order: the entry of
                   P(i, c) couples with P(i', c) through A(i, i') (the block
                   A(I_c, I_c) of each column c, Eqs. (minblk), (11blk)).
* ``dense_C``      the block-diagonal constraint B~^T p = g (Eq. (Constr_Mat)),
                   one block B_c(J_i, :)^T per row i.
* ``kkt_solve``    the saddle-point system (sadsys), solved by
                   ``numpy.linalg.solve`` (``lstsq`` if singular).
* ``nullspace_pcg`` the null-space method the paper calls equivalent to the
                   restricted PCG (after Eq. (projSys)): CG on Z^T K Z with
                   preconditioner Z^T D_K^{-1} Z (or Z^T M_SGS^{-1} Z), Z from
                   a full QR of C^T.
* ``sgs_inverse``  (L + D)^{-T} D (L + D)^{-1} of K by dense triangular solves.
"""
from __future__ import annotations

import numpy as np


def entry_rows(prob):
    return np.repeat(np.arange(prob.n), np.diff(prob.P_rowptr))


def dense_A(prob):
    A = np.zeros((prob.n, prob.n))
    rows = np.repeat(np.arange(prob.n), np.diff(prob.A_rowptr))
    A[rows, prob.A_col] = prob.A_val
    return A


def dense_K(prob):
    A = dense_A(prob)
    r = entry_rows(prob)
    c = prob.P_col
    same = c[:, None] == c[None, :]
    return np.where(same, A[r[:, None], r[None, :]], 0.0)


def dense_C(prob):
    """k*n x nnz(P) constraint matrix: row (i, a) holds B_c(c_s, a) at entry s of row i."""
    k = prob.k
    C = np.zeros((prob.n * k, prob.nnz_p))
    r = entry_rows(prob)
    for a in range(k):
        C[r * k + a, np.arange(prob.nnz_p)] = prob.Bc[prob.P_col, a]
    return C


def kkt_solve(prob, K=None, g=None):
    """p minimising p^T K p subject to C p = g (g = vec B by default)."""
    K = dense_K(prob) if K is None else K
    C = dense_C(prob)
    g = prob.B.reshape(-1) if g is None else g
    m = C.shape[0]
    M = np.block([[2 * K, C.T], [C, np.zeros((m, m))]])
    rhs = np.concatenate([np.zeros(K.shape[0]), g])
    try:
        sol = np.linalg.solve(M, rhs)
    except np.linalg.LinAlgError:
        sol = np.linalg.lstsq(M, rhs, rcond=None)[0]
    return sol[:K.shape[0]], sol[K.shape[0]:]


def nullspace_basis(prob):
    C = dense_C(prob)
    Qf, Rf = np.linalg.qr(C.T, mode="complete")
    rank = np.linalg.matrix_rank(C)
    return Qf[:, rank:], Qf[:, :rank]


def sgs_inverse(K):
    """M_SGS^{-1} = (L + D)^{-T} D (L + D)^{-1} of K = L + D + L^T (Section 3.4),
    as a dense matrix, for p in K's own (row-wise) order."""
    LD = np.tril(K)
    D = np.diag(np.diag(K))
    Linv = np.linalg.solve(LD, np.eye(K.shape[0]))
    return Linv.T @ D @ Linv


def nullspace_pcg(prob, p0, maxit, precond="jacobi"):
    """Preconditioned CG on Z^T K Z x = -Z^T K p0 from x = 0, with the
    reduced preconditioner M^{-1} = Z^T D_K^{-1} Z (Jacobi, M_1) or
    Z^T M_SGS^{-1} Z (projected SGS, M_2).  Returns the iterates
    p0 + Z x_k (k = 0..maxit) and the energy decrements gamma_k alpha_k."""
    K = dense_K(prob)
    Z, _ = nullspace_basis(prob)
    d = np.diag(K)
    H = Z.T @ K @ Z
    if precond == "sgs":
        Minv = Z.T @ sgs_inverse(K) @ Z
    else:
        Minv = Z.T @ (Z / d[:, None])
    x = np.zeros(Z.shape[1])
    r = -Z.T @ (K @ p0)
    iters, dE = [p0.copy()], []
    y = None
    gold = None
    for it in range(maxit):
        z = Minv @ r
        g = r @ z
        if g == 0:
            break
        y = z.copy() if it == 0 else z + (g / gold) * y
        gold = g
        Hy = H @ y
        a = g / (y @ Hy)
        dE.append(g * a)
        x = x + a * y
        r = r - a * Hy
        iters.append(p0 + Z @ x)
    return iters, np.array(dE)


def energy(prob, p):
    """tr(P^T A P) from the dense A."""
    A = dense_A(prob)
    P = np.zeros((prob.n, prob.nc))
    P[entry_rows(prob), prob.P_col] = p
    return float(np.trace(P.T @ A @ P))
