"""Gradient of exactly n iterations of the minimisation, by PyTorch autograd.

TEST INFRASTRUCTURE (see ``oracle.py``).  Plain PyTorch on the CPU in
float64: Algorithm 2's least-norm correction of P0 and n steps of Algorithm 3
with the Jacobi preconditioner, written out densely (K as the nnz(P) x
nnz(P) matrix of Eqs. (minblk), (11blk); Pi_B = I - Q Q^T per row of P), and
differentiated by reverse-mode autograd with respect to the stored values of
A and the fine near-kernel block B (B_c held fixed).  This is the reference
for the library's unrolled adjoint: the same function, differentiated by a
different route.  Small problems only (dense nnz(P) x nnz(P) matrices).
"""
from __future__ import annotations

import numpy as np
import torch


def _structures(prob):
    n, nc, k = prob.n, prob.nc, prob.k
    Pp = np.asarray(prob.P_rowptr)
    rows = np.repeat(np.arange(n), np.diff(Pp))
    cols = np.asarray(prob.P_col)
    arow = np.repeat(np.arange(n), np.diff(prob.A_rowptr))
    return n, nc, k, Pp, rows, cols, arow


def forward(prob, A_val, B, n_iters):
    """P after Algorithm 2 and n_iters steps of Algorithm 3 (Jacobi), as a
    differentiable function of A_val (nnz(A)) and B (n x k) in float64."""
    n, nc, k, Pp, rows, cols, arow = _structures(prob)
    nnz = len(cols)
    A = torch.zeros((n, n), dtype=torch.float64)
    A = A.index_put((torch.as_tensor(arow), torch.as_tensor(np.asarray(prob.A_col))), A_val)
    same = torch.as_tensor(cols[:, None] == cols[None, :])
    r_t = torch.as_tensor(rows)
    K = torch.where(same, A[r_t[:, None], r_t[None, :]], torch.zeros((), dtype=torch.float64))
    Bc = torch.as_tensor(np.asarray(prob.Bc), dtype=torch.float64)
    P0_in = torch.as_tensor(np.asarray(prob.P0_val), dtype=torch.float64)
    # per row of P: B_i = B_c(J_i, :), least-norm correction and projector
    p0_parts, Qs = [], []
    for i in range(n):
        s0, s1 = int(Pp[i]), int(Pp[i + 1])
        Bi = Bc[torch.as_tensor(cols[s0:s1])]
        G = Bi.T @ Bi
        res = B[i] - Bi.T @ P0_in[s0:s1]
        p0_parts.append(P0_in[s0:s1] + Bi @ torch.linalg.solve(G, res))
        Q, _ = torch.linalg.qr(Bi)
        Qs.append(Q)
    p0 = torch.cat(p0_parts)

    def project(x):
        out = []
        for i in range(n):
            s0, s1 = int(Pp[i]), int(Pp[i + 1])
            xi = x[s0:s1]
            out.append(xi - Qs[i] @ (Qs[i].T @ xi))
        return torch.cat(out) if out else x

    dinv = 1.0 / torch.diagonal(A)[r_t]
    r = -project(K @ p0)
    dw = torch.zeros(nnz, dtype=torch.float64)
    y = None
    gamma_old = None
    for it in range(n_iters):
        z = project(dinv * r)
        gamma = r @ z
        y = z if it == 0 else z + (gamma / gamma_old) * y
        gamma_old = gamma
        yb = project(K @ y)
        alpha = gamma / (y @ yb)
        dw = dw + alpha * y
        r = r - alpha * yb
    return p0 + dw


def gradient(prob, dLdP, n_iters):
    """(dL/dA values, dL/dB) of L = <dLdP, P(A, B)> with P the n-iteration
    forward: the vector-Jacobian product of ``forward``."""
    A_val = torch.tensor(np.asarray(prob.A_val), dtype=torch.float64, requires_grad=True)
    B = torch.tensor(np.asarray(prob.B), dtype=torch.float64, requires_grad=True)
    P = forward(prob, A_val, B, n_iters)
    L = P @ torch.as_tensor(np.asarray(dLdP), dtype=torch.float64)
    gA, gB = torch.autograd.grad(L, [A_val, B])
    return P.detach().numpy(), gA.numpy(), gB.numpy()
