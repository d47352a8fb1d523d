"""PyTorch autograd wrappers of the library (marshalling only).

``EminSolve.apply(A_val, B, problem, n_iters, tol, adj_iters, adj_tol)``
    P* on P's pattern from the values of A and the fine near-kernel block B;
    its backward is the implicit adjoint of the constrained minimiser
    (``emin_backward``: one more restricted PCG with the same operator and the
    masked products mask_A(U P^T), mask_P(A U)).  The iterates are not kept:
    only the final P lives in the library context held by the graph.

``EminEnergy.apply(A_val, P_val, problem)``
    E = tr(P^T A P) = <P, mask_P(A P)> (Eq. (trace)) with its analytic
    backward dE/dP = 2 mask_P(A P) (A symmetric), dE/dA = mask_A(P P^T), all
    three formed by the library (``emin_energy_grad``).

The fixed data of a problem (patterns, P0, B_c) live in an ``EminProblem``.
Every computation runs in the CUDA library; tensors must be on the device.
"""
from __future__ import annotations

import torch

from .emin import Context


class EminProblem:
    """Fixed pattern data of one minimisation problem, as CUDA tensors:
    A's CSR pattern, P's pattern, the tentative P0, B_c, and a default B."""

    def __init__(self, n, nc, k, A_rowptr, A_col, P_rowptr, P_col, P0_val, B, Bc,
                 precision="fp64", device="cuda", precond="jacobi"):
        def t(x, dt):
            return torch.as_tensor(x).to(device=device, dtype=dt).contiguous()
        self.n, self.nc, self.k = int(n), int(nc), int(k)
        self.A_rowptr, self.A_col = t(A_rowptr, torch.int32), t(A_col, torch.int32)
        self.P_rowptr, self.P_col = t(P_rowptr, torch.int32), t(P_col, torch.int32)
        self.P0 = t(P0_val, torch.float64)
        self.B = t(B, torch.float64).reshape(self.n, self.k)
        self.Bc = t(Bc, torch.float64).reshape(self.nc, self.k)
        self.precision = precision
        self.precond = precond

    @classmethod
    def from_problem(cls, prob, precision="fp64", device="cuda", precond="jacobi"):
        return cls(prob.n, prob.nc, prob.k, prob.A_rowptr, prob.A_col, prob.P_rowptr,
                   prob.P_col, prob.P0_val, prob.B, prob.Bc, precision, device, precond)

    def context(self, A_val, B=None, precision=None):
        """A library context holding these values (stream: the current one)."""
        B = self.B if B is None else B
        precision = self.precision if precision is None else precision
        arrays = [self.A_rowptr, self.A_col, A_val.detach().contiguous().double(),
                  self.P_rowptr, self.P_col, self.P0,
                  B.detach().contiguous().double().reshape(self.n, self.k), self.Bc]
        return Context(n=self.n, nc=self.nc, k=self.k, arrays=arrays,
                       precision=precision, on_device=True, precond=self.precond)


class EminSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_val, B, problem, n_iters=200, tol=0.0, adj_iters=200, adj_tol=0.0):
        c = problem.context(A_val, B)
        c.iterate(int(n_iters), float(tol))
        P = torch.empty(problem.P_col.numel(), dtype=torch.float64, device=A_val.device)
        c.get_p(P)
        ctx.lib = c
        ctx.adj = (int(adj_iters), float(adj_tol))
        return P

    @staticmethod
    def backward(ctx, dP):
        dA, dB, _ = ctx.lib.backward(dP.detach().contiguous().double(), *ctx.adj)
        return dA, dB, None, None, None, None, None


class EminEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_val, P_val, problem):
        c = problem.context(A_val, precision="fp64")
        P = P_val.detach().contiguous().double()
        E, _, _ = c.energy_grad(P)
        ctx.save_for_backward(P)
        ctx.lib = c
        return torch.tensor(E, dtype=torch.float64, device=P.device)

    @staticmethod
    def backward(ctx, gE):
        (P,) = ctx.saved_tensors
        _, dP, dA = ctx.lib.energy_grad(P, float(gE), want_energy=False, want_dX=True,
                                        want_dA=True)
        return dA, dP, None
