"""Pins of the unrolled-iteration gradient oracle (PyTorch autograd through
n steps of Algorithms 2-3): its forward equals the C oracle's n-step result,
its gradient equals central differences of the C oracle's forward (a
different implementation), and for many steps it approaches the implicit
adjoint of the converged minimiser."""
import numpy as np
import pytest

from oracle import unrolled_torch as UT
from oracle.oracle import Oracle
from paper_2208_02995_gb300 import inputs as I

PROBS = [I.poisson2d(5, 2), I.random_problem(14, 5, 1, seed=2),
         I.random_problem(12, 6, 2, p_per_row=4, seed=8), I.elasticity3d(4, 0.3, 2)]
IDS = [p.name for p in PROBS]


def _with(prob, A_val=None, B=None):
    return I.Problem(prob.name, prob.n, prob.nc, prob.k, prob.A_rowptr, prob.A_col,
                     prob.A_val if A_val is None else A_val, prob.P_rowptr, prob.P_col,
                     prob.P0_val, prob.B if B is None else B, prob.Bc, prob.iters, prob.meta)


@pytest.mark.parametrize("prob", PROBS, ids=IDS)
def test_unrolled_forward_equals_oracle(prob):
    import torch
    for n in (1, 3, 6):
        P = UT.forward(prob, torch.tensor(prob.A_val), torch.tensor(prob.B), n).numpy()
        ref = Oracle(prob).minimize(n)["P"]
        assert np.abs(P - ref).max() <= 1e-12 * max(1, np.abs(ref).max()), n


@pytest.mark.parametrize("prob", PROBS, ids=IDS)
def test_unrolled_gradient_is_finite_difference_of_oracle(prob):
    n = 4
    rng = np.random.default_rng(3)
    dLdP = rng.standard_normal(prob.nnz_p)
    _, gA, gB = UT.gradient(prob, dLdP, n)

    def L(p):
        return float(dLdP @ Oracle(p).minimize(n)["P"])

    for e in rng.choice(prob.nnz_a, 6, replace=False):
        h = 1e-6 * max(abs(prob.A_val[e]), 1.0)
        Ap, Am = prob.A_val.copy(), prob.A_val.copy()
        Ap[e] += h
        Am[e] -= h
        fd = (L(_with(prob, A_val=Ap)) - L(_with(prob, A_val=Am))) / (2 * h)
        assert abs(fd - gA[e]) <= 1e-6 * max(abs(gA[e]), np.abs(gA).max() * 1e-3), e
    for idx in rng.choice(prob.n * prob.k, 4, replace=False):
        i, c = divmod(int(idx), prob.k)
        h = 1e-6 * max(abs(prob.B[i, c]), 1.0)
        Bp, Bm = prob.B.copy(), prob.B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (L(_with(prob, B=Bp)) - L(_with(prob, B=Bm))) / (2 * h)
        assert abs(fd - gB[i, c]) <= 1e-6 * max(abs(gB[i, c]), np.abs(gB).max() * 1e-3), (i, c)


def test_unrolled_gradient_approaches_implicit_adjoint():
    """Run to convergence, the n-step function's gradient becomes the
    gradient of the constrained minimiser (the implicit adjoint).  The C
    oracle converges in 10 steps here; 20 unrolled steps are past that but
    not yet deep into iterating on rounding noise (where the derivative of
    CG degrades: 4e-3 at 60 steps)."""
    prob = I.poisson2d(5, 2)
    o = Oracle(prob)
    P = o.minimize(200)["P"]
    dLdP = 2 * o.kprod(P) + 2 * P
    _, gA, gB = UT.gradient(prob, dLdP, 20)
    dA, dB, _, _ = o.backward(P, dLdP, 200)
    # the explicit term mask_A(P P^T) of d tr(P^T A P)/dA is not part of the VJP
    assert np.abs(gA - dA).max() <= 1e-5 * np.abs(dA).max()
    assert np.abs(gB - dB).max() <= 1e-6 * max(1, np.abs(dB).max())
