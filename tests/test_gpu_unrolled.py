"""The gradient of exactly n iterations (the unrolled adjoint, checkpointed
every ceil(sqrt(n)) steps) on the GPU against the PyTorch-autograd oracle of
the same n-step map, and at a larger size against central differences of
the C oracle's n-step forward."""
import numpy as np
import pytest

from oracle import unrolled_torch as UT
from oracle.oracle import Oracle
from paper_2208_02995_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_02995_gb300 import build
    build.build()


PROBS = [I.poisson2d(7, 2), I.diffusion3d_fv(6, 3), I.random_problem(30, 10, 1, seed=1),
         I.random_problem(20, 9, 2, p_per_row=5, seed=8), I.elasticity3d(4, 0.3, 2),
         I.classical(I.poisson2d(7, 2))]


@pytest.mark.parametrize("prob", PROBS, ids=[p.name for p in PROBS])
@pytest.mark.parametrize("n_iters", [1, 4, 7])
def test_unrolled_matches_autograd(prob, n_iters):
    from paper_2208_02995_gb300.emin import Context
    dLdP = np.random.default_rng(2).standard_normal(prob.nnz_p)
    _, gA, gB = UT.gradient(prob, dLdP, n_iters)
    c = Context(prob)
    dA, dB = c.backward_unrolled(dLdP, n_iters)
    assert np.linalg.norm(dA - gA) <= 1e-9 * np.linalg.norm(gA)
    assert np.linalg.norm(dB - gB) <= 1e-9 * max(np.linalg.norm(gB), 1e-300)


def test_unrolled_fd_fv12():
    """12^3 FV diffusion (1,728 rows), 10 steps: the gradient against central
    differences of the C oracle's 10-step forward on seeded entries."""
    from paper_2208_02995_gb300.emin import Context
    prob = I.diffusion3d_fv(12, 3)
    n_iters = 10
    rng = np.random.default_rng(4)
    dLdP = rng.standard_normal(prob.nnz_p)
    dA, dB = Context(prob).backward_unrolled(dLdP, n_iters)

    def L(A_val=None, B=None):
        p = I.Problem(prob.name, prob.n, prob.nc, prob.k, prob.A_rowptr, prob.A_col,
                      prob.A_val if A_val is None else A_val, prob.P_rowptr, prob.P_col,
                      prob.P0_val, prob.B if B is None else B, prob.Bc)
        return float(dLdP @ Oracle(p).minimize(n_iters)["P"])

    for e in rng.choice(prob.nnz_a, 8, replace=False):
        h = 1e-6 * max(abs(prob.A_val[e]), 1.0)
        Ap, Am = prob.A_val.copy(), prob.A_val.copy()
        Ap[e] += h
        Am[e] -= h
        fd = (L(A_val=Ap) - L(A_val=Am)) / (2 * h)
        assert abs(fd - dA[e]) <= 1e-6 * max(abs(dA[e]), 1e-3 * np.abs(dA).max()), e
    for idx in rng.choice(prob.n, 4, replace=False):
        h = 1e-6
        Bp, Bm = prob.B.copy(), prob.B.copy()
        Bp[idx, 0] += h
        Bm[idx, 0] -= h
        fd = (L(B=Bp) - L(B=Bm)) / (2 * h)
        assert abs(fd - dB[idx, 0]) <= 1e-6 * max(abs(dB[idx, 0]), 1e-3 * np.abs(dB).max())


def test_unrolled_rejects_mixed_and_sgs():
    from paper_2208_02995_gb300.emin import Context, EminError
    prob = I.poisson2d(8, 2)
    for kw in ({"precision": "mixed"}, {"precond": "sgs"}):
        c = Context(prob, **kw)
        with pytest.raises(EminError):
            c.backward_unrolled(np.ones(prob.nnz_p), 3)
