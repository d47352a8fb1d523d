"""The implicit adjoint and the autograd layer against the oracle and
against central finite differences of the CUDA forward.

Loss of the anisotropic workload: L(A, B) = tr(P*^T A P*) + ||P*||_F^2 with
P* the converged constrained minimiser.  dL/dA = mask_A(P* P*^T) (explicit)
- 2 mask_A(U P*^T) (through P*), dL/dB = mu; checked at 1e-6 relative
against central differences on seeded entries (symmetric pairs of A
perturbed together)."""
import numpy as np
import pytest

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


SMALL = [I.poisson2d(10, 2), I.random_problem(60, 20, 2, p_per_row=6, seed=7),
         I.elasticity3d(4, 0.3, 2)]


@pytest.mark.parametrize("prob", SMALL, ids=lambda p: p.name)
def test_autograd_matches_oracle(prob):
    import torch
    from paper_2208_02995_gb300.autograd import EminEnergy, EminProblem, EminSolve
    pb = EminProblem.from_problem(prob)
    A = torch.tensor(prob.A_val, dtype=torch.float64, device="cuda", requires_grad=True)
    B = torch.tensor(prob.B, dtype=torch.float64, device="cuda", requires_grad=True)
    P = EminSolve.apply(A, B, pb, 500, 0.0, 500, 0.0)
    L = EminEnergy.apply(A, P, pb) + (P * P).sum()
    L.backward()
    o = Oracle(prob)
    ref = o.minimize(500)
    Pr = ref["P"]
    assert np.linalg.norm(P.detach().cpu().numpy() - Pr) <= 1e-9 * np.linalg.norm(Pr)
    assert abs(L.item() - (o.energy(Pr) + Pr @ Pr)) <= 1e-9 * abs(L.item())
    dA, dB, _, _ = o.backward(Pr, 2 * o.kprod(Pr) + 2 * Pr, 500)
    gA = dA + o.outer(Pr, Pr)
    assert np.linalg.norm(A.grad.cpu().numpy() - gA) <= 1e-8 * np.linalg.norm(gA)
    assert np.linalg.norm(B.grad.cpu().numpy() - dB) <= 1e-8 * np.linalg.norm(dB)


def test_mixed_forward_adjoint():
    """Mixed-precision forward (float bulk) with the FP64 adjoint, on the
    heterogeneous elasticity recipe: the gradient agrees with the FP64
    oracle's to the accuracy of the float forward."""
    import torch
    from paper_2208_02995_gb300.emin import Context
    prob = I.elasticity3d(6, 0.25, 3, 1.5, 5)
    o = Oracle(prob)
    Pr = o.minimize(600)["P"]
    c = Context(prob, precision="mixed")
    c.iterate(600)
    P = c.get_p()
    rp = np.linalg.norm(P - Pr) / np.linalg.norm(Pr)  # float accuracy of the minimiser
    assert rp <= 1e-4
    assert o.constraint_error(P) <= 1e-12
    dLdP = 2 * o.kprod(P) + 2 * P
    dA, dB, _ = c.backward(dLdP, 600, 0.0)
    dA_ref, dB_ref, _, _ = o.backward(Pr, 2 * o.kprod(Pr) + 2 * Pr, 600)
    tol = max(10 * rp, 1e-6)
    assert np.linalg.norm(dA - dA_ref) <= tol * np.linalg.norm(dA_ref)
    assert np.linalg.norm(dB - dB_ref) <= tol * np.linalg.norm(dB_ref)


def test_workload4_finite_differences():
    """3D anisotropic Poisson 160^3 (4.1M rows): implicit-adjoint gradient of
    L = tr(P^T A P) + ||P||_F^2 against central differences on 50 seeded
    entries of A (symmetric pairs, diagonal included) and 50 of B (seed 4),
    forward solves run to convergence, the perturbed ones warm-started from
    the converged P* (so that the solver's own error scales with the
    perturbation and cancels between the + and - solves).  Differences of L
    are formed locally:
    L(+) - L(-) = <P+ - P-, A(P+ + P-)> + h (P+^T D P+ + P-^T D P-)
    + <P+ - P-, P+ + P->, never as a difference of two global totals."""
    import torch
    from paper_2208_02995_gb300.emin import Context, emin_outer
    prob = I.config(4)
    n, k = prob.n, prob.k
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    arrays = [dev(a) for a in prob.arrays()]
    Ad, Bd = arrays[2], arrays[6]
    base = Context(n=n, nc=prob.nc, k=k, arrays=arrays)
    its = 300
    base.iterate(its)
    P = torch.empty(prob.nnz_p, dtype=torch.float64, device="cuda")
    base.get_p(P)
    AP = base.kprod(P, project=False)
    dA, dB, adj_steps = base.backward(2 * AP + 2 * P, its, 0.0)
    gA = (dA + emin_outer(base.h, P, P)).cpu().numpy()
    gB = dB.cpu().numpy()
    assert adj_steps > 0

    pert = Context(n=n, nc=prob.nc, k=k, arrays=arrays)
    Pp, Pm = (torch.empty_like(P) for _ in range(2))
    prow = prob.P_rowptr
    Pcol = prob.P_col

    def solve(A=None, B=None, out=None):
        pert.set_values(A_val=Ad if A is None else A, B=Bd if B is None else B, P0_val=P,
                        on_device=True)
        pert.iterate(its)
        pert.get_p(out)

    def row_dot(Pv, a, b):
        """sum_c P(a,c) P(b,c) from the two rows of P (device tensor)."""
        ra = slice(int(prow[a]), int(prow[a + 1]))
        rb = slice(int(prow[b]), int(prow[b + 1]))
        va = dict(zip(Pcol[ra].tolist(), Pv[ra].cpu().tolist()))
        return sum(va.get(c, 0.0) * v for c, v in zip(Pcol[rb].tolist(), Pv[rb].cpu().tolist()))

    def dL_common():
        d, s = Pp - Pm, Pp + Pm
        return float(torch.dot(d, base.kprod(s, project=False)) + torch.dot(d, s))

    rows = np.repeat(np.arange(n), np.diff(prob.A_rowptr))
    rng = np.random.default_rng(4)
    picks = rng.choice(prob.nnz_a, 50, replace=False)
    worst = 0.0
    for e in picks:
        a, b = int(rows[e]), int(prob.A_col[e])
        lo, hi = prob.A_rowptr[b], prob.A_rowptr[b + 1]
        mirror = lo + int(np.searchsorted(prob.A_col[lo:hi], a))
        h = 1e-4 * max(abs(prob.A_val[e]), 1.0)
        for sgn, out in ((1.0, Pp), (-1.0, Pm)):
            Ah = Ad.clone()
            Ah[e] += sgn * h
            if mirror != e:
                Ah[mirror] += sgn * h
            solve(A=Ah, out=out)
        w = 1.0 if a == b else 2.0  # P^T D P for D = e_ab + e_ba (or e_aa)
        explicit = h * w * (row_dot(Pp, a, b) + row_dot(Pm, a, b))
        fd = (dL_common() + explicit) / (2 * h)
        g = gA[e] + (gA[mirror] if mirror != e else 0.0)
        err = abs(fd - g) / max(abs(g), 1e-8 * np.abs(gA).max())
        worst = max(worst, err)
        assert err <= 1e-6, (e, a, b, fd, g)
    for idx in rng.choice(n * k, 50, replace=False):
        i, c = divmod(int(idx), k)
        h = 1e-4 * max(abs(prob.B[i, c]), 1.0)
        for sgn, out in ((1.0, Pp), (-1.0, Pm)):
            Bh = Bd.clone()
            Bh[i, c] += sgn * h
            solve(B=Bh, out=out)
        fd = dL_common() / (2 * h)
        g = gB[i, c]
        err = abs(fd - g) / max(abs(g), 1e-8 * np.abs(gB).max())
        worst = max(worst, err)
        assert err <= 1e-6, (i, c, fd, g)
    print(f"worst relative FD error {worst:.2e}")
