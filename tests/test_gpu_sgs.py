"""The projected block symmetric Gauss-Seidel preconditioner (M_2 of
Section 3.4) on the GPU against the FP64 oracle running the same
preconditioner: iterates, energy decrements, the stop test, the adjoint,
the full 128^3 workload, and the paper's observation that M_2 lowers the
energy faster per iteration than Jacobi."""
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


def ctx(prob, precision="fp64", **kw):
    from paper_2208_02995_gb300.emin import Context
    return Context(prob, precision=precision, precond="sgs", **kw)


def relf(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SMALL = [
    I.poisson2d(64, 2),
    I.diffusion3d_fv(21, 3),
    I.diffusion3d_fv(23, 3),
    I.aniso3d(14, 1e-3, 2),
    I.ring1d(1001, 2),
    I.elasticity3d(7, 0.3, 3),
    I.elasticity3d(8, 0.25, 3, 1.5, 5),
    I.random_problem(300, 60, 1, seed=1, wide_rows=(3, 77), wide=40),
    I.random_problem(200, 90, 3, p_per_row=7, seed=2, wide_rows=(5,), wide=80),
    I.random_problem(150, 400, 2, p_per_row=5, seed=3, wide_rows=(9,), wide=300),
    I.classical(I.diffusion3d_fv(16, 3)),     # P = [W; I], rows of W up to 12
    I.classical(I.aniso3d(12, 1e-3, 2)),      # semi-coarsening by the strength filter
    I.classical(I.poisson2d(40, 2), grow=2),  # pattern grown twice
]
IDS = [p.name for p in SMALL]


@pytest.mark.parametrize("prob", SMALL, ids=IDS)
def test_fp64_sgs_iterations_match_oracle(prob):
    o = Oracle(prob, precond="sgs")
    its = 8
    ref = o.minimize(its, 0.0)
    c = ctx(prob)
    done, _ = c.iterate(its, 0.0)
    assert done == ref["applied"]
    P = c.get_p()
    assert relf(P, ref["P"]) <= 1e-9
    assert np.allclose(c.stats()["dE"], ref["dE"], rtol=1e-9, atol=1e-13 * ref["dE"][0])
    assert o.constraint_error(P) <= 1e-12


@pytest.mark.parametrize("prob", SMALL, ids=IDS)
def test_mixed_sgs_energy_matches_oracle(prob):
    o = Oracle(prob, precond="sgs")
    ref = o.minimize(8, 0.0)
    c = ctx(prob, "mixed")
    c.iterate(8, 0.0)
    P = c.get_p()
    Eref = o.energy(ref["P"])
    assert abs(c.energy() - Eref) <= 1e-5 * abs(Eref)
    assert o.constraint_error(P) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sgs_workload2_full_size(precision):
    """3D FV diffusion 128^3, 20 iterations with M_2, element-wise (FP64) or
    in energy (mixed) against the oracle with M_2."""
    prob = I.config(2)
    o = Oracle(prob, precond="sgs")
    ref = o.minimize(prob.iters, 0.0)
    c = ctx(prob, precision)
    done, _ = c.iterate(prob.iters, 0.0)
    assert done == ref["applied"]
    P = c.get_p()
    if precision == "fp64":
        assert relf(P, ref["P"]) <= 1e-9
        assert np.allclose(c.stats()["dE"], ref["dE"], rtol=1e-9, atol=1e-13 * ref["dE"][0])
    else:
        Eref = o.energy(ref["P"])
        assert abs(c.energy() - Eref) <= 1e-5 * abs(Eref)
    assert o.constraint_error(P) <= 1e-12


@pytest.mark.parametrize("tau", [0.1, 1e-3])
def test_sgs_energy_stop(tau):
    prob = I.diffusion3d_fv(24, 3)
    o = Oracle(prob, precond="sgs")
    ref = o.minimize(200, tau)
    c = ctx(prob)
    done, rel = c.iterate(200, tau)
    assert done == ref["applied"] < 200
    assert relf(c.get_p(), ref["P"]) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sgs_while_graph_matches_direct_launches(precision):
    import torch
    from paper_2208_02995_gb300.emin import Context
    prob = I.diffusion3d_fv(20, 3)
    a = ctx(prob, precision)
    da, _ = a.iterate(15, 0.0)
    b = Context(prob, precision=precision, precond="sgs", stream=torch.cuda.Stream())
    db, _ = b.iterate(15, 0.0)
    assert da == db
    assert np.array_equal(a.get_p(), b.get_p())


def test_sgs_backward_matches_oracle():
    """The implicit adjoint with M_2 in the adjoint PCG (FP64) against the
    oracle's adjoint with M_2, after a converged forward."""
    prob = I.elasticity3d(5, 0.3, 2)
    o = Oracle(prob, precond="sgs")
    Pr = o.minimize(300)["P"]
    c = ctx(prob)
    c.iterate(300)
    P = c.get_p()
    assert relf(P, Pr) <= 1e-9
    dLdP = 2 * o.kprod(Pr) + 2 * Pr
    dA, dB, _ = c.backward(dLdP, 300, 0.0)
    dA_ref, dB_ref, _, _ = o.backward(Pr, dLdP, 300)
    assert np.linalg.norm(dA - dA_ref) <= 1e-8 * np.linalg.norm(dA_ref)
    assert np.linalg.norm(dB - dB_ref) <= 1e-8 * np.linalg.norm(dB_ref)


def test_sgs_lowers_energy_faster_than_jacobi():
    """The paper's observation on the 128^3 workload: after the same number
    of iterations M_2 has reached a lower energy than M_1."""
    from paper_2208_02995_gb300.emin import Context
    prob = I.config(2)
    j = Context(prob, precision="mixed")
    s = ctx(prob, "mixed")
    for its in (2, 5):
        j.reset()
        s.reset()
        j.iterate(its)
        s.iterate(its)
        assert s.energy() < j.energy()
