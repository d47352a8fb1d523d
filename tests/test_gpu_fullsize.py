"""Full-size workloads on the GPU.

Workload 4 (3D anisotropic 160^3): element-wise against the oracle after the
fixed 15 iterations (FP64), energy for the mixed path.  Elasticity
workloads 3 (64^3 nodes) and 5 (96^3 nodes, heterogeneous): element-wise on
what the oracle computes in seconds at that size (the corrected P0, one
masked product with projection), then, after the workload's iterations,
the properties the paper fixes: the constraint P B_c = B, the energy
decrement identity E(P0) - E(P_k) = sum of dE (Eq. (CG_dEa)) and the
monotone decrease."""
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


def relf(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_workload4_full_size():
    from paper_2208_02995_gb300.emin import Context
    prob = I.config(4)
    o = Oracle(prob)
    ref = o.minimize(prob.iters)
    c = Context(prob)
    done, _ = c.iterate(prob.iters)
    assert done == ref["applied"]
    P = c.get_p()
    assert relf(P, ref["P"]) <= 1e-9
    assert np.allclose(c.stats()["dE"], ref["dE"], rtol=1e-9, atol=1e-13 * ref["dE"][0])
    assert o.constraint_error(P) <= 1e-12
    Eref = o.energy(ref["P"])
    m = Context(prob, precision="mixed")
    m.iterate(prob.iters)
    assert abs(m.energy() - Eref) <= 1e-5 * abs(Eref)
    assert o.constraint_error(m.get_p()) <= 1e-12


def _elasticity_checks(prob, precision, kprod_tol, ident_tol):
    from paper_2208_02995_gb300.emin import Context
    o = Oracle(prob)
    c = Context(prob, precision=precision)
    # corrected P0 (Algorithm 2) element-wise
    P0 = c.get_p()
    assert np.abs(P0 - o.P0).max() <= 1e-12 * np.abs(o.P0).max()
    E0 = o.energy(o.P0)
    # one masked product with projection, element-wise
    X = np.random.default_rng(1).standard_normal(prob.nnz_p)
    ref = o.project(o.kprod(X))
    got = c.kprod(X, project=True)
    assert np.abs(got - ref).max() <= kprod_tol * np.abs(ref).max()
    # the workload's iterations: constraint, energy identity, monotone decrease
    done, _ = c.iterate(prob.iters)
    assert done == prob.iters
    P = c.get_p()
    assert o.constraint_error(P) <= 1e-12
    dE = c.stats()["dE"]
    assert np.all(dE > 0) and len(dE) == prob.iters
    E = c.energy()
    assert abs((E0 - E) - dE.sum()) <= ident_tol * E0
    return c, o, P


def test_workload3_full_size():
    prob = I.config(3)
    _elasticity_checks(prob, "fp64", 1e-12, 1e-10)


def test_workload5_full_size_mixed_with_adjoint():
    """Mixed path on 96^3 heterogeneous elasticity.  The float application of
    Pi_B amplifies rounding by cond(G_i) (the rigid-body Gram matrix of a
    small region, ill-conditioned), so one projected product is within 1e-4
    relative; the bars of the mixed path are the energy (1e-5 of the FP64
    result) and the restored constraint (1e-12)."""
    from paper_2208_02995_gb300.emin import Context
    prob = I.config(5)
    c, o, P = _elasticity_checks(prob, "mixed", 1e-4, 1e-5)
    d = Context(prob, precision="fp64")
    d.iterate(prob.iters)
    Ed = d.energy()
    assert abs(c.energy() - Ed) <= 1e-5 * abs(Ed)
    # implicit adjoint (FP64) of L = tr(P^T A P) + ||P||^2 after the mixed forward
    dLdP = 2 * c.kprod(P, project=False) + 2 * P
    dA, dB, steps = c.backward(dLdP, 200, 0.0)
    assert steps > 0
    assert np.all(np.isfinite(dA)) and np.all(np.isfinite(dB))
    assert np.abs(dB).max() < 1e6 * (1 + np.abs(prob.B).max())
