"""The bounds-check mode (emin_opts.checks = 1) of the kernels that gather
through the plan of the fixed pattern: on valid inputs it reports no fault
and its results are bit-identical to the unchecked kernels, for every
product kernel the problems select (packed and plain SELL plans, the
row and warp kernels, the node-block and staged elasticity products, the
projected SGS sweeps) and at the full size of the 128^3 workload.

Only valid inputs are used: an out-of-range index is never constructed on
the device (invalid patterns are rejected on the device before any plan is
built, which the ABI tests cover)."""
import numpy as np
import pytest

from paper_2208_02995_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_02995_gb300 import build
    build.build()


CASES = [
    (I.diffusion3d_fv(18, 3), "jacobi"),          # packed SELL plan
    (I.ring1d(1001, 2), "jacobi"),                # plain SELL plan (wide offsets)
    (I.random_problem(200, 90, 3, p_per_row=7, seed=2, wide_rows=(5,), wide=80), "jacobi"),
    (I.classical(I.diffusion3d_fv(12, 3)), "jacobi"),  # rows of P up to 12: warp kernel
    (I.elasticity3d(8, 0.25, 3, 1.5, 5), "jacobi"),    # node-block / staged products
    (I.diffusion3d_fv(14, 3), "sgs"),             # SGS sweeps (batched and level)
    (I.elasticity3d(6, 0.3, 2), "sgs"),
]


def _run(prob, precision, precond, checks, its=8):
    from paper_2208_02995_gb300.emin import Context
    c = Context(prob, precision=precision, precond=precond, checks=checks)
    X = np.random.default_rng(3).standard_normal(prob.nnz_p)
    kp = c.kprod(X, project=True)
    c.iterate(its)
    P = c.get_p()
    E = c.energy()
    c.close()
    return kp, P, E


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0].name}-{c[1]}")
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checks_bit_identical(case, precision):
    prob, precond = case
    a = _run(prob, precision, precond, False)
    b = _run(prob, precision, precond, True)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_checks_full_size_workload2():
    prob = I.config(2)
    for precision in ("mixed", "fp64"):
        a = _run(prob, precision, "jacobi", False, its=prob.iters)
        b = _run(prob, precision, "jacobi", True, its=prob.iters)
        assert np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_checks_adjoint_bit_identical():
    from paper_2208_02995_gb300.emin import Context
    prob = I.elasticity3d(6, 0.25, 3, 1.5, 5)
    out = []
    for checks in (False, True):
        c = Context(prob, checks=checks)
        c.iterate(200)
        P = c.get_p()
        _, g, _ = c.energy_grad(P, 1.0, want_energy=False, want_dX=True)
        dA, dB, _ = c.backward(g + 2 * P, 100, 1e-20)
        out.append((dA, dB))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
