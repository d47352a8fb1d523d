"""Host-side helpers of bench.py: the counts of candidate and in-pattern
products of one masked product, at node level for node-blocked (elasticity)
problems, against a brute-force count over every stored entry of A."""
import numpy as np
import pytest

from paper_2208_02995_gb300 import inputs as I


def brute_force(p):
    """For every stored a_il: |J_l| candidates, |J_i & J_l| in pattern."""
    n = p.n
    m = np.diff(p.P_rowptr)
    w = int(m.max())
    J = np.full((n, w), -1, dtype=np.int64)
    rows = np.repeat(np.arange(n), m)
    J[rows, np.arange(p.nnz_p) - p.P_rowptr[rows]] = p.P_col
    arow = np.repeat(np.arange(n), np.diff(p.A_rowptr))
    Ji, Jl = J[arow], J[p.A_col]
    hits = int(((Ji[:, :, None] == Jl[:, None, :]) & (Ji[:, :, None] >= 0)).sum())
    return int(m[p.A_col].sum()), hits


@pytest.mark.parametrize("p", [I.elasticity3d(5, 0.3, 2), I.elasticity3d(7, 0.25, 3, 1.5, 5)],
                         ids=lambda p: p.name)
def test_blocked_product_count(p):
    import bench
    assert bench.in_pattern_products_blocked(p) == brute_force(p)
    assert bench.products(p) == brute_force(p)


def test_scalar_product_count():
    import bench
    p = I.diffusion3d_fv(9, 3)
    assert bench.in_pattern_products(p) == brute_force(p)
