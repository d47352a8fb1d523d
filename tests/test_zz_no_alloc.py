"""The allocation-free entry point (emin_masked_product_noalloc), for
callers that must not let the library allocate device memory: its output
equals the existing entry point's (emin_kprod without projection, and the
dot product of that output with Y), within the masked-product tolerance of
the other GPU tests, on two calls in a row sharing the scratch array.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before this one."""
import numpy as np
import pytest

from paper_2208_02995_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KPROD_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_02995_gb300 import build
    build.build()


@pytest.mark.parametrize("prob", [I.diffusion3d_fv(16, 3),
                                  I.random_problem(300, 90, 3, p_per_row=7, seed=2,
                                                   wide_rows=(5,), wide=80)],
                         ids=lambda p: p.name)
def test_noalloc_matches_existing_entry_point(prob):
    import torch
    from paper_2208_02995_gb300.emin import Context, emin_masked_product_noalloc
    c = Context(prob)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
           (prob.A_rowptr, prob.A_col, prob.A_val, prob.P_rowptr, prob.P_col)]
    rng = np.random.default_rng(11)
    for call in range(2):
        X = rng.standard_normal(prob.nnz_p)
        ref = c.kprod(X, project=False)
        Xd = torch.from_numpy(X).cuda()
        out = torch.full((prob.nnz_p,), float("nan"), dtype=torch.float64, device="cuda")
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        emin_masked_product_noalloc(prob.n, prob.nc, *dev, Xd, out, dot)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= KPROD_TOL * np.abs(ref).max(), call
        dref = float(X @ ref)
        assert abs(dot.item() - dref) <= KPROD_TOL * max(abs(dref), np.abs(X).dot(np.abs(ref))), call
