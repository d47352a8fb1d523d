"""The allocation-free entry point (emin_masked_product_noalloc).

It serves callers that must not let a library allocate device memory: a
process whose device memory belongs to another allocator's pool, or a
request path that cannot afford the device synchronisation of cudaMalloc /
cudaFree.  Its output is checked against the oracle's masked product and
against the existing entry point (emin_kprod without projection), within
the masked-product tolerance of the other GPU tests, on two calls in a row
that share the scratch array; its documented edge cases are checked too.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before this one."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2208_02995_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KPROD_TOL = 1e-12
MAX_ROWS = 16384 * 256  # the scratch array's limit


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_02995_gb300 import build
    build.build()


def _device_arrays(prob):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
            (prob.A_rowptr, prob.A_col, prob.A_val, prob.P_rowptr, prob.P_col)]


@pytest.mark.parametrize("prob", [I.diffusion3d_fv(16, 3),
                                  I.random_problem(300, 90, 3, p_per_row=7, seed=2,
                                                   wide_rows=(5,), wide=80)],
                         ids=lambda p: p.name)
def test_noalloc_matches_oracle_and_existing_entry_point(prob):
    import torch
    from paper_2208_02995_gb300.emin import Context, emin_masked_product_noalloc
    o = Oracle(prob)
    c = Context(prob)
    dev = _device_arrays(prob)
    rng = np.random.default_rng(11)
    for call in range(2):
        X = rng.standard_normal(prob.nnz_p)
        ref = o.kprod(X)
        lib_ref = c.kprod(X, project=False)
        Xd = torch.from_numpy(X).cuda()
        out = torch.full((prob.nnz_p,), float("nan"), dtype=torch.float64, device="cuda")
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        emin_masked_product_noalloc(prob.n, prob.nc, *dev, Xd, out, dot)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= KPROD_TOL * scale, call
        assert np.abs(got - lib_ref).max() <= KPROD_TOL * scale, call
        dref = float(X @ ref)
        assert abs(dot.item() - dref) <= KPROD_TOL * np.abs(X).dot(np.abs(ref)), call


def test_noalloc_empty_problem_writes_zero_dot():
    import torch
    from paper_2208_02995_gb300.emin import emin_masked_product_noalloc
    z32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    e32 = torch.zeros(0, dtype=torch.int32, device="cuda")
    e64 = torch.zeros(0, dtype=torch.float64, device="cuda")
    dot = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    emin_masked_product_noalloc(0, 0, z32, e32, e64, z32, e32, e64, e64, dot)
    torch.cuda.synchronize()
    assert dot.item() == 0.0


def test_noalloc_rejects_rows_beyond_the_scratch_size():
    # the size check returns before anything is queued, so the (small)
    # arrays passed are never read
    import torch
    from paper_2208_02995_gb300.emin import EminError, emin_masked_product_noalloc, EMIN_ERR_ARG
    i32 = torch.zeros(4, dtype=torch.int32, device="cuda")
    f64 = torch.zeros(4, dtype=torch.float64, device="cuda")
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(EminError) as err:
        emin_masked_product_noalloc(MAX_ROWS + 1, 4, i32, i32, f64, i32, i32, f64, f64, dot)
    assert err.value.status == EMIN_ERR_ARG


def test_noalloc_rejects_host_arrays():
    import torch
    from paper_2208_02995_gb300.emin import emin_masked_product_noalloc
    prob = I.diffusion3d_fv(6, 3)
    dev = _device_arrays(prob)
    Y = torch.zeros(prob.nnz_p, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(Y)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    host = list(dev)
    host[1] = prob.A_col  # a NumPy (host) array
    with pytest.raises(ValueError):
        emin_masked_product_noalloc(prob.n, prob.nc, *host, Y, out, dot)
    with pytest.raises(ValueError):  # wrong dtype: no converted temporary is passed
        emin_masked_product_noalloc(prob.n, prob.nc, *dev[:2], dev[2].float(), *dev[3:], Y,
                                    out, dot)


def test_noalloc_out_of_range_column_gives_nan_dot():
    """A column index of A equal to n: the kernel checks every index before
    it reads through it, skips that entry and reports NaN in *dot; rows that
    do not hold the bad entry are unchanged."""
    import torch
    from paper_2208_02995_gb300.emin import emin_masked_product_noalloc
    prob = I.diffusion3d_fv(8, 3)
    o = Oracle(prob)
    X = np.random.default_rng(3).standard_normal(prob.nnz_p)
    ref = o.kprod(X)
    bad_row = prob.n // 2
    A_col = prob.A_col.copy()
    A_col[prob.A_rowptr[bad_row]] = prob.n
    dev = _device_arrays(prob)
    dev[1] = torch.from_numpy(A_col).cuda()
    out = torch.zeros(prob.nnz_p, dtype=torch.float64, device="cuda")
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    emin_masked_product_noalloc(prob.n, prob.nc, *dev, torch.from_numpy(X).cuda(), out, dot)
    torch.cuda.synchronize()
    assert np.isnan(dot.item())
    got = out.cpu().numpy()
    keep = np.ones(prob.nnz_p, dtype=bool)
    keep[prob.P_rowptr[bad_row]:prob.P_rowptr[bad_row + 1]] = False
    assert np.abs(got[keep] - ref[keep]).max() <= KPROD_TOL * np.abs(ref).max()
    # the next call on valid arrays starts from cleared counters
    emin_masked_product_noalloc(prob.n, prob.nc, *_device_arrays(prob),
                                torch.from_numpy(X).cuda(), out, dot)
    torch.cuda.synchronize()
    assert abs(dot.item() - float(X @ ref)) <= KPROD_TOL * np.abs(X).dot(np.abs(ref))
