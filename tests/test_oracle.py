"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle
with a different computation (dense products, NumPy QR / lstsq / solve, the
null-space method, a hand-derived closed form) or with an identity the
paper proves (Theorem 1, its corollary, the energy decrement of
Eq. (CG_dEa), the envelope theorem for the adjoint)."""
import numpy as np
import pytest

from oracle import kkt_dense as KD
from oracle.oracle import Oracle, OracleError
from paper_2208_02995_gb300 import inputs as I
from tests.golden_fixtures import problem_1d4

TINY = [
    I.poisson2d(8, 2),
    I.diffusion3d_fv(6, 3),
    I.aniso3d(4, 1e-3, 2),
    I.elasticity3d(4, 0.3, 2),
    I.random_problem(30, 10, 1, seed=1),
    I.random_problem(30, 12, 2, p_per_row=6, seed=3),
    I.random_problem(24, 14, 3, p_per_row=7, seed=5, wide_rows=(3,), wide=14),
    I.classical(I.poisson2d(7, 2)),
    I.classical(I.aniso3d(5, 0.1, 2)),
    I.classical(I.diffusion3d_fv(5, 3)),
]
IDS = [p.name for p in TINY]


def _dense_P(prob, vals):
    P = np.zeros((prob.n, prob.nc))
    P[KD.entry_rows(prob), prob.P_col] = vals
    return P


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_kprod_is_masked_dense_product(prob):
    """mask_P(A Y) = dense A @ Y read at P's pattern (Section 4)."""
    o = Oracle(prob)
    Y = np.random.default_rng(1).standard_normal(prob.nnz_p)
    full = KD.dense_A(prob) @ _dense_P(prob, Y)
    ref = full[KD.entry_rows(prob), prob.P_col]
    assert np.abs(o.kprod(Y) - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_kprod_self_adjoint(prob):
    o = Oracle(prob)
    rng = np.random.default_rng(2)
    X, Y = rng.standard_normal((2, prob.nnz_p))
    a, b = X @ o.kprod(Y), o.kprod(X) @ Y
    assert abs(a - b) <= 1e-12 * (abs(a) + 1)


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_projection(prob):
    """Pi_B = I - Q Q^T with Q an orthonormal basis of range(B_i) per row."""
    o = Oracle(prob)
    x = np.random.default_rng(3).standard_normal(prob.nnz_p)
    px = o.project(x)
    assert np.abs(o.project(px) - px).max() < 1e-13
    for i in range(prob.n):
        s0, s1 = prob.P_rowptr[i], prob.P_rowptr[i + 1]
        Bi = prob.Bc[prob.P_col[s0:s1]]
        assert np.abs(Bi.T @ px[s0:s1]).max() < 1e-12 * max(1, np.abs(Bi).max())
        Qn, _ = np.linalg.qr(Bi)
        ref = x[s0:s1] - Qn @ (Qn.T @ x[s0:s1])
        assert np.abs(px[s0:s1] - ref).max() < 1e-12


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_setup_least_norm_correction(prob):
    """Algorithm 2: the corrected P0 satisfies P0 B_c = B, and the correction
    is the least-norm solution of B_i^T d = r_i (numpy lstsq)."""
    o = Oracle(prob)
    assert o.constraint_error(o.P0) <= 1e-12
    d = o.P0 - prob.P0_val
    for i in range(prob.n):
        s0, s1 = prob.P_rowptr[i], prob.P_rowptr[i + 1]
        Bi = prob.Bc[prob.P_col[s0:s1]]
        r = prob.B[i] - Bi.T @ prob.P0_val[s0:s1]
        ref = np.linalg.lstsq(Bi.T, r, rcond=None)[0]
        assert np.abs(d[s0:s1] - ref).max() < 1e-11


@pytest.mark.parametrize("prob", TINY[:4], ids=IDS[:4])
def test_theorem1_and_corollary(prob):
    """diag(Z^T K Z) = A_ii per row and Z^T D_K Q = 0 (Theorem 1 and its
    corollary), so the Jacobi step leaves range(Pi_B) invariant: the
    oracle's Pi_B M^{-1} r equals M^{-1} r for r in range(Pi_B)."""
    o = Oracle(prob)
    K = KD.dense_K(prob)
    rows = KD.entry_rows(prob)
    for i in range(0, prob.n, max(1, prob.n // 7)):
        sl = np.nonzero(rows == i)[0]
        Bi = prob.Bc[prob.P_col[sl]]
        Qf, _ = np.linalg.qr(Bi, mode="complete")
        Q, Z = Qf[:, :prob.k], Qf[:, prob.k:]
        Kii = K[np.ix_(sl, sl)]
        if Z.shape[1] == 0:
            continue
        assert np.allclose(np.diag(Z.T @ Kii @ Z), K[sl[0], sl[0]], rtol=0, atol=1e-12)
        assert np.abs(Z.T @ np.diag(np.diag(Kii)) @ Q).max() < 1e-12
    r = o.project(np.random.default_rng(4).standard_normal(prob.nnz_p))
    z = o.dinv[rows] * r
    assert np.abs(o.project(z) - z).max() < 1e-12 * np.abs(z).max()


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_pcg_equals_nullspace_method(prob):
    """Algorithm 3 is the null-space method on (sadsys): the restricted PCG
    iterates equal p0 + Z x_k of preconditioned CG on Z^T K Z with
    M^{-1} = Z^T D_K^{-1} Z (dense, Z from a full QR of C^T)."""
    o = Oracle(prob)
    its, dE = KD.nullspace_pcg(prob, o.P0, 6)
    for j in range(1, len(its)):
        res = o.minimize(j, 0.0)
        scale = np.abs(its[j]).max()
        assert np.abs(res["P"] - its[j]).max() <= 1e-10 * scale, j
        assert np.allclose(res["dE"], dE[:j], rtol=1e-9, atol=0)


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_energy_decrement_identity(prob):
    """E(P_k) - E(P_{k+1}) = gamma_k alpha_k (Eq. (CG_dEa), sign read as a
    decrease) and the energy decreases monotonically."""
    o = Oracle(prob)
    E = [o.energy(o.P0)]
    for j in range(1, 7):
        E.append(o.energy(o.minimize(j, 0.0)["P"]))
    dE = o.minimize(6, 0.0)["dE"]
    for j in range(len(dE)):
        assert E[j + 1] <= E[j] + 1e-12 * abs(E[0])
        assert abs((E[j] - E[j + 1]) - dE[j]) <= 1e-9 * abs(E[0])


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_energy_is_trace(prob):
    o = Oracle(prob)
    p = o.P0 + 0.1 * np.random.default_rng(5).standard_normal(prob.nnz_p)
    P = _dense_P(prob, p)
    ref = np.trace(P.T @ KD.dense_A(prob) @ P)
    assert abs(o.energy(p) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_limit_is_kkt_solution(prob):
    """Run to convergence: P equals the dense saddle-point solution."""
    o = Oracle(prob)
    res = o.minimize(400, 0.0)
    assert res["status"] == 0
    p_kkt, _ = KD.kkt_solve(prob)
    scale = np.abs(p_kkt).max()
    assert np.abs(res["P"] - p_kkt).max() <= 1e-8 * scale
    assert o.constraint_error(res["P"]) <= 1e-12
    # the energy reached is not above the KKT energy (up to rounding)
    assert o.energy(res["P"]) <= KD.energy(prob, p_kkt) * (1 + 1e-12)


def test_golden_1d4():
    prob, g = problem_1d4()
    o = Oracle(prob)
    assert np.allclose(o.P0, g["P0"], rtol=0, atol=1e-15)
    assert abs(o.energy(o.P0) - g["E0"][0]) < 1e-14
    res = o.minimize(5, 0.0)
    assert res["status"] == 0
    assert len(res["dE"]) == 1 and res["applied"] == 1  # second gamma is zero
    assert abs(res["dE"][0] - g["dE1"][0]) < 1e-14
    assert np.abs(res["P"] - np.array(g["P_star"])).max() < 1e-15
    assert abs(o.energy(res["P"]) - g["E_star"][0]) < 1e-14


def test_no_freedom_keeps_p0():
    """Pattern = pattern(P0) with k = 1: every row has one entry fixed by the
    constraint, so P = P0 and no step is taken."""
    prob = I.poisson2d(8, 2)
    keep = prob.P0_val != 0
    rows = KD.entry_rows(prob)
    Pp = np.zeros(prob.n + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows[keep], minlength=prob.n), out=Pp[1:])
    p2 = I.Problem("p0pattern", prob.n, prob.nc, 1, prob.A_rowptr, prob.A_col, prob.A_val,
                   Pp, prob.P_col[keep], prob.P0_val[keep], prob.B, prob.Bc)
    o = Oracle(p2)
    res = o.minimize(10, 0.0)
    assert res["applied"] == 0 and res["status"] == 0
    assert np.array_equal(res["P"], o.P0)


def test_rank_deficient_rows():
    """Rows with m_i < k: strict policy fails; the pseudo-inverse policy
    (the SVD branch of Algorithm 2) gives the least-squares correction."""
    prob = I.random_problem(20, 9, 3, p_per_row=4, seed=11)
    # make row 5 have only two entries
    Pp, Pj, P0 = prob.P_rowptr.copy(), prob.P_col.copy(), prob.P0_val.copy()
    s0, s1 = Pp[5], Pp[6]
    drop = np.arange(s0 + 2, s1)
    Pj, P0 = np.delete(Pj, drop), np.delete(P0, drop)
    Pp[6:] -= len(drop)
    p2 = I.Problem("rankdef", prob.n, prob.nc, 3, prob.A_rowptr, prob.A_col, prob.A_val,
                   Pp, Pj, P0, prob.B, prob.Bc)
    with pytest.raises(OracleError):
        Oracle(p2)
    o = Oracle(p2, pinv=True)
    assert o.n_deficient == 1
    s0, s1 = Pp[5], Pp[6]
    Bi = p2.Bc[Pj[s0:s1]]
    r = p2.B[5] - Bi.T @ P0[s0:s1]
    ref = np.linalg.lstsq(Bi.T, r, rcond=None)[0]
    assert np.abs(o.P0[s0:s1] - P0[s0:s1] - ref).max() < 1e-12
    # Pi_B removes range(B_i) from the row, which is all of R^2 here
    x = np.random.default_rng(0).standard_normal(p2.nnz_p)
    assert np.abs(o.project(x)[s0:s1]).max() < 1e-12
    assert o.minimize(5, 0.0)["status"] == 0


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
BWD = [I.poisson2d(6, 2), I.random_problem(18, 7, 1, seed=2),
       I.random_problem(16, 9, 2, p_per_row=5, seed=8), I.elasticity3d(3, 0.3, 2)]


@pytest.mark.parametrize("prob", BWD, ids=[p.name for p in BWD])
def test_backward_envelope(prob):
    """For L = E(P*): dL/dp = 2 K p* lies in range(C^T), so U = 0,
    dL/dA = mask_A(P* P*^T) (explicit term only, the adjoint part vanishes)
    and dL/dB = mu = -lambda of the dense saddle-point system."""
    o = Oracle(prob)
    P = o.minimize(500, 0.0)["P"]
    dLdP = 2 * o.kprod(P)
    dA, dB, U, _ = o.backward(P, dLdP, 500, 0.0)
    assert np.abs(U).max() <= 1e-9 * np.abs(P).max()
    assert np.abs(dA).max() <= 1e-8 * np.abs(P).max() ** 2
    p_kkt, lam = KD.kkt_solve(prob)
    ref = -lam.reshape(prob.n, prob.k)
    assert np.abs(dB - ref).max() <= 1e-7 * max(1, np.abs(ref).max())


@pytest.mark.parametrize("prob", BWD, ids=[p.name for p in BWD])
def test_backward_vs_dense_finite_differences(prob):
    """L(A, B) = tr(P*^T A P*) + ||P*||_F^2 with P* from the dense KKT solve;
    central differences of that dense function against the oracle adjoint
    (plus the explicit term mask_A(P P^T))."""
    o = Oracle(prob)
    P = o.minimize(500, 0.0)["P"]
    dLdP = 2 * o.kprod(P) + 2 * P
    dA, dB, _, _ = o.backward(P, dLdP, 500, 0.0)
    gA = dA + o.outer(P, P)

    def L(Aval, Bm):
        q = I.Problem("fd", prob.n, prob.nc, prob.k, prob.A_rowptr, prob.A_col, Aval,
                      prob.P_rowptr, prob.P_col, prob.P0_val, Bm, prob.Bc)
        p, _ = KD.kkt_solve(q)
        return KD.energy(q, p) + p @ p

    rows = np.repeat(np.arange(prob.n), np.diff(prob.A_rowptr))
    rng = np.random.default_rng(9)
    for e in rng.choice(prob.nnz_a, 6, replace=False):
        a, b = rows[e], prob.A_col[e]
        # perturb the symmetric pair together
        mirror = np.nonzero((rows == b) & (prob.A_col == a))[0][0]
        h = 1e-5 * max(1.0, abs(prob.A_val[e]))
        Ap, Am = prob.A_val.copy(), prob.A_val.copy()
        Ap[e] += h
        Am[e] -= h
        if mirror != e:
            Ap[mirror] += h
            Am[mirror] -= h
        fd = (L(Ap, prob.B) - L(Am, prob.B)) / (2 * h)
        g = gA[e] + (gA[mirror] if mirror != e else 0.0)
        assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (e, fd, g)
    for _ in range(4):
        i, c = rng.integers(prob.n), rng.integers(prob.k)
        h = 1e-5
        Bp, Bm = prob.B.copy(), prob.B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = (L(prob.A_val, Bp) - L(prob.A_val, Bm)) / (2 * h)
        assert abs(fd - dB[i, c]) <= 1e-5 * max(1.0, abs(dB[i, c])), (i, c, fd, dB[i, c])


# ---------------------------------------------------------------------------
# projected block symmetric Gauss-Seidel (M_2 of Section 3.4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_sgs_is_dense_formula(prob):
    """The oracle's block SGS equals (L + D)^{-T} D (L + D)^{-1} r with
    K = L + D + L^T taken densely in the row-wise order of p (dense
    triangular solves over the whole K: the blocks come out by themselves)."""
    o = Oracle(prob, precond="sgs")
    r = np.random.default_rng(11).standard_normal(prob.nnz_p)
    ref = KD.sgs_inverse(KD.dense_K(prob)) @ r
    assert np.abs(o.sgs(r) - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("prob", TINY[:4], ids=IDS[:4])
def test_sgs_symmetric_positive(prob):
    o = Oracle(prob, precond="sgs")
    rng = np.random.default_rng(12)
    x, y = rng.standard_normal((2, prob.nnz_p))
    a, b = x @ o.sgs(y), y @ o.sgs(x)
    assert abs(a - b) <= 1e-12 * (abs(a) + 1)
    assert x @ o.sgs(x) > 0


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_sgs_pcg_equals_nullspace_method(prob):
    """Algorithm 3 with z = Pi_B M_SGS^{-1} r equals dense preconditioned CG
    on Z^T K Z with M_2^{-1} = Z^T M_SGS^{-1} Z (Pi_B = Z Z^T)."""
    o = Oracle(prob, precond="sgs")
    its, dE = KD.nullspace_pcg(prob, o.P0, 5, precond="sgs")
    for j in range(1, len(its)):
        res = o.minimize(j, 0.0)
        scale = np.abs(its[j]).max()
        assert np.abs(res["P"] - its[j]).max() <= 1e-10 * scale, j
        assert np.allclose(res["dE"], dE[:j], rtol=1e-9, atol=0)


@pytest.mark.parametrize("prob", TINY, ids=IDS)
def test_sgs_energy_identity_and_limit(prob):
    """Energy decrement identity and monotone decrease with M_2, and the
    same constrained minimiser as the dense KKT solve (the preconditioner
    changes the path, not the limit)."""
    o = Oracle(prob, precond="sgs")
    E = [o.energy(o.P0)]
    for j in range(1, 6):
        E.append(o.energy(o.minimize(j, 0.0)["P"]))
    dE = o.minimize(5, 0.0)["dE"]
    for j in range(len(dE)):
        assert E[j + 1] <= E[j] + 1e-12 * abs(E[0])
        assert abs((E[j] - E[j + 1]) - dE[j]) <= 1e-9 * abs(E[0])
    res = o.minimize(300, 0.0)
    assert res["status"] == 0
    p_kkt, _ = KD.kkt_solve(prob)
    assert np.abs(res["P"] - p_kkt).max() <= 1e-8 * np.abs(p_kkt).max()


def test_sgs_reduces_energy_faster_than_jacobi():
    """The paper's observation (Section 5.1): M_2 reduces the energy faster
    per iteration than Jacobi; pinned on the heterogeneous FV recipe."""
    prob = I.diffusion3d_fv(12, 3)
    j, s = Oracle(prob), Oracle(prob, precond="sgs")
    for its in (2, 4, 8):
        assert s.energy(s.minimize(its)["P"]) < j.energy(j.minimize(its)["P"])


@pytest.mark.parametrize("prob", BWD, ids=[p.name for p in BWD])
def test_backward_sgs_equals_jacobi(prob):
    """The implicit adjoint solves one more constrained system; run to
    convergence, its solution U and the gradients do not depend on which
    preconditioner (M_1 or M_2) the restricted PCG uses."""
    j, s = Oracle(prob), Oracle(prob, precond="sgs")
    P = j.minimize(500, 0.0)["P"]
    dLdP = 2 * j.kprod(P) + 2 * P
    dAj, dBj, Uj, _ = j.backward(P, dLdP, 500, 0.0)
    dAs, dBs, Us, _ = s.backward(P, dLdP, 500, 0.0)
    assert np.abs(Us - Uj).max() <= 1e-9 * max(1, np.abs(Uj).max())
    assert np.abs(dAs - dAj).max() <= 1e-8 * max(1, np.abs(dAj).max())
    assert np.abs(dBs - dBj).max() <= 1e-8 * max(1, np.abs(dBj).max())


def _full_w(base):
    """The classical form with a full W pattern (every F row holds every
    coarse column) on the operator of ``base``."""
    p = I.classical(base)
    n, nc = p.n, p.nc
    isC = np.zeros(n, dtype=bool)
    isC[p.meta["cpoints"]] = True
    rows0 = np.repeat(np.arange(n), np.diff(p.P_rowptr))
    P0 = np.zeros((n, nc))
    P0[rows0, p.P_col] = p.P0_val
    mask = np.zeros((n, nc), dtype=bool)
    mask[~isC] = True
    mask[isC, np.arange(nc)] = True
    r, c = np.nonzero(mask)
    Pp = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(np.bincount(r, minlength=n), out=Pp[1:])
    return I.Problem(p.name + "_fullW", n, nc, 1, p.A_rowptr, p.A_col, p.A_val, Pp,
                     c.astype(np.int32), P0[r, c], p.B, p.Bc, p.iters, p.meta), isC


@pytest.mark.parametrize("base", [I.ring1d(24, 2), I.diffusion3d_fv(4, 2)],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("precond", ["jacobi", "sgs"])
def test_classical_full_pattern_is_ideal_prolongation(base, precond):
    """With a full W pattern the energy minimiser of P = [W; I] is the ideal
    prolongation W = -A_ff^{-1} A_fc (each column minimises p^T A p with its
    C entry fixed, Eq. (minblk)); on a Neumann operator (A 1 = 0) it also
    interpolates the constant, A_ff 1 + A_fc 1 = 0, so the constraint holds
    and the constrained minimiser is the same.  The C rows, one entry each,
    stay identity rows under the constraint."""
    p, isC = _full_w(base)
    o = Oracle(p, precond=precond)
    P = o.minimize(800, 0.0)["P"]
    A = KD.dense_A(p)
    Wideal = -np.linalg.solve(A[np.ix_(~isC, ~isC)], A[np.ix_(~isC, isC)])
    Pd = _dense_P(p, P)
    assert np.abs(Pd[~isC] - Wideal).max() <= 1e-9 * max(1, np.abs(Wideal).max())
    assert np.abs(Pd[isC] - np.eye(p.nc)).max() <= 1e-14
