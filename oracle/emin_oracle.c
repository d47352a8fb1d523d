/*
 * emin_oracle.c -- plain, slow, FP64 CPU oracle of the energy-minimisation
 * prolongation loop (Janna, Franceschini, Schroder, Olson, "Parallel
 * Energy-Minimization Prolongation for Algebraic Multigrid", Sections 3-4).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this library; the product path never does.
 * It shares no code with the CUDA library: it factorises each local block
 * with a Householder QR (the paper's Algorithm 2) where the CUDA path uses a
 * Gram/Cholesky factorisation, it forms the masked product by computing a
 * full row of A*Y in a dense scratch row and then masking it (the plain
 * definition), and it runs Algorithm 3 literally, projecting after the
 * preconditioner step as the algorithm prints it.  The preconditioner is
 * Jacobi (M_1) or the projected block symmetric Gauss-Seidel (M_2), the
 * latter swept column block by column block through the transposed pattern
 * of P with a binary search for every coupled entry.
 *
 * Notation (Sections 3.1-3.4): P is n x nc with fixed pattern; J_i is the
 * sorted column set of row i (m_i entries); B_i = B_c(J_i,:) is m_i x k;
 * the constraint of row i is B_i^T p_i = B(i,:)^T (Eq. (Constr), with
 * V_c = B_c and v_i = B(i,:)); K is block diagonal by columns of P and
 * K*y is the masked product mask_P(A*Y) (Section 4); Pi_B = I - Q Q^T with
 * Q an orthonormal basis of range(B_i) per row.
 *
 * Compiled with -ffp-contract=off so that every multiply and add rounds
 * separately, on every host.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_RANK = -3, ORC_ERR_DIAG = -4,
       ORC_ERR_BREAKDOWN = -5, ORC_ERR_NOMEM = -7 };

/* ------------------------------------------------------------------------
 * Local factorisation of one row block (Algorithm 2).
 *
 * Bi is m x k row-major.  On return Q (m x k row-major) holds an orthonormal
 * basis of range(Bi) in its first `rank` columns (zeros after), and W (k x k
 * row-major) is such that the least-norm solution of Bi^T d = r is
 * d = Q W r, and the least-squares solution of Bi mu = x is mu = W^T Q^T x.
 *   full rank:      Bi = Q R (thin QR, diag(R) > 0),  W = R^{-T}
 *   rank deficient: Bi = U S V^T (one-sided Jacobi SVD), Q = U_r,
 *                   W = S_r^{-1} V_r^T               (Algorithm 2, SVD branch)
 * Rank deficient means m < k, or R_jj^2 <= tol * max_j ||Bi(:,j)||^2; the SVD
 * drops singular values with s^2 <= tol * s_max^2.
 * Returns the rank, or -1 if the block is rank deficient and pinv == 0.
 * ------------------------------------------------------------------------ */
static int local_svd(int m, int k, const double *Bi, double *Q, double *W, double tol)
{
    /* one-sided (Hestenes) Jacobi on the columns of M = Bi; V accumulates */
    double *M = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * k);
    double V[64], s[8];
    int order[8];
    memcpy(M, Bi, sizeof(double) * (size_t)m * k);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) V[a * k + b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                double al = 0, be = 0, ga = 0;
                for (int r = 0; r < m; ++r) {
                    al += M[r * k + p] * M[r * k + p];
                    be += M[r * k + q] * M[r * k + q];
                    ga += M[r * k + p] * M[r * k + q];
                }
                if (fabs(ga) <= 1e-15 * sqrt(al * be) || ga == 0.0) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int r = 0; r < m; ++r) {
                    double x = M[r * k + p], y = M[r * k + q];
                    M[r * k + p] = c * x - sn * y;
                    M[r * k + q] = sn * x + c * y;
                }
                for (int r = 0; r < k; ++r) {
                    double x = V[r * k + p], y = V[r * k + q];
                    V[r * k + p] = c * x - sn * y;
                    V[r * k + q] = sn * x + c * y;
                }
            }
        if (!rotated) break;
    }
    double smax = 0;
    for (int j = 0; j < k; ++j) {
        double nn = 0;
        for (int r = 0; r < m; ++r) nn += M[r * k + j] * M[r * k + j];
        s[j] = sqrt(nn);
        if (s[j] > smax) smax = s[j];
        order[j] = j;
    }
    /* order by decreasing singular value (insertion sort, k <= 8) */
    for (int a = 1; a < k; ++a) {
        int v = order[a], b = a - 1;
        while (b >= 0 && s[order[b]] < s[v]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = v;
    }
    int rank = 0;
    memset(Q, 0, sizeof(double) * (size_t)m * k);
    memset(W, 0, sizeof(double) * (size_t)k * k);
    for (int a = 0; a < k; ++a) {
        int j = order[a];
        if (!(s[j] > 0) || s[j] * s[j] <= tol * smax * smax) continue;
        for (int r = 0; r < m; ++r) Q[r * k + rank] = M[r * k + j] / s[j];
        for (int b = 0; b < k; ++b) W[rank * k + b] = V[b * k + j] / s[j];
        ++rank;
    }
    free(M);
    return rank;
}

static int local_factor(int m, int k, const double *Bi, double *Q, double *W,
                        double tol, int pinv)
{
    if (k < 1 || k > 8) return -1;
    if (m < k) return pinv ? local_svd(m, k, Bi, Q, W, tol) : -1;
    /* Householder QR of the tall block (economy size), Algorithm 2 */
    double *Aw = (double *)malloc(sizeof(double) * (size_t)m * k);
    double *Vh = (double *)malloc(sizeof(double) * (size_t)m * k);
    double R[64], cn2max = 0;
    memcpy(Aw, Bi, sizeof(double) * (size_t)m * k);
    for (int j = 0; j < k; ++j) {
        double nn = 0;
        for (int r = 0; r < m; ++r) nn += Bi[r * k + j] * Bi[r * k + j];
        if (nn > cn2max) cn2max = nn;
    }
    memset(Vh, 0, sizeof(double) * (size_t)m * k);
    for (int j = 0; j < k; ++j) {
        double nx = 0;
        for (int r = j; r < m; ++r) nx += Aw[r * k + j] * Aw[r * k + j];
        nx = sqrt(nx);
        double x0 = Aw[j * k + j];
        double alpha = (x0 >= 0) ? -nx : nx;
        /* v = x - alpha e1, normalised */
        for (int r = j; r < m; ++r) Vh[r * k + j] = Aw[r * k + j];
        Vh[j * k + j] -= alpha;
        double nv = 0;
        for (int r = j; r < m; ++r) nv += Vh[r * k + j] * Vh[r * k + j];
        nv = sqrt(nv);
        if (nv > 0)
            for (int r = j; r < m; ++r) Vh[r * k + j] /= nv;
        /* apply H = I - 2 v v^T to the trailing columns */
        for (int c = j; c < k; ++c) {
            double d = 0;
            for (int r = j; r < m; ++r) d += Vh[r * k + j] * Aw[r * k + c];
            for (int r = j; r < m; ++r) Aw[r * k + c] -= 2.0 * Vh[r * k + j] * d;
        }
    }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) R[a * k + b] = (b >= a) ? Aw[a * k + b] : 0.0;
    int full = 1;
    for (int j = 0; j < k; ++j)
        if (!(R[j * k + j] * R[j * k + j] > tol * cn2max)) full = 0;
    if (!full) {
        free(Aw); free(Vh);
        return pinv ? local_svd(m, k, Bi, Q, W, tol) : -1;
    }
    /* thin Q = H_0 H_1 ... H_{k-1} [I_k; 0] */
    memset(Q, 0, sizeof(double) * (size_t)m * k);
    for (int j = 0; j < k; ++j) Q[j * k + j] = 1.0;
    for (int j = k - 1; j >= 0; --j)
        for (int c = 0; c < k; ++c) {
            double d = 0;
            for (int r = j; r < m; ++r) d += Vh[r * k + j] * Q[r * k + c];
            for (int r = j; r < m; ++r) Q[r * k + c] -= 2.0 * Vh[r * k + j] * d;
        }
    /* make diag(R) positive */
    for (int j = 0; j < k; ++j)
        if (R[j * k + j] < 0) {
            for (int b = 0; b < k; ++b) R[j * k + b] = -R[j * k + b];
            for (int r = 0; r < m; ++r) Q[r * k + j] = -Q[r * k + j];
        }
    /* W = R^{-T}: lower triangular, column by column (R^T W = I) */
    memset(W, 0, sizeof(double) * (size_t)k * k);
    for (int c = 0; c < k; ++c)
        for (int a = 0; a < k; ++a) {
            double v = (a == c) ? 1.0 : 0.0;
            for (int b = 0; b < a; ++b) v -= R[b * k + a] * W[b * k + c];
            W[a * k + c] = v / R[a * k + a];
        }
    free(Aw); free(Vh);
    return k;
}

/* ------------------------------------------------------------------------
 * Algorithm 2 (EMIN_SetUp), all rows free.  For every row i: gather B_i,
 * r_i = B(i,:)^T - B_i^T p0_i, factorise, delta_i = Q W r_i (least-norm
 * correction, Eq. (resEq) with the orientation read as B_i tall), and
 * p0_i += delta_i.  Q is stored per row at offset P_rowptr[i]*k, W at i*k*k.
 * ------------------------------------------------------------------------ */
int orc_setup(int n, int nc, int k, const int *Pp, const int *Pj, const double *Bc,
              const double *B, double *P0, double *Q, double *W, int *rank,
              double tol, int pinv, int *n_deficient)
{
    (void)nc;
    int ndef = 0, status = ORC_OK;
    int mmax = 0;
    for (int i = 0; i < n; ++i)
        if (Pp[i + 1] - Pp[i] > mmax) mmax = Pp[i + 1] - Pp[i];
    double *Bi = (double *)malloc(sizeof(double) * (size_t)(mmax + 1) * k);
    if (!Bi) return ORC_ERR_NOMEM;
    for (int i = 0; i < n; ++i) {
        int s0 = Pp[i], m = Pp[i + 1] - Pp[i];
        for (int s = 0; s < m; ++s)
            for (int c = 0; c < k; ++c) Bi[s * k + c] = Bc[(size_t)Pj[s0 + s] * k + c];
        double *Qi = Q + (size_t)s0 * k, *Wi = W + (size_t)i * k * k;
        int rk = local_factor(m, k, Bi, Qi, Wi, tol, pinv);
        if (rk < 0) { rank[i] = -1; status = ORC_ERR_RANK; continue; }
        rank[i] = rk;
        if (rk < k) ++ndef;
        double r[8], t[8];
        for (int c = 0; c < k; ++c) {
            double v = B[(size_t)i * k + c];
            for (int s = 0; s < m; ++s) v -= Bi[s * k + c] * P0[s0 + s];
            r[c] = v;
        }
        for (int a = 0; a < k; ++a) {
            double v = 0;
            for (int c = 0; c < k; ++c) v += Wi[a * k + c] * r[c];
            t[a] = v;
        }
        for (int s = 0; s < m; ++s) {
            double v = 0;
            for (int a = 0; a < k; ++a) v += Qi[s * k + a] * t[a];
            P0[s0 + s] += v;
        }
    }
    free(Bi);
    if (n_deficient) *n_deficient = ndef;
    return status;
}

/* Pi_B x = x - Q Q^T x, row by row (Pi_B = I - Q Q^T after Eq. (projSys)). */
void orc_project(int n, int k, const int *Pp, const double *Q, double *x)
{
    for (int i = 0; i < n; ++i) {
        int s0 = Pp[i], m = Pp[i + 1] - Pp[i];
        const double *Qi = Q + (size_t)s0 * k;
        double t[8];
        for (int a = 0; a < k; ++a) {
            double v = 0;
            for (int s = 0; s < m; ++s) v += Qi[s * k + a] * x[s0 + s];
            t[a] = v;
        }
        for (int s = 0; s < m; ++s) {
            double v = 0;
            for (int a = 0; a < k; ++a) v += Qi[s * k + a] * t[a];
            x[s0 + s] -= v;
        }
    }
}

/* K*y as the fixed-pattern product mask_P(A*Y) (Section 4): the full row
 * i of A*Y is accumulated in a dense scratch row of length nc, then read at
 * the columns J_i. */
int orc_kprod(int n, int nc, const int *Ap, const int *Aj, const double *Av,
              const int *Pp, const int *Pj, const double *Y, double *out)
{
    double *row = (double *)calloc((size_t)nc + 1, sizeof(double));
    if (!row) return ORC_ERR_NOMEM;
    for (int i = 0; i < n; ++i) {
        for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
            int l = Aj[e];
            double a = Av[e];
            for (int q = Pp[l]; q < Pp[l + 1]; ++q) row[Pj[q]] += a * Y[q];
        }
        for (int s = Pp[i]; s < Pp[i + 1]; ++s) out[s] = row[Pj[s]];
        /* clear every column touched by row i */
        for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
            int l = Aj[e];
            for (int q = Pp[l]; q < Pp[l + 1]; ++q) row[Pj[q]] = 0.0;
        }
    }
    free(row);
    return ORC_OK;
}

/* The Jacobi preconditioner M_J = diag(K): every entry of row i of P sits on
 * the diagonal A(i,i) of its column block (Theorem 1), so M_J^{-1} scales
 * row i by 1/A(i,i). */
int orc_diag_inverse(int n, const int *Ap, const int *Aj, const double *Av, double *dinv)
{
    for (int i = 0; i < n; ++i) {
        double d = 0;
        int found = 0;
        for (int e = Ap[i]; e < Ap[i + 1]; ++e)
            if (Aj[e] == i) { d = Av[e]; found = 1; }
        if (!found || !(d > 0)) return ORC_ERR_DIAG;
        dinv[i] = 1.0 / d;
    }
    return ORC_OK;
}

/* Position of entry (l, j) of P in the row-wise value arrays, -1 if row l
 * does not hold column j (columns of a row are sorted). */
static long find_entry(const int *Pp, const int *Pj, int l, int j)
{
    int lo = Pp[l], hi = Pp[l + 1];
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (Pj[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < Pp[l + 1] && Pj[lo] == j) ? (long)lo : -1;
}

/* ------------------------------------------------------------------------
 * Block symmetric Gauss-Seidel on K (Section 3.4, the M_SGS of the projected
 * SGS preconditioner M_2): z = (L + D)^{-T} D (L + D)^{-1} r with
 * K = L + D + L^T, p ordered row-wise.  K couples only entries of the same
 * column of P, so its block for column j is A(I_j, I_j) (I_j = the rows of P
 * holding column j), and in the row-wise order of p the rows of a block come
 * in increasing row index: L of a block is the strictly lower part of
 * A(I_j, I_j).  Each block is swept on its own:
 *   forward   (L + D) u = r     (rows of I_j in increasing order),
 *   diagonal  w = D u,
 *   backward  (L + D)^T z = w   (rows in decreasing order; the entry
 *             (L + D)^T(i, l) = K(l, i) = A(l, i) = A(i, l), A symmetric).
 * ------------------------------------------------------------------------ */
int orc_sgs_apply(int n, int nc, const int *Ap, const int *Aj, const double *Av,
                  const int *Pp, const int *Pj, const double *r, double *z)
{
    long nnz = Pp[n];
    /* the rows of every column of P, in increasing row order */
    int *colp = (int *)calloc((size_t)nc + 2, sizeof(int));
    int *crow = (int *)malloc(sizeof(int) * (size_t)(nnz + 1));
    long *cpos = (long *)malloc(sizeof(long) * (size_t)(nnz + 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!colp || !crow || !cpos || !u) {
        free(colp); free(crow); free(cpos); free(u);
        return ORC_ERR_NOMEM;
    }
    for (long q = 0; q < nnz; ++q) colp[Pj[q] + 1]++;
    for (int j = 0; j < nc; ++j) colp[j + 1] += colp[j];
    for (int i = 0; i < n; ++i)
        for (int q = Pp[i]; q < Pp[i + 1]; ++q) {
            int t = colp[Pj[q]]++;
            crow[t] = i;
            cpos[t] = q;
        }
    for (int j = nc; j > 0; --j) colp[j] = colp[j - 1];
    colp[0] = 0;
    int status = ORC_OK;
    for (int j = 0; j < nc && status == ORC_OK; ++j) {
        for (int t = colp[j]; t < colp[j + 1]; ++t) {
            int i = crow[t];
            double acc = r[cpos[t]], d = 0;
            for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
                int l = Aj[e];
                if (l == i) {
                    d = Av[e];
                } else if (l < i) {
                    long ql = find_entry(Pp, Pj, l, j);
                    if (ql >= 0) acc -= Av[e] * u[ql];
                }
            }
            if (!(d > 0)) { status = ORC_ERR_DIAG; break; }
            u[cpos[t]] = acc / d;
        }
        for (int t = colp[j + 1] - 1; t >= colp[j] && status == ORC_OK; --t) {
            int i = crow[t];
            double d = 0;
            for (int e = Ap[i]; e < Ap[i + 1]; ++e)
                if (Aj[e] == i) d = Av[e];
            double acc = d * u[cpos[t]];
            for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
                int l = Aj[e];
                if (l > i) {
                    long ql = find_entry(Pp, Pj, l, j);
                    if (ql >= 0) acc -= Av[e] * z[ql];
                }
            }
            z[cpos[t]] = acc / d;
        }
    }
    free(colp); free(crow); free(cpos); free(u);
    return status;
}

/* M^{-1} r for the preconditioners of Section 3.4: Jacobi M_J = diag(K)
 * (precond 0) or block SGS (precond 1). */
static int apply_minv(int n, int nc, const int *Ap, const int *Aj, const double *Av,
                      const int *Pp, const int *Pj, const double *dinv, int precond,
                      const double *r, double *z)
{
    if (precond == 1) return orc_sgs_apply(n, nc, Ap, Aj, Av, Pp, Pj, r, z);
    for (int i = 0; i < n; ++i)
        for (int s = Pp[i]; s < Pp[i + 1]; ++s) z[s] = dinv[i] * r[s];
    return ORC_OK;
}

double orc_dot(long nnz, const double *x, const double *y)
{
    double s = 0;
    for (long q = 0; q < nnz; ++q) s += x[q] * y[q];
    return s;
}

/* ------------------------------------------------------------------------
 * Algorithm 3 (EMIN_PCG) on Pi_B K Pi_B from the residual r (overwritten)
 * and the correction dw (accumulated, usually 0), with the Jacobi
 * preconditioner (precond 0) or the projected block SGS (precond 1).
 *   z = Pi_B M^{-1} r;  gamma = r^T z;  y = z (first) or z + (gamma/gamma_old) y;
 *   y_ = Pi_B K y;  alpha = gamma / y^T y_;  dE_k = gamma alpha;
 *   stop if dE_k < tau dE_1 (step not applied);  dw += alpha y;  r -= alpha y_.
 * gamma <= gamma_floor means the projected residual has reached rounding
 * level (or, at the first iteration, that there is no freedom at all): stop
 * with no step and no error.  The caller sets gamma_floor = 1e-28 times the
 * unprojected reference <b, M^{-1} b> (b = K p0 in the forward).
 * dE_hist receives dE_k of every computed iteration (*n_computed of them);
 * *n_applied counts the applied steps.  Returns ORC_ERR_BREAKDOWN if
 * y^T y_ <= 0 or a scalar is not finite.
 * ------------------------------------------------------------------------ */
int orc_pcg(int n, int nc, int k, const int *Ap, const int *Aj, const double *Av,
            const int *Pp, const int *Pj, const double *Q, const double *dinv,
            double *r, double *dw, int maxit, double tau, double gamma_floor,
            double *dE_hist, int *n_computed, int *n_applied, double *gamma_last,
            int precond)
{
    long nnz = Pp[n];
    double *z = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *yb = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!z || !y || !yb) { free(z); free(y); free(yb); return ORC_ERR_NOMEM; }
    double gamma_old = 0, dE1 = 0, gamma = 0;
    int status = ORC_OK, computed = 0, applied = 0;
    for (int it = 1; it <= maxit; ++it) {
        status = apply_minv(n, nc, Ap, Aj, Av, Pp, Pj, dinv, precond, r, z);
        if (status != ORC_OK) break;
        orc_project(n, k, Pp, Q, z);
        gamma = orc_dot(nnz, r, z);
        if (gamma <= gamma_floor) break;
        if (it == 1) {
            memcpy(y, z, sizeof(double) * (size_t)nnz);
        } else {
            double beta = gamma / gamma_old;
            for (long q = 0; q < nnz; ++q) y[q] = z[q] + beta * y[q];
        }
        gamma_old = gamma;
        orc_kprod(n, nc, Ap, Aj, Av, Pp, Pj, y, yb);
        orc_project(n, k, Pp, Q, yb);
        double yKy = orc_dot(nnz, y, yb);
        if (!(yKy > 0) || !isfinite(yKy) || !isfinite(gamma)) {
            status = ORC_ERR_BREAKDOWN;
            break;
        }
        double alpha = gamma / yKy;
        double dE = gamma * alpha;
        dE_hist[computed++] = dE;
        if (it == 1) dE1 = dE;
        if (dE < tau * dE1) break;
        for (long q = 0; q < nnz; ++q) dw[q] += alpha * y[q];
        for (long q = 0; q < nnz; ++q) r[q] -= alpha * yb[q];
        ++applied;
    }
    free(z); free(y); free(yb);
    *n_computed = computed;
    *n_applied = applied;
    if (gamma_last) *gamma_last = gamma;
    return status;
}

/* Energy tr(P^T A P) = <P, mask_P(A P)> (Eq. (trace)); P vanishes outside its
 * pattern, so the masked product loses nothing. */
int orc_energy(int n, int nc, const int *Ap, const int *Aj, const double *Av,
               const int *Pp, const int *Pj, const double *P, double *E)
{
    long nnz = Pp[n];
    double *KP = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!KP) return ORC_ERR_NOMEM;
    int st = orc_kprod(n, nc, Ap, Aj, Av, Pp, Pj, P, KP);
    *E = orc_dot(nnz, P, KP);
    free(KP);
    return st;
}

/* Whole forward: Algorithm 2 then Algorithm 3 with r = -Pi_B K p0 (f = 0,
 * every row of P free), then P = P0 + dw.  P is in: starting P0, out: P. */
int orc_minimize(int n, int nc, int k, const int *Ap, const int *Aj, const double *Av,
                 const int *Pp, const int *Pj, const double *B, const double *Bc,
                 double *P, double *P0_restored, double *Q, double *W, int *rank,
                 double tol, int pinv, int maxit, double tau,
                 double *dE_hist, int *n_computed, int *n_applied, int *n_deficient,
                 int precond)
{
    long nnz = Pp[n];
    int st = orc_setup(n, nc, k, Pp, Pj, Bc, B, P, Q, W, rank, tol, pinv, n_deficient);
    if (st != ORC_OK) return st;
    if (P0_restored) memcpy(P0_restored, P, sizeof(double) * (size_t)nnz);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *dw = (double *)calloc((size_t)nnz + 1, sizeof(double));
    if (!dinv || !r || !dw) { free(dinv); free(r); free(dw); return ORC_ERR_NOMEM; }
    st = orc_diag_inverse(n, Ap, Aj, Av, dinv);
    if (st == ORC_OK) {
        orc_kprod(n, nc, Ap, Aj, Av, Pp, Pj, P, r);
        double ref = 0;
        for (int i = 0; i < n; ++i)
            for (int s = Pp[i]; s < Pp[i + 1]; ++s) ref += r[s] * dinv[i] * r[s];
        orc_project(n, k, Pp, Q, r);
        for (long q = 0; q < nnz; ++q) r[q] = -r[q];
        st = orc_pcg(n, nc, k, Ap, Aj, Av, Pp, Pj, Q, dinv, r, dw, maxit, tau,
                     1e-28 * ref, dE_hist, n_computed, n_applied, NULL, precond);
        for (long q = 0; q < nnz; ++q) P[q] += dw[q];
    }
    free(dinv); free(r); free(dw);
    return st;
}

/* mask_A(U V^T): for every stored (a, b) of A, sum_c U(a,c) V(b,c) over the
 * columns c present in both row a of U and row b of V (U, V on P's pattern). */
int orc_outer(int n, int nc, const int *Ap, const int *Aj, const int *Pp, const int *Pj,
              const double *U, const double *V, double *out)
{
    double *row = (double *)calloc((size_t)nc + 1, sizeof(double));
    if (!row) return ORC_ERR_NOMEM;
    for (int a = 0; a < n; ++a) {
        for (int s = Pp[a]; s < Pp[a + 1]; ++s) row[Pj[s]] = U[s];
        for (int e = Ap[a]; e < Ap[a + 1]; ++e) {
            int b = Aj[e];
            double v = 0;
            for (int q = Pp[b]; q < Pp[b + 1]; ++q) v += row[Pj[q]] * V[q];
            out[e] = v;
        }
        for (int s = Pp[a]; s < Pp[a + 1]; ++s) row[Pj[s]] = 0.0;
    }
    free(row);
    return ORC_OK;
}

/* Per-row least squares B_i mu_i = x_i: mu_i = W^T Q^T x_i (n x k out). */
void orc_lsq(int n, int k, const int *Pp, const double *Q, const double *W,
             const double *x, double *mu)
{
    for (int i = 0; i < n; ++i) {
        int s0 = Pp[i], m = Pp[i + 1] - Pp[i];
        const double *Qi = Q + (size_t)s0 * k, *Wi = W + (size_t)i * k * k;
        double t[8];
        for (int a = 0; a < k; ++a) {
            double v = 0;
            for (int s = 0; s < m; ++s) v += Qi[s * k + a] * x[s0 + s];
            t[a] = v;
        }
        for (int b = 0; b < k; ++b) {
            double v = 0;
            for (int a = 0; a < k; ++a) v += Wi[a * k + b] * t[a];
            mu[(size_t)i * k + b] = v;
        }
    }
}

/* ------------------------------------------------------------------------
 * Implicit adjoint of the constrained minimiser P* (derived from the
 * saddle-point system (sadsys); the paper has no backward).  With
 * [2K C^T; C 0][u; mu] = [dL/dp; 0]:
 *   Pi K Pi u = 1/2 Pi dL/dp   (Algorithm 3 from u = 0, r = 1/2 Pi dL/dp),
 *   mu_i = least squares of B_i mu_i = (dL/dp - 2 K u)_i,
 *   dL/dA_ab = -2 (U P^T)_ab on A's pattern,  dL/dB(i,:) = mu_i.
 * P is the converged prolongation; the explicit dependence of L on A is the
 * caller's.  Q, W, dinv come from the forward set-up.
 * ------------------------------------------------------------------------ */
int orc_backward(int n, int nc, int k, const int *Ap, const int *Aj, const double *Av,
                 const int *Pp, const int *Pj, const double *Q, const double *W,
                 const double *P, const double *dLdP, int maxit, double tau,
                 double *U, double *dLdA, double *dLdB, int *n_applied, int precond)
{
    long nnz = Pp[n];
    double *dinv = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    double *hist = (double *)malloc(sizeof(double) * (size_t)(maxit + 1));
    if (!dinv || !r || !S || !hist) { free(dinv); free(r); free(S); free(hist); return ORC_ERR_NOMEM; }
    int st = orc_diag_inverse(n, Ap, Aj, Av, dinv);
    int computed = 0, applied = 0;
    if (st == ORC_OK) {
        double ref = 0;
        for (long q = 0; q < nnz; ++q) { r[q] = 0.5 * dLdP[q]; U[q] = 0.0; }
        for (int i = 0; i < n; ++i)
            for (int s = Pp[i]; s < Pp[i + 1]; ++s) ref += r[s] * dinv[i] * r[s];
        orc_project(n, k, Pp, Q, r);
        st = orc_pcg(n, nc, k, Ap, Aj, Av, Pp, Pj, Q, dinv, r, U, maxit, tau,
                     1e-28 * ref, hist, &computed, &applied, NULL, precond);
    }
    if (st == ORC_OK) {
        orc_kprod(n, nc, Ap, Aj, Av, Pp, Pj, U, S);
        for (long q = 0; q < nnz; ++q) S[q] = dLdP[q] - 2.0 * S[q];
        orc_lsq(n, k, Pp, Q, W, S, dLdB);
        orc_outer(n, nc, Ap, Aj, Pp, Pj, U, P, dLdA);
        for (long e = 0; e < (long)Ap[n]; ++e) dLdA[e] *= -2.0;
    }
    if (n_applied) *n_applied = applied;
    free(dinv); free(r); free(S); free(hist);
    return st;
}
