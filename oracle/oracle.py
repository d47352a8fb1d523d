"""Python front of the plain FP64 CPU oracle (``emin_oracle.c``).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` import this module; the product path
(``paper_2208_02995_gb300``) never does, and the oracle imports nothing from
it.  The C library is compiled on first use with gcc (``-O2
-ffp-contract=off``), single-threaded.

Every entry point follows one step of the paper's method:
  * ``setup``      Algorithm 2 (per-row QR, least-norm correction of P0)
  * ``project``    Pi_B = I - Q Q^T (Section 3.1)
  * ``kprod``      K y as the fixed-pattern product mask_P(A Y) (Section 4)
  * ``pcg``        Algorithm 3 with the Jacobi preconditioner (Section 3.4)
  * ``energy``     tr(P^T A P), Eq. (trace)
  * ``backward``   implicit adjoint of the minimiser, derived from (sadsys)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emin_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libemin_oracle.so")
_lock = threading.Lock()
_lib = None

RANK_TOL = 1e-12

_I = ctypes.POINTER(ctypes.c_int)
_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build`` (gcc, no OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_setup.restype = ctypes.c_int
            L.orc_kprod.restype = ctypes.c_int
            L.orc_pcg.restype = ctypes.c_int
            L.orc_energy.restype = ctypes.c_int
            L.orc_minimize.restype = ctypes.c_int
            L.orc_backward.restype = ctypes.c_int
            L.orc_outer.restype = ctypes.c_int
            L.orc_diag_inverse.restype = ctypes.c_int
            L.orc_sgs_apply.restype = ctypes.c_int
            L.orc_dot.restype = ctypes.c_double
            _lib = L
    return _lib


def _ip(a):
    return a.ctypes.data_as(_I)


def _dp(a):
    return a.ctypes.data_as(_D)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


class Oracle:
    """Plain FP64 oracle bound to one problem (A, pattern of P, B, B_c)."""

    PRECONDS = {"jacobi": 0, "sgs": 1}

    def __init__(self, prob, pinv: bool = False, tol: float = RANK_TOL, precond: str = "jacobi"):
        """precond: "jacobi" (M_1 of Section 3.4) or "sgs" (the projected
        block symmetric Gauss-Seidel M_2)."""
        self.precond = self.PRECONDS[precond]
        self.n, self.nc, self.k = prob.n, prob.nc, prob.k
        self.Ap, self.Aj, self.Av = _i32(prob.A_rowptr), _i32(prob.A_col), _f64(prob.A_val)
        self.Pp, self.Pj = _i32(prob.P_rowptr), _i32(prob.P_col)
        self.B, self.Bc = _f64(prob.B), _f64(prob.Bc)
        self.P0_in = _f64(prob.P0_val)
        self.pinv, self.tol = pinv, tol
        self.nnz_p = int(self.Pp[-1])
        self.nnz_a = int(self.Ap[-1])
        self._setup()

    # Algorithm 2
    def _setup(self):
        L = lib()
        self.P0 = self.P0_in.copy()
        self.Q = np.zeros(self.nnz_p * self.k + 1)
        self.W = np.zeros(self.n * self.k * self.k + 1)
        self.rank = np.zeros(self.n, dtype=np.int32)
        ndef = ctypes.c_int(0)
        st = L.orc_setup(self.n, self.nc, self.k, _ip(self.Pp), _ip(self.Pj), _dp(self.Bc),
                         _dp(self.B), _dp(self.P0), _dp(self.Q), _dp(self.W),
                         _ip(self.rank), ctypes.c_double(self.tol), int(self.pinv),
                         ctypes.byref(ndef))
        self.setup_status = st
        self.n_deficient = ndef.value
        if st != 0:
            raise OracleError(st, "set-up (Algorithm 2)")
        self.dinv = np.zeros(self.n)
        st = L.orc_diag_inverse(self.n, _ip(self.Ap), _ip(self.Aj), _dp(self.Av), _dp(self.dinv))
        if st != 0:
            raise OracleError(st, "diagonal")

    def kprod(self, Y):
        """mask_P(A Y) for Y on P's pattern."""
        Y = _f64(Y)
        out = np.zeros(self.nnz_p)
        lib().orc_kprod(self.n, self.nc, _ip(self.Ap), _ip(self.Aj), _dp(self.Av),
                        _ip(self.Pp), _ip(self.Pj), _dp(Y), _dp(out))
        return out

    def sgs(self, r):
        """(L + D)^{-T} D (L + D)^{-1} r, K = L + D + L^T block by block."""
        z = np.zeros(self.nnz_p)
        st = lib().orc_sgs_apply(self.n, self.nc, _ip(self.Ap), _ip(self.Aj), _dp(self.Av),
                                 _ip(self.Pp), _ip(self.Pj), _dp(_f64(r)), _dp(z))
        if st != 0:
            raise OracleError(st, "sgs")
        return z

    def project(self, x):
        x = _f64(x).copy()
        lib().orc_project(self.n, self.k, _ip(self.Pp), _dp(self.Q), _dp(x))
        return x

    def lsq(self, x):
        """Per-row least squares B_i mu_i = x_i (n x k)."""
        x = _f64(x)
        mu = np.zeros((self.n, self.k))
        lib().orc_lsq(self.n, self.k, _ip(self.Pp), _dp(self.Q), _dp(self.W), _dp(x), _dp(mu))
        return mu

    def energy(self, P):
        E = ctypes.c_double(0)
        lib().orc_energy(self.n, self.nc, _ip(self.Ap), _ip(self.Aj), _dp(self.Av),
                         _ip(self.Pp), _ip(self.Pj), _dp(_f64(P)), ctypes.byref(E))
        return E.value

    def outer(self, U, V):
        """mask_A(U V^T) on A's pattern."""
        out = np.zeros(self.nnz_a)
        lib().orc_outer(self.n, self.nc, _ip(self.Ap), _ip(self.Aj), _ip(self.Pp),
                        _ip(self.Pj), _dp(_f64(U)), _dp(_f64(V)), _dp(out))
        return out

    def initial_residual(self, P0=None):
        """r = -Pi_B K p0 (Algorithm 3 with f = 0) and the convergence floor
        1e-28 <K p0, M^{-1} K p0> of gamma."""
        Kp = self.kprod(self.P0 if P0 is None else P0)
        rows = np.repeat(np.arange(self.n), np.diff(self.Pp))
        floor = 1e-28 * float(np.sum(Kp * self.dinv[rows] * Kp))
        return -self.project(Kp), floor

    def pcg(self, r, maxit, tau=0.0, dw=None, gamma_floor=0.0):
        """Algorithm 3 from residual r; returns (dw, dE history, applied, status)."""
        r = _f64(r).copy()
        dw = np.zeros(self.nnz_p) if dw is None else _f64(dw).copy()
        hist = np.zeros(max(maxit, 1))
        nc_, na_ = ctypes.c_int(0), ctypes.c_int(0)
        g = ctypes.c_double(0)
        st = lib().orc_pcg(self.n, self.nc, self.k, _ip(self.Ap), _ip(self.Aj), _dp(self.Av),
                           _ip(self.Pp), _ip(self.Pj), _dp(self.Q), _dp(self.dinv),
                           _dp(r), _dp(dw), int(maxit), ctypes.c_double(tau),
                           ctypes.c_double(gamma_floor), _dp(hist),
                           ctypes.byref(nc_), ctypes.byref(na_), ctypes.byref(g),
                           int(self.precond))
        return dw, hist[:nc_.value].copy(), na_.value, st

    def minimize(self, maxit, tau=0.0):
        """Algorithms 2 + 3: returns dict(P, P0, dE, applied, status)."""
        r, floor = self.initial_residual()
        dw, hist, applied, st = self.pcg(r, maxit, tau, gamma_floor=floor)
        return {"P": self.P0 + dw, "P0": self.P0.copy(), "dE": hist,
                "applied": applied, "status": st}

    def backward(self, P, dLdP, maxit, tau=0.0):
        """Implicit adjoint: returns (dL/dA values, dL/dB (n x k), U, applied)."""
        U = np.zeros(self.nnz_p)
        dA = np.zeros(self.nnz_a)
        dB = np.zeros((self.n, self.k))
        na_ = ctypes.c_int(0)
        st = lib().orc_backward(self.n, self.nc, self.k, _ip(self.Ap), _ip(self.Aj),
                                _dp(self.Av), _ip(self.Pp), _ip(self.Pj), _dp(self.Q),
                                _dp(self.W), _dp(_f64(P)), _dp(_f64(dLdP)), int(maxit),
                                ctypes.c_double(tau), _dp(U), _dp(dA), _dp(dB),
                                ctypes.byref(na_), int(self.precond))
        if st != 0:
            raise OracleError(st, "backward")
        return dA, dB, U, na_.value

    def constraint_error(self, P):
        """max-abs entry of P B_c - B."""
        rows = np.repeat(np.arange(self.n), np.diff(self.Pp))
        PB = np.zeros((self.n, self.k))
        np.add.at(PB, rows, P[:, None] * self.Bc[self.Pj])
        return float(np.abs(PB - self.B).max()) if self.n else 0.0
