"""Thin Python binding of libemin (the C ABI of ``include/emin.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Inputs may be NumPy arrays (host) or CUDA tensors
of PyTorch (device; their stream is the stream given at creation).  The
library file must have been built (``__graft_entry__.build()`` or
``python -m paper_2208_02995_gb300.build``); importing it fails loudly
otherwise - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

EMIN_OK = 0
EMIN_ERR_ARG = -1
EMIN_ERR_PATTERN = -2
EMIN_ERR_RANK = -3
EMIN_ERR_DIAG = -4
EMIN_ERR_BREAKDOWN = -5
EMIN_ERR_CUDA = -6
EMIN_ERR_NOMEM = -7
EMIN_ERR_TIMEOUT = -8
EMIN_ERR_STATE = -9

EMIN_FP64 = 0
EMIN_MIXED = 1
EMIN_JACOBI = 0
EMIN_SGS = 1
EMIN_RANK_STRICT = 0
EMIN_RANK_PINV = 1

SYMBOLS = ("emin_default_opts", "emin_create", "emin_set_values", "emin_reset", "emin_iterate",
           "emin_energy", "emin_get_p", "emin_kprod", "emin_outer", "emin_backward",
           "emin_backward_unrolled",
           "emin_stats", "emin_sizes", "emin_strerror", "emin_destroy", "emin_set_timing",
           "emin_timing", "emin_masked_product_noalloc", "emin_last_error",
           "emin_trim_memory", "emin_energy_grad", "emin_fma_rate")


class emin_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("rank_policy", ctypes.c_int), ("checks", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class EminError(RuntimeError):
    def __init__(self, status, call):
        self.status = status
        detail = emin_last_error() if status in (EMIN_ERR_CUDA, EMIN_ERR_NOMEM) else ""
        super().__init__(f"{call}: {strerror(status)} (status {status})"
                         + (f" [{detail}]" if detail else ""))


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """The loaded libemin (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libemin.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        L.emin_default_opts.argtypes = [ctypes.POINTER(emin_opts)]
        L.emin_default_opts.restype = None
        L.emin_create.argtypes = [ctypes.POINTER(_VP), _I, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP,
                                  _VP, _VP, ctypes.POINTER(emin_opts), _I]
        L.emin_set_values.argtypes = [_VP, _VP, _VP, _VP, _I]
        L.emin_reset.argtypes = [_VP]
        L.emin_trim_memory.argtypes = []
        L.emin_iterate.argtypes = [_VP, _I, _D, ctypes.POINTER(_I), ctypes.POINTER(_D)]
        L.emin_energy.argtypes = [_VP, ctypes.POINTER(_D)]
        L.emin_get_p.argtypes = [_VP, _VP, _I]
        L.emin_kprod.argtypes = [_VP, _VP, _VP, _I, _I]
        L.emin_outer.argtypes = [_VP, _VP, _VP, _VP, _I]
        L.emin_energy_grad.argtypes = [_VP, _VP, _D, ctypes.POINTER(_D), _VP, _VP, _I]
        L.emin_fma_rate.argtypes = [_I, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP]
        L.emin_backward.argtypes = [_VP, _VP, _VP, _VP, _I, _D, _I, ctypes.POINTER(_I)]
        L.emin_backward_unrolled.argtypes = [_VP, _VP, _I, _VP, _VP, _I]
        L.emin_stats.argtypes = [_VP, _VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I)]
        L.emin_sizes.argtypes = [_VP, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong)]
        L.emin_strerror.argtypes = [_I]
        L.emin_strerror.restype = ctypes.c_char_p
        L.emin_last_error.argtypes = []
        L.emin_last_error.restype = ctypes.c_char_p
        L.emin_set_timing.argtypes = [_VP, _I]
        L.emin_timing.argtypes = [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_longlong)]
        L.emin_masked_product_noalloc.argtypes = [_I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                                  _VP, _VP]
        L.emin_destroy.argtypes = [_VP]
        L.emin_destroy.restype = None
        for s in SYMBOLS:
            if s not in ("emin_default_opts", "emin_strerror", "emin_destroy", "emin_last_error"):
                getattr(L, s).restype = _I
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().emin_strerror(int(status)).decode()


def emin_strerror(status: int) -> str:
    return strerror(status)


def emin_last_error() -> str:
    return lib().emin_last_error().decode()


def _check(status, call):
    if status != EMIN_OK:
        raise EminError(status, call)


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x, dtype, keep):
    """Pointer to the data of x (NumPy array or torch tensor), converted to
    a contiguous array of `dtype` when needed; `keep` holds temporaries."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        import torch
        tdt = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
        t = x.contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        keep.append(t)
        return t.data_ptr()
    a = np.ascontiguousarray(x, dtype=dtype)
    keep.append(a)
    return a.ctypes.data


# ---------------------------------------------------------------------------
# functions with the names of the C ABI
# ---------------------------------------------------------------------------
def emin_default_opts() -> emin_opts:
    o = emin_opts()
    lib().emin_default_opts(ctypes.byref(o))
    return o


def emin_create(n, nc, k, A_rowptr, A_col, A_val, P_rowptr, P_col, P0_val, B, Bc,
                opts: emin_opts | None = None, inputs_on_device: bool | None = None):
    keep = []
    if inputs_on_device is None:
        inputs_on_device = _is_cuda_tensor(A_rowptr)
    h = _VP()
    ptrs = [_ptr(A_rowptr, np.int32, keep), _ptr(A_col, np.int32, keep),
            _ptr(A_val, np.float64, keep), _ptr(P_rowptr, np.int32, keep),
            _ptr(P_col, np.int32, keep), _ptr(P0_val, np.float64, keep),
            _ptr(B, np.float64, keep), _ptr(Bc, np.float64, keep)]
    st = lib().emin_create(ctypes.byref(h), int(n), int(nc), int(k), *ptrs,
                           ctypes.byref(opts) if opts is not None else None, int(inputs_on_device))
    _check(st, "emin_create")
    return h


def emin_set_values(h, A_val=None, B=None, P0_val=None, on_device=False):
    keep = []
    _check(lib().emin_set_values(h, _ptr(A_val, np.float64, keep), _ptr(B, np.float64, keep),
                                 _ptr(P0_val, np.float64, keep), int(on_device)),
           "emin_set_values")


def emin_reset(h):
    _check(lib().emin_reset(h), "emin_reset")


def emin_iterate(h, n_iters, tol=0.0):
    done, rel = _I(0), _D(0)
    _check(lib().emin_iterate(h, int(n_iters), float(tol), ctypes.byref(done), ctypes.byref(rel)),
           "emin_iterate")
    return done.value, rel.value


def emin_energy(h) -> float:
    E = _D(0)
    _check(lib().emin_energy(h, ctypes.byref(E)), "emin_energy")
    return E.value


def emin_sizes(h):
    a, p = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(lib().emin_sizes(h, ctypes.byref(a), ctypes.byref(p)), "emin_sizes")
    return a.value, p.value


def emin_get_p(h, out=None):
    """P on P's pattern; into `out` (CUDA tensor or NumPy array) or a new
    NumPy array."""
    _, nnzp = emin_sizes(h)
    if out is None:
        out = np.empty(nnzp)
    dev = _is_cuda_tensor(out)
    ptr = out.data_ptr() if dev else out.ctypes.data
    _check(lib().emin_get_p(h, ptr, int(dev)), "emin_get_p")
    return out


def emin_kprod(h, X, project=True, out=None):
    _, nnzp = emin_sizes(h)
    keep = []
    dev = _is_cuda_tensor(X)
    if out is None:
        if dev:
            import torch
            out = torch.empty(nnzp, dtype=torch.float64, device=X.device)
        else:
            out = np.empty(nnzp)
    optr = out.data_ptr() if dev else out.ctypes.data
    _check(lib().emin_kprod(h, _ptr(X, np.float64, keep), optr, int(bool(project)), int(dev)),
           "emin_kprod")
    return out


def emin_outer(h, U, V, out=None):
    nnza, _ = emin_sizes(h)
    keep = []
    dev = _is_cuda_tensor(U)
    if out is None:
        if dev:
            import torch
            out = torch.empty(nnza, dtype=torch.float64, device=U.device)
        else:
            out = np.empty(nnza)
    optr = out.data_ptr() if dev else out.ctypes.data
    _check(lib().emin_outer(h, _ptr(U, np.float64, keep), _ptr(V, np.float64, keep), optr, int(dev)),
           "emin_outer")
    return out


def emin_energy_grad(h, X, scale=1.0, want_energy=True, want_dX=False, want_dA=False):
    """(E, dE/dX, dE/dA) for X on P's pattern; each part only when asked
    (else None).  Gradients are scaled by `scale`; they are CUDA tensors when
    X is one, else NumPy arrays."""
    nnza, nnzp = emin_sizes(h)
    keep = []
    dev = _is_cuda_tensor(X)

    def new(count):
        if dev:
            import torch
            return torch.empty(count, dtype=torch.float64, device=X.device)
        return np.empty(count)

    dX = new(nnzp) if want_dX else None
    dA = new(nnza) if want_dA else None
    E = _D(0)

    def ptr(a):
        if a is None:
            return None
        return a.data_ptr() if dev else a.ctypes.data

    _check(lib().emin_energy_grad(h, _ptr(X, np.float64, keep), float(scale),
                                  ctypes.byref(E) if want_energy else None, ptr(dX), ptr(dA),
                                  int(dev)), "emin_energy_grad")
    return (E.value if want_energy else None), dX, dA


def emin_backward(h, dL_dP, n_rows, k, max_adj_iters=200, adj_tol=0.0, want_A=True, want_B=True):
    """Returns (dL/dA values, dL/dB (n x k), adjoint steps)."""
    nnza, _ = emin_sizes(h)
    keep = []
    dev = _is_cuda_tensor(dL_dP)
    if dev:
        import torch
        dA = torch.empty(nnza, dtype=torch.float64, device=dL_dP.device) if want_A else None
        dB = torch.empty((n_rows, k), dtype=torch.float64, device=dL_dP.device) if want_B else None
        pa = dA.data_ptr() if want_A else None
        pb = dB.data_ptr() if want_B else None
    else:
        dA = np.empty(nnza) if want_A else None
        dB = np.empty((n_rows, k)) if want_B else None
        pa = dA.ctypes.data if want_A else None
        pb = dB.ctypes.data if want_B else None
    it = _I(0)
    _check(lib().emin_backward(h, _ptr(dL_dP, np.float64, keep), pa, pb, int(max_adj_iters),
                               float(adj_tol), int(dev), ctypes.byref(it)), "emin_backward")
    return dA, dB, it.value


def emin_backward_unrolled(h, dL_dP, n_rows, k, n_iters, want_A=True, want_B=True):
    """Gradient of exactly n_iters steps: returns (dL/dA values, dL/dB (n x k))."""
    nnza, _ = emin_sizes(h)
    keep = []
    dev = _is_cuda_tensor(dL_dP)
    if dev:
        import torch
        dA = torch.empty(nnza, dtype=torch.float64, device=dL_dP.device) if want_A else None
        dB = torch.empty((n_rows, k), dtype=torch.float64, device=dL_dP.device) if want_B else None
        pa = dA.data_ptr() if want_A else None
        pb = dB.data_ptr() if want_B else None
    else:
        dA = np.empty(nnza) if want_A else None
        dB = np.empty((n_rows, k)) if want_B else None
        pa = dA.ctypes.data if want_A else None
        pb = dB.ctypes.data if want_B else None
    _check(lib().emin_backward_unrolled(h, _ptr(dL_dP, np.float64, keep), int(n_iters), pa, pb,
                                        int(dev)), "emin_backward_unrolled")
    return dA, dB


def emin_stats(h, cap=4096):
    hist = np.zeros(max(cap, 1))
    nh, nd, na = _I(0), _I(0), _I(0)
    _check(lib().emin_stats(h, hist.ctypes.data, int(cap), ctypes.byref(nh), ctypes.byref(nd),
                            ctypes.byref(na)), "emin_stats")
    return {"dE": hist[:min(nh.value, cap)].copy(), "n_computed": nh.value,
            "n_rank_deficient": nd.value, "n_applied": na.value}


def emin_set_timing(h, period=1):
    """Time the masked product of every `period`-th iteration (0: off)."""
    _check(lib().emin_set_timing(h, int(period)), "emin_set_timing")


def emin_timing(h):
    """Per kernel class (kprod, ydir, update): summed event ms and launches;
    plus all kernels the library launched since the context was created."""
    ms = np.zeros(3)
    n = np.zeros(3, dtype=np.int64)
    tot = ctypes.c_longlong(0)
    _check(lib().emin_timing(h, ms.ctypes.data, n.ctypes.data, ctypes.byref(tot)), "emin_timing")
    return {"ms": ms, "launches": n, "total_launches": tot.value}


def emin_masked_product_noalloc(n, nc, A_rowptr, A_col, A_val, P_rowptr, P_col, Y, out, dot,
                                stream=None):
    """out = mask_P(A Y), dot[0] = <Y, out> for CUDA tensors, without any
    device allocation by the library (for callers whose device memory is
    owned by another allocator, or that cannot afford cudaMalloc's device
    synchronisation).  Queued on `stream` (default: the current torch
    stream); returns without waiting."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    # the kernel reads these arrays after the call returns, on the current
    # device: no host array and no converted temporary may be passed
    dev = torch.cuda.current_device()
    named = (("A_rowptr", A_rowptr, torch.int32), ("A_col", A_col, torch.int32),
             ("A_val", A_val, torch.float64), ("P_rowptr", P_rowptr, torch.int32),
             ("P_col", P_col, torch.int32), ("Y", Y, torch.float64),
             ("out", out, torch.float64), ("dot", dot, torch.float64))
    for name, t, dt in named:
        if not (_is_cuda_tensor(t) and t.dtype == dt and t.is_contiguous()
                and t.device.index == dev):
            raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor on the current "
                             f"device (cuda:{dev})")
    ptrs = [t.data_ptr() for _, t, _ in named]
    _check(lib().emin_masked_product_noalloc(int(n), int(nc), *ptrs, stream),
           "emin_masked_product_noalloc")
    return out, dot


def emin_fma_rate(precision="fp64", stream=None):
    """(FMAs per second, ms of the timed launch) of the current device's FMA
    pipe in double ("fp64") or float ("mixed")."""
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rate, ms = _D(0), _D(0)
    _check(lib().emin_fma_rate({"fp64": EMIN_FP64, "mixed": EMIN_MIXED}[precision],
                               ctypes.byref(rate), ctypes.byref(ms), stream), "emin_fma_rate")
    return rate.value, ms.value


def emin_destroy(h):
    if h:
        lib().emin_destroy(h)


def emin_trim_memory():
    """Give the device memory cached by destroyed contexts back to the driver."""
    _check(lib().emin_trim_memory(), "emin_trim_memory")


# ---------------------------------------------------------------------------
# convenience object
# ---------------------------------------------------------------------------
class Context:
    """Owns one library context.  ``precision``: "fp64" or "mixed";
    ``precond``: "jacobi" (M_1) or "sgs" (the projected block SGS, M_2);
    ``checks``: bounds checks in the gather kernels (see emin_opts.checks);
    ``stream``: a torch.cuda.Stream or raw cudaStream_t (int), default the
    current torch stream when inputs are CUDA tensors, else the legacy
    default stream."""

    def __init__(self, prob=None, *, n=None, nc=None, k=None, arrays=None, precision="fp64",
                 rank_policy="strict", stream=None, on_device=None, precond="jacobi",
                 checks=False):
        if prob is not None:
            n, nc, k, arrays = prob.n, prob.nc, prob.k, prob.arrays()
        self.n, self.nc, self.k = int(n), int(nc), int(k)
        opts = emin_default_opts()
        opts.precision = {"fp64": EMIN_FP64, "mixed": EMIN_MIXED}[precision]
        opts.rank_policy = {"strict": EMIN_RANK_STRICT, "pinv": EMIN_RANK_PINV}[rank_policy]
        opts.precond = {"jacobi": EMIN_JACOBI, "sgs": EMIN_SGS}[precond]
        opts.checks = 1 if checks else 0
        if on_device is None:
            on_device = _is_cuda_tensor(arrays[0])
        if stream is None and on_device:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        opts.stream = stream
        self.precision = precision
        self.precond = precond
        self.h = emin_create(self.n, self.nc, self.k, *arrays, opts=opts,
                             inputs_on_device=on_device)
        self.nnz_a, self.nnz_p = emin_sizes(self.h)

    def close(self):
        if getattr(self, "h", None):
            emin_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, n_iters, tol=0.0):
        return emin_iterate(self.h, n_iters, tol)

    def energy(self):
        return emin_energy(self.h)

    def get_p(self, out=None):
        return emin_get_p(self.h, out)

    def kprod(self, X, project=True, out=None):
        return emin_kprod(self.h, X, project, out)

    def outer(self, U, V, out=None):
        return emin_outer(self.h, U, V, out)

    def energy_grad(self, X, scale=1.0, want_energy=True, want_dX=False, want_dA=False):
        return emin_energy_grad(self.h, X, scale, want_energy, want_dX, want_dA)

    def backward(self, dL_dP, max_adj_iters=200, adj_tol=0.0):
        return emin_backward(self.h, dL_dP, self.n, self.k, max_adj_iters, adj_tol)

    def stats(self):
        return emin_stats(self.h)

    def backward_unrolled(self, dLdP, n_iters):
        """Gradient of exactly n_iters FP64 Jacobi steps (see emin.h)."""
        return emin_backward_unrolled(self.h, dLdP, self.n, self.k, n_iters)

    def reset(self):
        emin_reset(self.h)

    def set_values(self, A_val=None, B=None, P0_val=None, on_device=None):
        if on_device is None:
            on_device = any(_is_cuda_tensor(x) for x in (A_val, B, P0_val) if x is not None)
        emin_set_values(self.h, A_val, B, P0_val, on_device)
