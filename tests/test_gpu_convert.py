"""The integer-pipe conversions of csrc/convert.cuh against the GPU's own
double <-> float conversions, bit for bit, on the cases IEEE 754's
roundTiesToEven has to get right: exact ties in the normal and subnormal
ranges, the overflow threshold, the underflow to zero, signed zeros,
infinities, NaN, and random bit patterns over every exponent."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2208_02995_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = str(tmp_path_factory.mktemp("convert") / "convert_check.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC,
                           os.path.join(HERE, "convert_check.cu"), "-o", so])
    return ctypes.CDLL(so)


def f64_cases(rng):
    parts = []
    # random bit patterns: every exponent, mostly far outside the float range
    parts.append(rng.integers(0, 2**64, 200_000, dtype=np.uint64).view(np.float64))
    # exponents around the float range, from below the subnormals to overflow
    e = rng.integers(-160, 131, 400_000)
    m = rng.random(400_000) + 1.0
    parts.append(np.ldexp(m, e) * rng.choice([-1.0, 1.0], 400_000))
    # exact ties and their neighbours: float values plus / minus half an ulp
    fb = rng.integers(0, 0x7f800000, 200_000, dtype=np.uint32)
    f = fb.view(np.float32).astype(np.float64)
    up = np.nextafter(fb.view(np.float32), np.float32(np.inf)).astype(np.float64)
    mid = f + (up - f) / 2  # exact in double, ties between consecutive floats
    parts += [mid, -mid, np.nextafter(mid, 0.0), np.nextafter(mid, np.inf)]
    fmax = float(np.finfo(np.float32).max)
    tiny = 2.0 ** -149
    special = [0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0 ** -25),
               fmax * (1 + 2.0 ** -24), np.nextafter(fmax * (1 + 2.0 ** -24), 0.0), 2.0 ** 128,
               tiny, tiny / 2, np.nextafter(tiny / 2, 1.0), tiny * 1.5, tiny * 2.5,
               2.0 ** -126, np.nextafter(2.0 ** -126, 0.0), 2.0 ** -126 - tiny / 2,
               5e-324, -5e-324, 2.0 ** -1022, 1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24,
               0.1, 1e-40, 1e-45, 3e38, 3.5e38]
    parts.append(np.array(special))
    return np.concatenate(parts)


def test_conversions_match_hardware(lib):
    import torch
    rng = np.random.default_rng(7)
    x = f64_cases(rng)
    fb = np.concatenate([rng.integers(0, 2**32, 500_000, dtype=np.uint64).astype(np.uint32),
                         np.arange(0, 0x800000, 97, dtype=np.uint32),  # subnormals
                         np.array([0, 0x80000000, 0x7f800000, 0xff800000, 0x7fc00000,
                                   0x7f800001, 0x00000001, 0x007fffff, 0x00800000,
                                   0x7f7fffff], dtype=np.uint32)])
    f = fb.view(np.float32)
    n = max(len(x), len(f))
    x = np.resize(x, n)
    f = np.resize(f, n)
    dx = torch.from_numpy(x).cuda()
    df = torch.from_numpy(f).cuda()
    sw32 = torch.empty(n, dtype=torch.float32, device="cuda")
    hw32 = torch.empty_like(sw32)
    sw64 = torch.empty(n, dtype=torch.float64, device="cuda")
    hw64 = torch.empty_like(sw64)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.convert_check(ctypes.c_longlong(n), vp(dx), vp(sw32), vp(hw32), vp(df), vp(sw64),
                             vp(hw64)) == 0
    a, b = sw32.cpu().numpy(), hw32.cpu().numpy()
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    bad = np.flatnonzero(a[~nan].view(np.uint32) != b[~nan].view(np.uint32))
    assert bad.size == 0, (x[~nan][bad[:5]], a[~nan][bad[:5]], b[~nan][bad[:5]])
    # and against numpy's own IEEE narrowing
    with np.errstate(over="ignore"):
        ref = x[~nan].astype(np.float32)
    assert np.array_equal(a[~nan].view(np.uint32), ref.view(np.uint32))
    a, b = sw64.cpu().numpy(), hw64.cpu().numpy()
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    assert np.array_equal(a[~nan].view(np.uint64), b[~nan].view(np.uint64))
    assert np.array_equal(a[~nan].view(np.uint64), f[~nan].astype(np.float64).view(np.uint64))
