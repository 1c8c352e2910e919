"""The integer FP64 -> FP32 (round to nearest even) and FP32 -> FP64 conversions
of the mixed-precision GEMM tiles (paper_2008_03237_gb300/csrc/pf12_device.cuh)
against the hardware conversions, bit for bit: random values over the whole
exponent range, ties (odd and even kept fraction), values one unit either side
of a tie, the normal / subnormal boundary, the overflow boundary, zeros,
subnormals, infinities and NaN.  A NaN input must give a NaN of either
width; its payload is not compared (the integer conversions return a quiet
NaN with the input's sign, not the hardware's canonical pattern)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness():
    out = os.path.join(ROOT, "_build", "libconvert_harness.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    src = os.path.join(ROOT, "tests", "csrc", "convert_harness.cu")
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", src, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.convert_harness.restype = ctypes.c_int
    lib.convert_harness.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 5
    return lib


def _doubles(rng, n):
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    exp = rng.integers(1023 - 160, 1023 + 140, n, dtype=np.uint64) << np.uint64(52)
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    rand = (sign | exp | frac).view(np.float64)
    # ties and their neighbours: a float's fraction followed by 29 chosen bits
    f = rng.standard_normal(n).astype(np.float32) * np.float32(2.0) ** rng.integers(-120, 120, n)
    base = f.astype(np.float64).view(np.uint64)
    ties = []
    for rest in (0x10000000, 0x0FFFFFFF, 0x10000001, 0x1FFFFFFF, 0x00000001):
        ties.append((base | np.uint64(rest)).view(np.float64))
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, tiny, -tiny, tiny * (1 - 2 ** -30),
                        tiny * (1 + 2 ** -24), 2.0 ** -149, 2.0 ** -150, 2.0 ** -151, fmax, -fmax,
                        fmax + 2.0 ** 103, fmax + 2.0 ** 103 - 2.0 ** 80, fmax * 2, 1e300, -1e-300,
                        5e-324, 1.0, -1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 3.0, 0.1],
                       dtype=np.float64)
    return np.concatenate([rand] + ties + [special])


def _floats(rng, n):
    bits = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40, 1.0, 3.4e38],
                       dtype=np.float32)
    return np.concatenate([bits.view(np.float32), special])


def test_conversions_bitwise(harness):
    rng = np.random.default_rng(2008)
    x = _doubles(rng, 200_000)
    y = _floats(rng, 200_000)
    n = max(len(x), len(y))
    x = np.resize(x, n)
    y = np.resize(y, n)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    f_int = torch.empty(n, dtype=torch.float32, device="cuda")
    f_hw = torch.empty_like(f_int)
    d_int = torch.empty(n, dtype=torch.float64, device="cuda")
    d_hw = torch.empty_like(d_int)
    rc = harness.convert_harness(xd.data_ptr(), n, f_int.data_ptr(), f_hw.data_ptr(), yd.data_ptr(),
                                 d_int.data_ptr(), d_hw.data_ptr())
    assert rc == 0, rc
    fi = f_int.cpu().numpy()
    a, b = fi.view(np.uint32), f_hw.cpu().numpy().view(np.uint32)
    nan_x = np.isnan(x)
    assert np.isnan(fi[nan_x]).all()
    bad = np.nonzero((a != b) & ~nan_x)[0]
    assert bad.size == 0, [(x[i], hex(a[i]), hex(b[i])) for i in bad[:5]]
    di = d_int.cpu().numpy()
    c, d = di.view(np.uint64), d_hw.cpu().numpy().view(np.uint64)
    nan_y = np.isnan(y)
    assert np.isnan(di[nan_y]).all()
    bad = np.nonzero((c != d) & ~nan_y)[0]
    assert bad.size == 0, [(y[i], hex(c[i]), hex(d[i])) for i in bad[:5]]
    # the host's IEEE conversion agrees as well (finite inputs)
    fin = np.isfinite(x)
    with np.errstate(over="ignore"):
        host = x[fin].astype(np.float32)
    assert np.array_equal(a[fin], host.view(np.uint32))
