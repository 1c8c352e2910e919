"""The tcgen05 split-TF32 GEMM tile (paper_2008_03237_gb300/csrc/pf12_tc.cuh)
against FP64 products, through a one-CTA harness built from the same header."""
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
    out = os.path.join(ROOT, "_build", "libtc_harness.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    src = os.path.join(ROOT, "tests", "csrc", "tc_harness.cu")
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", src, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.tc_harness.restype = ctypes.c_int
    lib.tc_harness.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int64] * 3 + \
        [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    return lib


def _run(lib, M, N, K, ta, tb, alpha=1.0, accumulate=False, seed=0):
    rng = np.random.default_rng(seed)
    Ad = rng.standard_normal((K, M) if ta else (M, K))
    Bd = rng.standard_normal((K, N) if tb else (N, K))
    Ar = Ad.T if ta else Ad            # A(r, t)
    Br = Bd.T if tb else Bd            # B(n, t)
    init = rng.standard_normal((N, M))
    ref = alpha * (Ar @ Br.T).T + (init if accumulate else 0.0)
    A = torch.from_numpy(Ad).cuda()
    B = torch.from_numpy(Bd).cuda()
    O = torch.from_numpy(init.copy()).cuda()
    flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = lib.tc_harness(M, N, K, A.data_ptr(), Ad.shape[1], B.data_ptr(), Bd.shape[1],
                        O.data_ptr(), M, int(ta), int(tb), alpha, int(accumulate), flag.data_ptr())
    assert rc == 0, rc
    assert int(flag.item()) == 0
    got = O.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    return err


@pytest.mark.parametrize("M,N,K", [(128, 16, 32), (128, 16, 8), (130, 40, 200), (300, 80, 517),
                                   (64, 8, 64), (257, 130, 96)])
@pytest.mark.parametrize("ta,tb", [(True, True), (False, False), (True, False), (False, True)])
def test_tc_gemm_matches_fp64(harness, M, N, K, ta, tb):
    err = _run(harness, M, N, K, ta, tb)
    assert err < 2e-6, err


def test_tc_gemm_accumulate_alpha(harness):
    err = _run(harness, 200, 33, 150, False, False, alpha=-1.0, accumulate=True, seed=3)
    assert err < 2e-6, err
