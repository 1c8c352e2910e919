"""Fill packed workload tensors directly in device memory (bit-identical to the
host generator in workloads.py), for workloads too large to draw on the host.

Uses libpf12synth.so (synthetic/csrc/synth_gen.cu): Philox4x32-10 draws of the
DF factors and of the integer matrices behind J = c2 Z Z^T + 0.1 I.  Q and T
are drawn on the host and copied.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf12synth.so")
_SRC = os.path.join(_HERE, "csrc", "synth_gen.cu")

META = np.dtype([("off", "<i8"), ("rows", "<i4"), ("cols", "<i4"), ("key", "<i4"),
                 ("tid", "<i4"), ("scale", "<f8")])
_lib = None


def build(force=False):
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) > os.path.getmtime(_SRC):
        return LIB_PATH
    nvcc = "nvcc"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", _SRC, "-o", LIB_PATH + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building libpf12synth failed:\n" + r.stderr)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} missing: run synthetic.device.build()")
        _lib = ctypes.CDLL(LIB_PATH)
        _lib.synth_fill_gauss16.restype = ctypes.c_int
        _lib.synth_fill_gauss16.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                            ctypes.c_void_p, ctypes.c_void_p]
        _lib.synth_fill_metrics.restype = ctypes.c_int
        _lib.synth_fill_metrics.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_double, ctypes.c_uint32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return _lib


def allocate(wl, device="cuda", with_metrics=True):
    """Zeroed packed float64 tensors for wl and their offsets."""
    import torch
    lay = W.packed_offsets(wl)
    t = {}
    for n in ("Agi", "Agj", "Afi", "Afj"):
        t[n] = torch.zeros(max(lay["len_pm"], 2), dtype=torch.float64, device=device)
    if with_metrics:
        for n in ("Jg", "Jf"):
            t[n] = torch.zeros(max(lay["len_mm"], 2), dtype=torch.float64, device=device)
    t["Q"] = torch.zeros(max(lay["len_pk"], 2), dtype=torch.float64, device=device)
    t["T"] = torch.zeros(max(lay["len_kk"], 2), dtype=torch.float64, device=device)
    return t, lay


def fill(wl, t, lay, scratch_bytes=1 << 30):
    """Draw every pair of wl into the packed device tensors t (from allocate)."""
    import torch
    lib = _load()
    n = wl.n_pairs
    if n == 0:
        return t
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    keys = np.array([wl.pair_key(P) for P in range(n)], np.int32)
    diag = wl.pi == wl.pj
    scale = np.array([W.factor_scale(s) for s in wl.decay], np.float64)
    tids = {"Agi": W.TID_AGI, "Agj": W.TID_AGJ, "Afi": W.TID_AFI, "Afj": W.TID_AFJ}
    for name, tid in tids.items():
        meta = np.zeros(n, META)
        meta["off"] = lay["off_pm"]
        meta["rows"] = wl.n_rows
        meta["cols"] = wl.n_aux
        meta["key"] = keys
        tt = np.full(n, tid, np.int32)
        if name == "Agj":
            tt[diag] = W.TID_AGI
        if name == "Afj":
            tt[diag] = W.TID_AFI
        meta["tid"] = tt
        meta["scale"] = scale
        rc = lib.synth_fill_gauss16(n, meta.ctypes.data, W_seed(wl), ctypes.c_void_p(t[name].data_ptr()), stream)
        if rc != 0:
            raise RuntimeError(f"synth_fill_gauss16 failed ({rc})")
    if "Jg" in t:
        mmax = int(wl.n_aux.max())
        elems = max(scratch_bytes // 4, mmax * mmax)
        scratch = torch.empty(elems, dtype=torch.float32, device=t["Jg"].device)
        c2 = np.array([W.metric_scale(m) for m in wl.n_aux], np.float64)
        for name, tid in (("Jg", W.TID_XG), ("Jf", W.TID_XF)):
            meta = np.zeros(n, META)
            meta["off"] = lay["off_mm"]
            meta["rows"] = wl.n_aux
            meta["cols"] = wl.n_aux
            meta["key"] = keys
            meta["tid"] = tid
            rc = lib.synth_fill_metrics(n, meta.ctypes.data, c2.ctypes.data, wl.metric_shift,
                                        W_seed(wl), ctypes.c_void_p(t[name].data_ptr()),
                                        ctypes.c_void_p(scratch.data_ptr()), elems, stream)
            if rc != 0:
                raise RuntimeError(f"synth_fill_metrics failed ({rc})")
        del scratch
    q = np.zeros(lay["len_pk"])
    tt = np.zeros(lay["len_kk"])
    for P in range(n):
        Q = W.pno_coefficients(wl, P)
        T = W.amplitudes(wl, P)
        o = lay["off_pk"][P]
        q[o:o + Q.size] = Q.ravel()
        o = lay["off_kk"][P]
        tt[o:o + T.size] = T.ravel()
    t["Q"][:q.size].copy_(torch.from_numpy(q))
    t["T"][:tt.size].copy_(torch.from_numpy(tt))
    torch.cuda.synchronize()
    return t


def W_seed(wl):
    return ctypes.c_uint32(wl.seed & 0xFFFFFFFF)
