"""Fill packed workload tensors directly in device memory (bit-identical to the
host generator in workloads.py), for workloads too large to draw on the host.

Uses libpf12synth.so (synthetic/csrc/synth_gen.cu): Philox4x32-10 draws of the
DF factors and of the integer matrices behind J = c2 Z Z^T + 0.1 I.  Q and T
are drawn on the host first and copied last.
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
    q_host, t_host = host_pno_and_amplitudes(wl, lay)
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
    t["Q"][:q_host.size].copy_(torch.from_numpy(q_host))
    t["T"][:t_host.size].copy_(torch.from_numpy(t_host))
    torch.cuda.current_stream().synchronize()   # this stream only: callers may overlap it
    return t


def host_pno_and_amplitudes(wl, lay):
    """Q and T of every pair of wl, drawn on the host into packed arrays.  The
    fills draw these first: this host work then overlaps whatever the device
    is still running, before the device fills queue behind it."""
    q = np.zeros(lay["len_pk"])
    tt = np.zeros(lay["len_kk"])
    for P in range(wl.n_pairs):
        Q = W.pno_coefficients(wl, P)
        T = W.amplitudes(wl, P)
        o = lay["off_pk"][P]
        q[o:o + Q.size] = Q.ravel()
        o = lay["off_kk"][P]
        tt[o:o + T.size] = T.ravel()
    return q, tt


FULL_META = np.dtype([("dst", "<i8"), ("src", "<i8"), ("p", "<i4"), ("k", "<i4"), ("m", "<i4"),
                      ("key", "<i4"), ("tid", "<i4"), ("tid2", "<i4"), ("tid3", "<i4"),
                      ("canon", "<i4"), ("scale", "<f8"), ("eps", "<f8")])


def allocate_full(wl, device="cuda"):
    """Zeroed packed float64 tensors of the full-energy layout and its offsets."""
    import torch
    from . import full as FU
    lay = FU.full_offsets(wl)
    t = {}
    for n in FU.FACTOR_NAMES:
        t[n] = torch.zeros(max(lay["len_pm"], 2), dtype=torch.float64, device=device)
    for n in FU.METRIC_NAMES:
        t[n] = torch.zeros(max(lay["len_mm"], 2), dtype=torch.float64, device=device)
    for n, key in (("Q", "pk"), ("T", "kk"), ("Fv", "pp"), ("S", "s"), ("B", "b")):
        t[n] = torch.zeros(max(lay["len_" + key], 2), dtype=torch.float64, device=device)
    return t, lay


def fill_full(wl, t, lay, scratch_bytes=1 << 30):
    """Draw every pair of wl's full-energy inputs into t (from allocate_full),
    bit-identical to synthetic.full.full_packed_inputs."""
    import torch
    from . import full as FU
    lib = _load()
    if not hasattr(lib, "_full_set"):
        lib.synth_fill_full.restype = ctypes.c_int
        lib.synth_fill_full.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib._full_set = True
    n = wl.n_pairs
    if n == 0:
        return t
    q_host, t_host = host_pno_and_amplitudes(wl, lay)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    seed = W_seed(wl)
    keys = np.array([wl.pair_key(P) for P in range(n)], np.int32)
    diag = wl.pi == wl.pj
    p = wl.n_pao.astype(np.int64)
    k = wl.n_pno.astype(np.int64)
    m = wl.n_aux.astype(np.int64)
    c = np.array([W.factor_scale(s) for s in wl.decay], np.float64)
    off = lay["off_pm"]

    def gauss(name, offs, rows, cols, tids, scale):
        meta = np.zeros(n, META)
        meta["off"], meta["rows"], meta["cols"], meta["key"] = offs, rows, cols, keys
        meta["tid"], meta["scale"] = tids, scale
        rc = lib.synth_fill_gauss16(n, meta.ctypes.data, seed, ctypes.c_void_p(t[name].data_ptr()), stream)
        if rc != 0:
            raise RuntimeError(f"synth_fill_gauss16 failed ({rc})")

    def tid(a, b=None):
        x = np.full(n, a, np.int32)
        if b is not None:
            x[diag] = b
        return x
    # PAO rows of the Coulomb and V-kernel factors: the amplitude-term streams
    gauss("Agi", off, p, m, tid(W.TID_AGI), c)
    gauss("Agj", off, p, m, tid(W.TID_AGJ, W.TID_AGI), c)
    gauss("Afi", off, p, m, tid(W.TID_AFI), c)
    gauss("Afj", off, p, m, tid(W.TID_AFJ, W.TID_AFI), c)
    # occupied rows: i blocks (ii, ij), j blocks (ij, jj); all ii on a diagonal pair
    for x, (tii, tjj, tij) in (("g", (FU.TID_OCCG_II, FU.TID_OCCG_JJ, FU.TID_OCCG_IJ)),
                               ("f", (FU.TID_OCCF_II, FU.TID_OCCF_JJ, FU.TID_OCCF_IJ))):
        co = c * FU.OCC_SCALE
        gauss("A%si" % x, off + p * m, 1, m, tid(tii), co)
        gauss("A%si" % x, off + (p + 1) * m, 1, m, tid(tij, tii), co)
        gauss("A%sj" % x, off + p * m, 1, m, tid(tij, tii), co)
        gauss("A%sj" % x, off + (p + 1) * m, 1, m, tid(tjj, tii), co)
    cr = c * FU.R_SCALE
    gauss("Ari", off, p, m, tid(FU.TID_ARI), cr)
    gauss("Arj", off, p, m, tid(FU.TID_ARJ, FU.TID_ARI), cr)
    # Fock-transformed factors from the PAO rows just drawn
    eps = FU.orbital_energies(wl)
    canon = int(FU.canonical(wl))
    for dst, src, orb, t_nd, t_d, sc in (("AgiF", "Agi", wl.pi, FU.TID_NGIF, FU.TID_NGIF, c),
                                         ("AgjF", "Agj", wl.pj, FU.TID_NGJF, FU.TID_NGIF, c),
                                         ("AriF", "Ari", wl.pi, FU.TID_NRIF, FU.TID_NRIF, cr),
                                         ("ArjF", "Arj", wl.pj, FU.TID_NRJF, FU.TID_NRIF, cr)):
        meta = np.zeros(n, FULL_META)
        meta["dst"], meta["src"], meta["p"], meta["k"], meta["m"] = off, off, p, k, m
        meta["key"], meta["tid"], meta["canon"] = keys, tid(t_nd, t_d), canon
        meta["scale"], meta["eps"] = sc * FU.FOCK_NOISE, eps[orb]
        rc = lib.synth_fill_full(0, n, meta.ctypes.data, seed, ctypes.c_void_p(t[src].data_ptr()),
                                 ctypes.c_void_p(t[dst].data_ptr()), stream)
        if rc != 0:
            raise RuntimeError(f"synth_fill_full failed ({rc})")
    # metrics: J_g, J_f as for the amplitude term, J_r scaled by the geminal's power of two
    mmax = int(m.max())
    elems = max(scratch_bytes // 4, mmax * mmax)
    scratch = torch.empty(elems, dtype=torch.float32, device=t["Jg"].device)
    c2 = np.array([W.metric_scale(x) for x in wl.n_aux], np.float64)
    for name, tidm in (("Jg", W.TID_XG), ("Jf", W.TID_XF), ("Jr", FU.TID_XR)):
        meta = np.zeros(n, META)
        meta["off"], meta["rows"], meta["cols"], meta["key"], meta["tid"] = lay["off_mm"], m, m, keys, tidm
        rc = lib.synth_fill_metrics(n, meta.ctypes.data, c2.ctypes.data, wl.metric_shift, seed,
                                    ctypes.c_void_p(t[name].data_ptr()),
                                    ctypes.c_void_p(scratch.data_ptr()), elems, stream)
        if rc != 0:
            raise RuntimeError(f"synth_fill_metrics failed ({rc})")
    del scratch
    t["Jr"].mul_(FU.R_SCALE)                 # a power of two: exact
    # virtual Fock blocks, singles, PNO-pair factors
    for kind, name, offs, tids in ((1, "Fv", lay["off_pp"], (FU.TID_FV, 0, 0)),
                                   (2, "B", lay["off_b"], (FU.TID_B, FU.TID_B_I, FU.TID_B_J))):
        meta = np.zeros(n, FULL_META)
        meta["dst"], meta["p"], meta["k"], meta["m"], meta["key"] = offs, p, k, m, keys
        meta["tid"], meta["tid2"], meta["tid3"] = tids[0], tids[1], tid(tids[2], tids[1]) if kind == 2 else 0
        meta["canon"] = canon if kind == 1 else 0
        meta["scale"] = (W.IH16_INV_STD * FU.FV_OFFDIAG) if kind == 1 else (W.IH16_INV_STD * FU.B_SCALE)
        rc = lib.synth_fill_full(kind, n, meta.ctypes.data, seed, None,
                                 ctypes.c_void_p(t[name].data_ptr()), stream)
        if rc != 0:
            raise RuntimeError(f"synth_fill_full failed ({rc})")
    cs = W.IH16_INV_STD * FU.SINGLES_STD
    gauss("S", lay["off_s"], 1, k, tid(FU.TID_S_I), cs)
    gauss("S", lay["off_s"] + k, 1, k, tid(FU.TID_S_J, FU.TID_S_I), cs)
    # Q, T from the host
    t["Q"][:q_host.size].copy_(torch.from_numpy(q_host))
    t["T"][:t_host.size].copy_(torch.from_numpy(t_host))
    torch.cuda.current_stream().synchronize()   # this stream only: callers may overlap it
    return t


def W_seed(wl):
    return ctypes.c_uint32(wl.seed & 0xFFFFFFFF)
