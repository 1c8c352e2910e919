"""The allocation-free entry point pf12_energy_noalloc against the context path.

pf12_energy_noalloc serves callers that cannot allocate device memory (code
running inside a memory pool or arena it does not own, plugins whose host
program owns every allocation, callers just refused more memory): its scratch
is a fixed 64 MiB array inside the library.  Here it is called twice in a row
through the C ABI and must reproduce the energies and V of the regular
pf12_upload_pairs / pf12_fit / pf12_energy path within the FP64 parity bar.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

import synthetic as S
from gpu_helpers import run, upload_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _call(lib, wl, t, lay, precision, V, e):
    """pf12_energy_noalloc through ctypes on torch's current stream; only
    host-side marshalling here (no device allocation, no read-back)."""
    from paper_2008_03237_gb300 import _lib as L
    kind = np.ascontiguousarray(wl.orb_kind.astype(np.int8))
    meta = [np.ascontiguousarray(a.astype(np.int32)) for a in (wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux)]
    offs = {n: np.ascontiguousarray(lay[n].astype(np.int64)) for n in ("off_pm", "off_mm", "off_pk", "off_kk")}
    tt = L.Tensors()
    for py, c in zip(("Agi", "Agj", "Afi", "Afj", "Jg", "Jf", "Q", "T"),
                     ("Ag_i", "Ag_j", "Af_i", "Af_j", "Jg", "Jf", "Q", "T")):
        setattr(tt, c, ctypes.c_void_p(t[py].data_ptr()))
    for n, a in offs.items():
        setattr(tt, n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    tt.len_pm, tt.len_mm = t["Agi"].numel(), t["Jg"].numel()
    tt.len_pk, tt.len_kk = t["Q"].numel(), t["T"].numel()
    E = ctypes.c_double(float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pf12_energy_noalloc(
        wl.n_orb, kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), wl.n_pairs,
        *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in meta], ctypes.byref(tt),
        L.PRECISION[precision], stream, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(e.data_ptr()),
        ctypes.byref(E))
    return rc, E.value


def _noalloc(lib, wl, t, lay, precision):
    V = torch.zeros(t["T"].numel(), dtype=torch.float64, device="cuda")
    e = torch.zeros((wl.n_pairs, 3), dtype=torch.float64, device="cuda")
    rc, E = _call(lib, wl, t, lay, precision, V, e)
    torch.cuda.synchronize()
    return rc, E, e.cpu().numpy(), V.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_noalloc_matches_context_path_twice(built, precision):
    import paper_2008_03237_gb300 as pf
    lib = pf.lib()
    wl = S.custom(5, 2, None, (40, 120), ("uniform", 1, 60), (30, 180), name="noalloc")
    t, lay = upload_host(wl)
    ref = run(wl, precision, t=t, lay=lay, want_V=True)
    Vref = np.concatenate([v.ravel() for v in ref["V"]])
    for call in range(2):
        rc, E, e, V = _noalloc(lib, wl, t, lay, precision)
        assert rc == 0, (call, rc)
        assert np.abs(e - ref["e_pair"]).max() <= 1e-10, call
        assert abs(E - ref["E"]) <= 1e-10 * max(1.0, abs(ref["E"])), call
        got = np.concatenate([S.unpack(V, lay["off_kk"], P, int(k), int(k)).ravel()
                              for P, k in enumerate(wl.n_pno)])
        assert np.abs(got - Vref).max() <= 1e-11 * np.abs(Vref).max(), call


def test_noalloc_rejects_sizes_beyond_its_scratch(built):
    import paper_2008_03237_gb300 as pf
    lib = pf.lib()
    from gpu_helpers import sized_workload
    wl = sized_workload([(8, 4, 4000)])      # one slab of ~128 MB > 64 MiB
    lay = S.packed_offsets(wl)
    t = {n: torch.zeros(max(lay[key], 2), dtype=torch.float64, device="cuda")
         for n, key in (("Agi", "len_pm"), ("Agj", "len_pm"), ("Afi", "len_pm"), ("Afj", "len_pm"),
                        ("Jg", "len_mm"), ("Jf", "len_mm"), ("Q", "len_pk"), ("T", "len_kk"))}
    rc, _, _, _ = _noalloc(lib, wl, t, lay, "fp64")
    assert rc == -1


def test_noalloc_reports_not_spd_pair_and_keeps_the_others(built):
    """A pair whose J_g is indefinite: the call returns PF12_ERR_NOT_SPD (-2),
    that pair's energies are NaN, and every other pair still matches the
    context path on the same inputs within the FP64 bar."""
    import paper_2008_03237_gb300 as pf
    lib = pf.lib()
    wl = S.custom(5, 2, None, (40, 120), ("uniform", 1, 60), (30, 180), name="noalloc-notspd")
    host, lay = S.packed_inputs(wl)
    bad = 4
    m = int(wl.n_aux[bad])
    o = lay["off_mm"][bad]
    host["Jg"][o:o + m * m].reshape(m, m)[...] -= 20.0 * np.eye(m)
    t, lay = upload_host(wl, (host, lay))
    eng = pf.PairF12("fp64")
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    _, e_ref = eng.energy(check=False)
    e_ref = e_ref.cpu().numpy()
    eng.close()
    for call in range(2):
        rc, E, e, _ = _noalloc(lib, wl, t, lay, "fp64")
        assert rc == -2, (call, rc)
        assert np.isnan(e[bad]).all()
        keep = np.arange(wl.n_pairs) != bad
        assert np.abs(e[keep] - e_ref[keep]).max() <= 1e-10, call


def test_noalloc_refuses_a_capturing_stream(built):
    """The call cannot be captured; it must say so before touching the capture."""
    import paper_2008_03237_gb300 as pf
    lib = pf.lib()
    wl = S.tiny()
    t, lay = upload_host(wl)
    V = torch.zeros(t["T"].numel(), dtype=torch.float64, device="cuda")
    e = torch.zeros((wl.n_pairs, 3), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    # an engine left unreferenced by an earlier test must not be finalised
    # (device frees) inside the capture: collect now, no collection during it
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                x.add_(1.0)
                rc, _ = _call(lib, wl, t, lay, "fp64", V, e)
            finally:
                g.capture_end()
    finally:
        gc.enable()
    assert rc == -7
    g.replay()                       # the caller's capture is intact
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0
