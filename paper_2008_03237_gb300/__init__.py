"""GB300-native pair-F12 energy path (arXiv 2008.03237) -- Python binding.

Every step of the path runs in libpairf12.so (hand-written sm_103a kernels);
this module only marshals arguments through the C ABI of include/pairf12.h and
wraps the energy in a torch.autograd.Function whose backward calls the
library's adjoint kernel.  PyTorch supplies device memory and streams.
"""
import ctypes

import numpy as np
import torch

from . import _lib

__all__ = ["PairF12", "PairF12Energy", "pair_f12_energy", "Pf12Error", "lib"]


class Pf12Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pf12 error {code} ({_lib.ERRORS.get(code, '?')}): {msg}")
        self.code = code


def lib():
    return _lib.load()


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _dev(t, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


TENSOR_NAMES = ("Agi", "Agj", "Afi", "Afj", "Jg", "Jf", "Q", "T")
_C_NAMES = ("Ag_i", "Ag_j", "Af_i", "Af_j", "Jg", "Jf", "Q", "T")


class PairF12:
    """One library context: a pair list, its packed device tensors and workspace.

    precision: "fp64" (plain mode) or "mixed_fp32".  FP64 Cholesky, solves and
    energy sums in both."""

    def __init__(self, precision="fp64", workspace_bytes=0, stream=None, tuner_cache=None,
                 variant=None, sieve_plain=False, debug_wait_timeout=False, augment_somo=False,
                 metric_packed=False):
        """variant: None = autotune, else 0 / 1 (SIMT, 2 / 3 CTAs per SM) or
        2 (tcgen05 tensor-core contractions, mixed precision only).
        augment_somo: SOMO-augmented PNO space (factor blocks (p + n_s) x m with
        the SOMO rows last, Q p x k, T and V (k + n_s) square).
        metric_packed: Jg, Jf given as packed lower triangles (m (m + 1) / 2
        per pair)."""
        self._L = lib()
        self._cache = tuner_cache.encode() if tuner_cache else None
        opts = _lib.Opts(_lib.PRECISION[precision], None, int(workspace_bytes), 1, self._cache,
                         -1 if variant is None else int(variant), int(bool(sieve_plain)),
                         int(bool(debug_wait_timeout)), int(bool(augment_somo)),
                         int(bool(metric_packed)))
        self.augment_somo = bool(augment_somo)
        self.metric_packed = bool(metric_packed)
        h = ctypes.c_void_p()
        self._check(self._L.pf12_create(ctypes.byref(h), ctypes.byref(opts)), None)
        self._h = h
        self.precision = precision
        self._keep = None
        self.n_pairs = 0

    # -------------------------------------------------------------- plumbing
    def _check(self, code, h=0):
        if code != _lib.PF12_OK:
            hh = self._h if h == 0 else h
            msg = self._L.pf12_last_error(hh).decode() if hh else "pf12_create failed"
            raise Pf12Error(code, msg)

    def _stream(self):
        s = torch.cuda.current_stream().cuda_stream
        self._check(self._L.pf12_set_stream(self._h, ctypes.c_void_p(s)))

    def close(self):
        if getattr(self, "_h", None):
            self._L.pf12_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- C ABI calls
    def upload_pairs(self, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, tensors, offsets):
        """tensors: dict of packed float64 CUDA tensors (TENSOR_NAMES);
        offsets: dict with off_pm/off_mm/off_pk/off_kk (int64 arrays)."""
        self._stream()
        kind = np.ascontiguousarray(np.asarray(orb_kind, dtype=np.int8))
        meta = [_i32(pi), _i32(pj), _i32(n_pao), _i32(n_pno), _i32(n_aux)]
        offs = {n: _i64(offsets[n]) for n in ("off_pm", "off_mm", "off_pk", "off_kk")}
        tt = _lib.Tensors()
        for py, c in zip(TENSOR_NAMES, _C_NAMES):
            setattr(tt, c, _dev(tensors[py], py))
        for n in offs:
            setattr(tt, n, _ptr(offs[n], ctypes.c_int64))
        tt.len_pm = tensors["Agi"].numel()
        tt.len_mm = tensors["Jg"].numel()
        tt.len_pk = tensors["Q"].numel()
        tt.len_kk = tensors["T"].numel()
        n = len(meta[0])
        self._check(self._L.pf12_upload_pairs(
            self._h, int(n_orb), _ptr(kind, ctypes.c_int8), n,
            *[_ptr(a, ctypes.c_int32) for a in meta], ctypes.byref(tt)))
        self._keep = (tensors, offs, meta, kind)
        self.n_pairs = n
        self.len_kk = tt.len_kk

    def set_arrival(self, group_end, ready, epoch):
        """Streamed inputs for the next fits (pf12_set_arrival): group_end
        (host int64, strictly increasing, last = n_pairs) splits the pair list
        into groups; ready (CUDA int32/uint32 tensor, one flag per group) is
        set to epoch by the caller's copy stream once a group's inputs are on
        the device.  An empty group_end turns streaming off."""
        ends = _i64(group_end)
        if len(ends) == 0:
            self._check(self._L.pf12_set_arrival(self._h, 0, None, None, 0))
            self._arrival = None
            return
        if not (ready.is_cuda and ready.dtype in (torch.int32, torch.uint32) and ready.is_contiguous()
                and ready.numel() >= len(ends)):
            raise ValueError("ready must be a contiguous int32 CUDA tensor with one flag per group")
        self._check(self._L.pf12_set_arrival(self._h, len(ends), _ptr(ends, ctypes.c_int64),
                                             ctypes.c_void_p(ready.data_ptr()),
                                             int(epoch) & 0xFFFFFFFF))
        self._arrival = (ends, ready)

    def upload_pairs_gather(self, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, blocks, orbitals,
                            maps, tensors, offsets):
        """Gather mode.  blocks: dict Bg, Bf (packed per-orbital float64 CUDA
        tensors); orbitals: dict off_orb, ext_pao, ext_aux, ext_ld (host);
        maps: dict map_pao, map_aux, off_map_pao, off_map_aux (host);
        tensors: Jg, Jf, Q, T (packed, CUDA); offsets: off_mm, off_pk, off_kk."""
        self._stream()
        kind = np.ascontiguousarray(np.asarray(orb_kind, dtype=np.int8))
        meta = [_i32(pi), _i32(pj), _i32(n_pao), _i32(n_pno), _i32(n_aux)]
        orb = {"off_orb": _i64(orbitals["off_orb"]), "ext_pao": _i32(orbitals["ext_pao"]),
               "ext_aux": _i32(orbitals["ext_aux"]), "ext_ld": _i32(orbitals["ext_ld"])}
        mp = {"map_pao": _i32(maps["map_pao"]), "map_aux": _i32(maps["map_aux"]),
              "off_map_pao": _i64(maps["off_map_pao"]), "off_map_aux": _i64(maps["off_map_aux"])}
        offs = {n: _i64(offsets[n]) for n in ("off_mm", "off_pk", "off_kk")}
        g = _lib.GatherTensors()
        g.Bg, g.Bf = _dev(blocks["Bg"], "Bg"), _dev(blocks["Bf"], "Bf")
        g.off_orb = _ptr(orb["off_orb"], ctypes.c_int64)
        for n in ("ext_pao", "ext_aux", "ext_ld"):
            setattr(g, n, _ptr(orb[n], ctypes.c_int32))
        g.len_orb = blocks["Bg"].numel()
        g.map_pao, g.map_aux = _ptr(mp["map_pao"], ctypes.c_int32), _ptr(mp["map_aux"], ctypes.c_int32)
        g.off_map_pao = _ptr(mp["off_map_pao"], ctypes.c_int64)
        g.off_map_aux = _ptr(mp["off_map_aux"], ctypes.c_int64)
        g.len_map_pao, g.len_map_aux = mp["map_pao"].size, mp["map_aux"].size
        for n in ("Jg", "Jf", "Q", "T"):
            setattr(g, n, _dev(tensors[n], n))
        for n in offs:
            setattr(g, n, _ptr(offs[n], ctypes.c_int64))
        g.len_mm, g.len_pk, g.len_kk = (tensors["Jg"].numel(), tensors["Q"].numel(),
                                        tensors["T"].numel())
        n = len(meta[0])
        self._check(self._L.pf12_upload_pairs_gather(
            self._h, int(n_orb), _ptr(kind, ctypes.c_int8), n,
            *[_ptr(a, ctypes.c_int32) for a in meta], ctypes.byref(g)))
        self._keep = (blocks, orb, mp, tensors, offs, meta, kind)
        self.n_pairs = n
        self.len_kk = g.len_kk

    # python names of the full-mode tensors, in the order of _lib.FULL_FACTORS / FULL_OTHERS
    FULL_NAMES = ("Agi", "Agj", "Afi", "Afj", "Ari", "Arj", "AgiF", "AgjF", "AriF", "ArjF",
                  "Jg", "Jf", "Jr", "Q", "T", "Fv", "S", "B")

    def upload_full(self, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, tensors, offsets):
        """Complete pair energy (pf12_upload_full).  tensors: dict of packed
        float64 CUDA tensors named as FULL_NAMES; offsets: off_pm, off_mm,
        off_pk, off_kk, off_pp, off_s, off_b (int64 host arrays)."""
        self._stream()
        kind = np.ascontiguousarray(np.asarray(orb_kind, dtype=np.int8))
        meta = [_i32(pi), _i32(pj), _i32(n_pao), _i32(n_pno), _i32(n_aux)]
        offs = {n: _i64(offsets[n]) for n in _lib.FULL_OFFSETS}
        ft = _lib.FullTensors()
        for py, c in zip(self.FULL_NAMES, _lib.FULL_FACTORS + _lib.FULL_OTHERS):
            setattr(ft, c, _dev(tensors[py], py))
        for n in _lib.FULL_OFFSETS:
            setattr(ft, n, _ptr(offs[n], ctypes.c_int64))
        lens = {"len_pm": "Agi", "len_mm": "Jg", "len_pk": "Q", "len_kk": "T", "len_pp": "Fv",
                "len_s": "S", "len_b": "B"}
        for n, src in lens.items():
            setattr(ft, n, tensors[src].numel())
        n = len(meta[0])
        self._check(self._L.pf12_upload_full(
            self._h, int(n_orb), _ptr(kind, ctypes.c_int8), n,
            *[_ptr(a, ctypes.c_int32) for a in meta], ctypes.byref(ft)))
        self._keep = (tensors, offs, meta, kind)
        self.n_pairs = n
        self.len_kk = tensors["T"].numel()

    def full_terms(self, terms=None):
        """Per-pair spatial terms of the last full-mode fit (n_pairs x 14)."""
        self._stream()
        if terms is None:
            terms = torch.zeros((self.n_pairs, 14), dtype=torch.float64, device="cuda")
        self._check(self._L.pf12_full_terms(self._h, _dev(terms, "terms")))
        return terms

    def backward_gather(self, dE=1.0, grads=None):
        """Gather mode: dE * dE_F12/d{Bg, Bf} (per-orbital blocks), dQ, dT."""
        self._stream()
        g = grads or {}
        args = [_dev(g.get(n), n) for n in ("Bg", "Bf", "Q", "T")]
        self._check(self._L.pf12_backward_gather(self._h, float(dE), *args))
        return g

    def fit(self):
        self._stream()
        self._check(self._L.pf12_fit(self._h))

    def build_v(self, V=None):
        self._stream()
        if V is None:
            V = torch.zeros(self.len_kk, dtype=torch.float64, device="cuda")
        self._check(self._L.pf12_build_v(self._h, _dev(V, "V")))
        return V

    def energy(self, e_pair=None, want_host=True, check=True):
        """Returns (E, e_pair): E a Python float (FP64, fixed-order total)."""
        self._stream()
        if e_pair is None:
            e_pair = torch.empty((self.n_pairs, 3), dtype=torch.float64, device="cuda")
        E = ctypes.c_double(float("nan"))
        code = self._L.pf12_energy(self._h, _dev(e_pair, "e_pair"),
                                   ctypes.byref(E) if want_host else None)
        if check:
            self._check(code)
        return E.value, e_pair

    def backward(self, dE=1.0, grads=None):
        """Writes dE * dE_F12/d{Agi,Agj,Afi,Afj,Q,T} into grads (dict of packed
        float64 CUDA tensors shaped like the inputs; missing keys are skipped)."""
        self._stream()
        g = grads or {}
        args = [_dev(g.get(n), n) for n in ("Agi", "Agj", "Afi", "Afj", "Q", "T")]
        self._check(self._L.pf12_backward(self._h, float(dE), *args))
        return g

    def pair_status(self):
        st = np.zeros(max(self.n_pairs, 1), dtype=np.int32)
        self._check(self._L.pf12_pair_status(self._h, _ptr(st, ctypes.c_int32)))
        return st[:self.n_pairs]

    def stats(self):
        s = _lib.Stats()
        self._check(self._L.pf12_stats(self._h, ctypes.byref(s)))
        out = {n: getattr(s, n) for n, _ in _lib.Stats._fields_}
        out["tune_ms"] = list(s.tune_ms)
        out["ctas_variant"] = list(s.ctas_variant)
        out["tune_bwd_ms"] = list(s.tune_bwd_ms)
        return out


class PairF12Energy(torch.autograd.Function):
    """E_F12 (sum of all pair energies) as a differentiable function of the DF
    factors, PNO coefficients and amplitudes; J_g and J_f are constants.

    forward(ctx, Agi, Agj, Afi, Afj, Jg, Jf, Q, T, meta) with meta a dict of
    n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, off_pm, off_mm, off_pk,
    off_kk and optionally precision, variant and tuner_cache (PairF12's
    options).  backward recomputes V per pair in the
    library's adjoint kernel.

    The library reads the inputs through raw device pointers, so forward saves
    them with save_for_backward: their storage stays alive until backward, and
    autograd raises if one of them is modified in place in between.  The
    engine is released after the first backward; a second backward
    (retain_graph=True) uploads the saved inputs into a new one."""

    @staticmethod
    def _engine(tensors, meta):
        eng = PairF12(meta.get("precision", "fp64"), variant=meta.get("variant"),
                      tuner_cache=meta.get("tuner_cache"))
        eng.upload_pairs(meta["n_orb"], meta["orb_kind"], meta["pi"], meta["pj"], meta["n_pao"],
                         meta["n_pno"], meta["n_aux"], tensors, meta)
        return eng

    @staticmethod
    def forward(ctx, Agi, Agj, Afi, Afj, Jg, Jf, Q, T, meta):
        inputs = (Agi, Agj, Afi, Afj, Jg, Jf, Q, T)
        eng = PairF12Energy._engine(dict(zip(TENSOR_NAMES, inputs)), meta)
        eng.fit()
        E, _ = eng.energy()
        ctx.meta = meta
        if not any(ctx.needs_input_grad[:8]):   # no backward will come: release now
            eng.close()
            ctx.eng = None
        else:
            ctx.save_for_backward(*inputs)
            ctx.eng = eng
        return torch.tensor(E, dtype=torch.float64, device=Agi.device)

    @staticmethod
    def backward(ctx, gE):
        saved = ctx.saved_tensors          # raises if an input was modified in place
        eng = ctx.eng
        if eng is None or getattr(eng, "_h", None) is None:
            eng = PairF12Energy._engine(dict(zip(TENSOR_NAMES, saved)), ctx.meta)
        need = ctx.needs_input_grad
        names = ("Agi", "Agj", "Afi", "Afj", "Q", "T")
        idx = (0, 1, 2, 3, 6, 7)
        grads = {}
        for n, i in zip(names, idx):
            if need[i]:
                grads[n] = torch.zeros_like(saved[i], memory_format=torch.contiguous_format)
        eng.backward(float(gE), grads)
        out = [grads.get(n) for n in names]
        eng.close()
        ctx.eng = None
        return out[0], out[1], out[2], out[3], None, None, out[4], out[5], None


def pair_f12_energy(Agi, Agj, Afi, Afj, Jg, Jf, Q, T, meta):
    return PairF12Energy.apply(Agi, Agj, Afi, Afj, Jg, Jf, Q, T, meta)
