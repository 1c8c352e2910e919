"""Helpers of the GPU tests: upload host-drawn inputs, run the library, unpack."""
import numpy as np
import torch

import synthetic as S
from synthetic import workloads as W


def sized_workload(sizes, kinds=None, name="sized", seed=W.SEED_BASE + 300, diag_every=0):
    """Workload whose pair P has (p, k, m) = sizes[P]; pairs run along a chain
    (P, P+1), with every diag_every-th pair diagonal (P, P)."""
    n = len(sizes)
    n_orb = n + 1
    kind = np.zeros(n_orb, np.int8) if kinds is None else np.asarray(kinds, np.int8)
    pi = np.arange(n, dtype=np.int32)
    pj = pi + 1
    if diag_every:
        pj[::diag_every] = pi[::diag_every]
    p = np.array([s[0] for s in sizes], np.int32)
    k = np.array([s[1] for s in sizes], np.int32)
    m = np.array([s[2] for s in sizes], np.int32)
    decay = np.array([W._decay_power(j - i) for i, j in zip(pi, pj)])
    return W.Workload(name, seed, int((kind == 0).sum()), int((kind == 1).sum()), kind, pi, pj,
                      p, k, m, decay)


def upload_host(wl, host=None):
    """Host-drawn packed inputs copied to the device."""
    buf, lay = host if host is not None else S.packed_inputs(wl)
    t = {n: torch.from_numpy(np.concatenate([v, np.zeros(2)]) if v.size < 2 else v).cuda()
         for n, v in buf.items()}
    return t, lay


def run(wl, precision="fp64", t=None, lay=None, want_V=True, want_grad=False, dE=1.0,
        variant=None):
    import paper_2008_03237_gb300 as pf
    if t is None:
        t, lay = upload_host(wl)
    eng = pf.PairF12(precision, variant=variant)
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    E, e_pair = eng.energy()
    out = {"E": E, "e_pair": e_pair.cpu().numpy(), "eng": eng, "t": t, "lay": lay}
    if want_V:
        V = eng.build_v()
        out["V"] = [S.unpack(V.cpu().numpy(), lay["off_kk"], P, int(wl.n_pno[P]), int(wl.n_pno[P]))
                    for P in range(wl.n_pairs)]
    if want_grad:
        g = {n: torch.zeros_like(t[n]) for n in ("Agi", "Agj", "Afi", "Afj", "Q", "T")}
        eng.backward(dE, g)
        out["grads"] = {n: v.cpu().numpy() for n, v in g.items()}
    torch.cuda.synchronize()
    return out


def grad_blocks(wl, lay, g, P):
    p, k, m = int(wl.n_pao[P]), int(wl.n_pno[P]), int(wl.n_aux[P])
    out = {}
    for n in ("Agi", "Agj", "Afi", "Afj"):
        out[n] = S.unpack(g[n], lay["off_pm"], P, p, m)
    out["Q"] = S.unpack(g["Q"], lay["off_pk"], P, p, k)
    out["T"] = S.unpack(g["T"], lay["off_kk"], P, k, k)
    return out


def normalised_error(dE, sum_abs, n_orb):
    """|dE| on the chemical scale (reading G1): energies rescaled so that
    sum_P |e_P| = 4.8 mEh per orbital."""
    return abs(dE) * 4.8e-3 * n_orb / sum_abs
