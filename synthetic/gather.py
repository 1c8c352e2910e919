"""Gather-mode synthetic workloads: per-orbital pair-extended DF blocks and the
per-pair index maps that sieve each pair's blocks out of them.

Stands in for the paper's pair-extended SparseMaps (Sec. "F12 integral
transformations"): the domain of orbital i is augmented with the domains of all
j it forms an F12 pair with, the three-index factors (i mu~|K|X) exist once per
orbital on that extended domain, and every pair takes the rows of its own PAO
domain and the columns of its own auxiliary domain from the blocks of i and j.

Domains are atom-complete (Sec. "Orbital domains"): whole atoms, each atom
contributing S_PAO PAOs and S_AUX auxiliary functions.  Orbital o sits at atom
2 o of a chain; its own PAO / aux domain is the window of atoms within a drawn
half-width; a pair's domain is the union of its two orbitals' windows; an
orbital's extended domain is the union of the domains of its pairs.

Values: entry (mu, X) of orbital o's block for kernel g or f is the Irwin-Hall
Gaussian of Philox counter (global aux function X, global PAO function mu,
o, tensor id), so a pair's sieved block is a function of global indices alone
and the oracle can draw it without the block storage.  J, Q and T are the
packed-mode draws of workloads.py for the pair's (p, k, m).
"""
from dataclasses import dataclass

import numpy as np

from . import workloads as W
from .philox import philox4x32

S_PAO = 10      # PAOs per atom (even: 16-byte aligned atom runs)
S_AUX = 40      # auxiliary functions per atom
TID_BG, TID_BF = 20, 21


@dataclass
class GatherWorkload:
    base: W.Workload                 # pair list, kinds, k per pair; its p, m are overwritten
    pao_atoms: list                  # per pair: sorted PAO atoms
    aux_atoms: list                  # per pair: sorted aux atoms
    ext_pao_atoms: list              # per orbital
    ext_aux_atoms: list              # per orbital

    @property
    def n_orb(self):
        return self.base.n_orb

    @property
    def n_pairs(self):
        return self.base.n_pairs


def _windows(seed, n_orb, lo, hi, tid):
    w = philox4x32(np.arange(n_orb), 0, 0, tid, seed, W.KEY_HI)[0]
    return np.array([W._uniform_int(x, lo, hi) for x in w], np.int64)


def make_gather(base, pao_halfwidth=(2, 5), aux_halfwidth=(3, 6)):
    """Atom-complete domains on the chain of base's orbitals; p, m of base are
    replaced by the domain sizes (k clipped to p)."""
    n_orb = base.n_orb
    hw_p = _windows(base.seed, n_orb, *pao_halfwidth, 40)
    hw_a = _windows(base.seed, n_orb, *aux_halfwidth, 41)
    n_atoms = 2 * n_orb + 2 * max(pao_halfwidth[1], aux_halfwidth[1]) + 2
    off = max(pao_halfwidth[1], aux_halfwidth[1]) + 1

    def dom(o, hw):
        c = 2 * o + off
        return set(range(max(0, c - hw[o]), min(n_atoms, c + hw[o] + 1)))
    pao, aux = [], []
    for i, j in zip(base.pi, base.pj):
        pao.append(sorted(dom(i, hw_p) | dom(j, hw_p)))
        aux.append(sorted(dom(i, hw_a) | dom(j, hw_a)))
    ext_p = [set() for _ in range(n_orb)]
    ext_a = [set() for _ in range(n_orb)]
    for P, (i, j) in enumerate(zip(base.pi, base.pj)):
        for o in (i, j):
            ext_p[o].update(pao[P])
            ext_a[o].update(aux[P])
    wl = W.Workload(base.name + "[gather]", base.seed, base.n_domo, base.n_somo, base.orb_kind,
                    base.pi, base.pj, base.n_pao.copy(), base.n_pno.copy(), base.n_aux.copy(),
                    np.ones(base.n_pairs), base.metric_shift, dict(base.meta))
    wl.n_pao[:] = [S_PAO * len(a) for a in pao]
    wl.n_aux[:] = [S_AUX * len(a) for a in aux]
    wl.n_pno[:] = np.minimum(wl.n_pno, wl.n_pao)
    return GatherWorkload(wl, pao, aux, [sorted(s) for s in ext_p], [sorted(s) for s in ext_a])


def _functions(atoms, per):
    return (np.repeat(np.asarray(atoms, np.int64) * per, per) +
            np.tile(np.arange(per, dtype=np.int64), len(atoms)))


def _values(seed, o, tid, mu_glob, x_glob):
    """Block entries for global PAO functions mu_glob (rows) x aux functions x_glob."""
    mu = np.asarray(mu_glob, np.int64)[:, None]
    x = np.asarray(x_glob, np.int64)[None, :]
    w = philox4x32(x, mu, o, tid, seed, W.KEY_HI)
    return W._ih16(w[0], w[1]).astype(np.float64) * W.IH16_INV_STD


def orbital_layout(gw):
    """Per-orbital block sizes P_o, M_o, leading dimensions (even) and offsets."""
    P = np.array([S_PAO * len(a) for a in gw.ext_pao_atoms], np.int32)
    M = np.array([S_AUX * len(a) for a in gw.ext_aux_atoms], np.int32)
    ld = (M + 1) // 2 * 2
    sz = (P.astype(np.int64) * ld + W.ALIGN - 1) // W.ALIGN * W.ALIGN
    off = np.zeros(len(P), np.int64)
    if len(P) > 1:
        off[1:] = np.cumsum(sz)[:-1]
    return P, M, ld.astype(np.int32), off, int(sz.sum())


def orbital_blocks(gw):
    """Host arrays Bg, Bf (packed per-orbital blocks) and the orbital layout."""
    P, M, ld, off, total = orbital_layout(gw)
    seed = gw.base.seed
    out = {}
    for name, tid in (("Bg", TID_BG), ("Bf", TID_BF)):
        buf = np.zeros(max(total, 2))
        for o in range(gw.n_orb):
            if P[o] == 0:
                continue
            vals = _values(seed, o, tid, _functions(gw.ext_pao_atoms[o], S_PAO),
                           _functions(gw.ext_aux_atoms[o], S_AUX))
            blk = np.zeros((P[o], ld[o]))
            blk[:, :M[o]] = vals
            buf[off[o]:off[o] + blk.size] = blk.ravel()
        out[name] = buf
    return out, (P, M, ld, off, total)


def pair_maps(gw):
    """Per pair: rows of the pair's PAOs in ext(i) then in ext(j) (2p entries)
    and columns of its aux functions in ext_aux(i) then ext_aux(j) (2m)."""
    mp, ma, op, oa = [], [], [0], [0]
    for P, (i, j) in enumerate(zip(gw.base.pi, gw.base.pj)):
        fp = _functions(gw.pao_atoms[P], S_PAO)
        fa = _functions(gw.aux_atoms[P], S_AUX)
        for o in (i, j):
            mp.append(np.searchsorted(_functions(gw.ext_pao_atoms[o], S_PAO), fp))
            ma.append(np.searchsorted(_functions(gw.ext_aux_atoms[o], S_AUX), fa))
        op.append(op[-1] + 2 * len(fp))
        oa.append(oa[-1] + 2 * len(fa))
    return (np.concatenate(mp).astype(np.int32) if mp else np.zeros(0, np.int32),
            np.concatenate(ma).astype(np.int32) if ma else np.zeros(0, np.int32),
            np.array(op[:-1], np.int64), np.array(oa[:-1], np.int64))


def pair_inputs(gw, P):
    """Oracle view of pair P: its sieved factors drawn from global indices, plus
    the packed-mode J, Q, T of the pair's (p, k, m)."""
    wl = gw.base
    i, j = int(wl.pi[P]), int(wl.pj[P])
    fp = _functions(gw.pao_atoms[P], S_PAO)
    fa = _functions(gw.aux_atoms[P], S_AUX)
    t = W.pair_inputs(wl, P)
    t["Agi"] = _values(wl.seed, i, TID_BG, fp, fa)
    t["Agj"] = _values(wl.seed, j, TID_BG, fp, fa)
    t["Afi"] = _values(wl.seed, i, TID_BF, fp, fa)
    t["Afj"] = _values(wl.seed, j, TID_BF, fp, fa)
    return t
