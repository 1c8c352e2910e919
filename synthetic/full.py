"""Seeded synthetic inputs of the complete pair-specific F12 energy: the terms of
E_(2)F12 beyond the amplitude term, i.e. the occupied block and singles of
Eq. Vtilde, the Fock coupling of Eq. C, the B~ / X intermediates with the
Fock-transformed occupied orbitals of Eqs. B, X, XAppr, and the PNO-projector
term of Eq. Qij.  Nothing here computes any part of the method; it only draws
inputs (bit-identical on the host here and on the device in csrc/synth_gen.cu).

Per pair P = (i, j), on top of the pair's PAO domain (p), auxiliary domain (m)
and PNOs (k):

* factor blocks of p + 2 rows: the p PAO rows, then the occupied orbitals i
  and j as bra functions of the pair's orbital basis (rows p, p + 1).
    Agi, Agj  Coulomb 3-index factors (i q|X), (j q|X)       rows p, p+1 used
    Afi, Afj  factors of the V kernel                         rows p, p+1 used
    Ari, Arj  factors of the geminal f12 (the R kernel)       PAO rows only
    AgiF, AgjF, AriF, ArjF  the same for the Fock-transformed occupied orbitals
              i_F, j_F (Eq. XAppr)                            PAO rows only
  (rows a block does not use are zero).  The occupied rows are consistent
  between the two sides: row p + 1 of the i blocks and row p of the j blocks
  are the same (ij|X).
* Jg, Jf, Jr: SPD auxiliary metrics of the three operators (Jr and the
  geminal factors carry the geminal's scale R_SCALE, a power of two).
* Q (p x k), T (k x k): as in the amplitude-term workloads.
* Fv (p x p, symmetric): the Fock matrix over the pair's PAO domain, which
  stands in for the complete virtual space (positive diagonal, weak coupling).
* S (2 x k): singles amplitudes of i and of j in the pair's PNO basis.
* B (k x m x (k + 2)): the PNO-pair factors (c q|X) of Eq. Qij, already
  contracted with the inverse square root of the Coulomb metric, for PNOs c
  and q in the PNOs, then i, then j; symmetric in (c, q) over the PNOs.

The Fock-transformed blocks are drawn as A_xF = fl(fl(eps_x A_x) + N) with
eps_x < 0 the orbital's diagonal occupied Fock element and N a weak Gaussian
(the couplings to the other occupied orbitals).  With canonical=True the
couplings vanish (N = 0, Fv = 1.5 I), the closed-shell canonical limit in
which B~ reduces to (2 f_v - eps_i - eps_j) X.
"""
import numpy as np

from . import workloads as W
from .philox import philox4x32

# Philox counter word c3 of the additional tensors
(TID_OCCG_II, TID_OCCG_JJ, TID_OCCG_IJ, TID_OCCF_II, TID_OCCF_JJ, TID_OCCF_IJ,
 TID_ARI, TID_ARJ, TID_XR, TID_NGIF, TID_NGJF, TID_NRIF, TID_NRJF,
 TID_FV, TID_S_I, TID_S_J, TID_B, TID_B_I, TID_B_J, TID_EPS) = range(9, 29)

R_SCALE = 2.0 ** -12   # geminal operator scale: its factors and its metric (exact power of 2)
OCC_SCALE = 0.25       # occupied rows (ii|X), (jj|X), (ij|X) relative to the PAO rows
FOCK_NOISE = 0.0625    # couplings of i_F to the other occupied orbitals
FV_OFFDIAG = 0.03125   # off-diagonal virtual Fock couplings
SINGLES_STD = 5e-3
B_SCALE = 0.0625
FV_CANONICAL = 1.5


def _unit20(w):
    """(w mod 2^20) 2^-20: an exact double in [0, 1)."""
    return float(int(w) & 0xFFFFF) * (2.0 ** -20)


def orbital_energies(wl):
    """Diagonal occupied Fock elements eps_o = -(u 2^-20) - 0.4, u a 20-bit uniform."""
    n = wl.n_orb
    w = philox4x32(np.arange(n, dtype=np.int64), 0, 0xFFFFFFFF, TID_EPS, wl.seed, W.KEY_HI)
    return np.array([-_unit20(w[0][o]) - 0.4 for o in range(n)], np.float64)


def canonical(wl):
    return bool(wl.meta.get("canonical", False))


def full_offsets(wl):
    """Element offsets and buffer lengths of the full-energy packed layout:
    off_pm ((p + 2) x m factor blocks), off_mm (m x m), off_pk (p x k),
    off_kk (k x k), off_pp (p x p), off_s (2 x k), off_b (k x m x (k + 2))."""
    p = wl.n_pao.astype(np.int64)
    k = wl.n_pno.astype(np.int64)
    m = wl.n_aux.astype(np.int64)
    sizes = {"pm": (p + 2) * m, "mm": m * m, "pk": p * k, "kk": k * k, "pp": p * p,
             "s": 2 * k, "b": k * m * (k + 2)}
    out = {}
    for name, sz in sizes.items():
        padded = (sz + W.ALIGN - 1) // W.ALIGN * W.ALIGN
        off = np.zeros(len(sz), np.int64)
        if len(sz) > 1:
            off[1:] = np.cumsum(padded)[:-1]
        out["off_" + name] = off
        out["len_" + name] = int(padded.sum()) if len(sz) else 0
    return out


FACTOR_NAMES = ("Agi", "Agj", "Afi", "Afj", "Ari", "Arj", "AgiF", "AgjF", "AriF", "ArjF")
METRIC_NAMES = ("Jg", "Jf", "Jr")


def full_pair_inputs(wl, P, eps=None):
    """Host tensors of pair P for the full energy (see the module docstring)."""
    key = wl.pair_key(P)
    i, j = int(wl.pi[P]), int(wl.pj[P])
    p, k, m = int(wl.n_pao[P]), int(wl.n_pno[P]), int(wl.n_aux[P])
    diag = i == j
    canon = canonical(wl)
    eps = orbital_energies(wl) if eps is None else eps
    base = W.pair_inputs(wl, P)      # PAO rows of Ag/Af, Jg, Jf, Q, T (unchanged streams)
    c = W.factor_scale(wl.decay[P])
    out = {}

    co = c * OCC_SCALE

    def occ_rows(tii, tjj, tij):
        ii = W._gauss16(wl.seed, key, tii, m, co)
        if diag:
            return ii, ii, ii
        return ii, W._gauss16(wl.seed, key, tjj, m, co), W._gauss16(wl.seed, key, tij, m, co)

    for x, tids in (("g", (TID_OCCG_II, TID_OCCG_JJ, TID_OCCG_IJ)),
                    ("f", (TID_OCCF_II, TID_OCCF_JJ, TID_OCCF_IJ))):
        ii, jj, ij = occ_rows(*tids)
        Ai = np.zeros((p + 2, m))
        Aj = np.zeros((p + 2, m))
        Ai[:p] = base["A%si" % x]
        Aj[:p] = base["A%sj" % x]
        Ai[p], Ai[p + 1] = ii, ij
        Aj[p], Aj[p + 1] = ij, jj
        out["A%si" % x], out["A%sj" % x] = Ai, Aj
    cr = c * R_SCALE
    Ari = W._gauss16(wl.seed, key, TID_ARI, p * m, cr).reshape(p, m)
    Arj = Ari.copy() if diag else W._gauss16(wl.seed, key, TID_ARJ, p * m, cr).reshape(p, m)
    for n, A in (("Ari", Ari), ("Arj", Arj)):
        out[n] = np.zeros((p + 2, m))
        out[n][:p] = A
    # Fock-transformed occupied orbitals: fl(fl(eps A) + N), N = 0 when canonical
    src = {"AgiF": (base["Agi"], i, TID_NGIF, c), "AgjF": (base["Agj"], j, TID_NGJF, c),
           "AriF": (Ari, i, TID_NRIF, cr), "ArjF": (Arj, j, TID_NRJF, cr)}
    if diag:
        src["AgjF"] = (base["Agj"], j, TID_NGIF, c)
        src["ArjF"] = (Arj, j, TID_NRIF, cr)
    for n, (A, o, tid, sc) in src.items():
        N = (np.zeros(p * m) if canon else W._gauss16(wl.seed, key, tid, p * m, sc * FOCK_NOISE))
        out[n] = np.zeros((p + 2, m))
        out[n][:p] = (eps[o] * A.ravel() + N).reshape(p, m)
    out["Jg"], out["Jf"] = base["Jg"], base["Jf"]
    out["Jr"] = R_SCALE * W.metric_from_int(W._ih4_matrix(wl.seed, key, TID_XR, m), m,
                                            wl.metric_shift)
    out["Q"], out["T"] = base["Q"], base["T"]
    out["Fv"] = fock_virtual(wl, P)
    out["S"] = singles(wl, P)
    out["B"] = pno_pair_factors(wl, P)
    return out


def fock_virtual(wl, P):
    """p x p symmetric: diagonal 0.5 + 2.5 u (u a 20-bit uniform), off-diagonal
    Gaussian x 2^-5 drawn for r < c and mirrored; 1.5 I when canonical."""
    p = int(wl.n_pao[P])
    if canonical(wl):
        return FV_CANONICAL * np.eye(p)
    key = wl.pair_key(P)
    g = W._gauss16(wl.seed, key, TID_FV, p * p, W.IH16_INV_STD * FV_OFFDIAG).reshape(p, p)
    F = np.triu(g, 1)
    F = F + F.T
    w = philox4x32(np.arange(p, dtype=np.int64), 1, key, TID_FV, wl.seed, W.KEY_HI)
    for r in range(p):
        F[r, r] = 0.5 + 2.5 * _unit20(w[0][r])
    return F


def singles(wl, P):
    """2 x k: singles amplitudes of i (row 0) and j (row 1) in the pair's PNO basis."""
    key = wl.pair_key(P)
    k = int(wl.n_pno[P])
    cs = W.IH16_INV_STD * SINGLES_STD
    si = W._gauss16(wl.seed, key, TID_S_I, k, cs)
    sj = si.copy() if wl.pi[P] == wl.pj[P] else W._gauss16(wl.seed, key, TID_S_J, k, cs)
    return np.stack([si, sj])


def pno_pair_factors(wl, P):
    """k x m x (k + 2): element (c, X, q) for q < k drawn at counter
    (min(c, q) m + X)(k + 2) + max(c, q) (symmetric in c, q); the columns
    q = k (i) and q = k + 1 (j) from their own streams at counter c m + X (the
    same stream for both on a diagonal pair)."""
    key = wl.pair_key(P)
    k, m = int(wl.n_pno[P]), int(wl.n_aux[P])
    cb = W.IH16_INV_STD * B_SCALE
    flat = W._gauss16(wl.seed, key, TID_B, k * m * (k + 2), cb).reshape(k, m, k + 2)
    out = np.empty((k, m, k + 2))
    for c in range(k):
        for q in range(k):
            lo, hi = min(c, q), max(c, q)
            out[c, :, q] = flat[lo, :, hi]
    bi = W._gauss16(wl.seed, key, TID_B_I, k * m, cb).reshape(k, m)
    bj = bi if wl.pi[P] == wl.pj[P] else W._gauss16(wl.seed, key, TID_B_J, k * m, cb).reshape(k, m)
    out[:, :, k] = bi
    out[:, :, k + 1] = bj
    return out


def full_packed_inputs(wl):
    """Host packed buffers of every pair (full energy), plus the offsets."""
    lay = full_offsets(wl)
    eps = orbital_energies(wl)
    buf = {n: np.zeros(max(lay["len_pm"], 2)) for n in FACTOR_NAMES}
    for n in METRIC_NAMES:
        buf[n] = np.zeros(max(lay["len_mm"], 2))
    for n, key in (("Q", "pk"), ("T", "kk"), ("Fv", "pp"), ("S", "s"), ("B", "b")):
        buf[n] = np.zeros(max(lay["len_" + key], 2))
    where = {**{n: "pm" for n in FACTOR_NAMES}, **{n: "mm" for n in METRIC_NAMES},
             "Q": "pk", "T": "kk", "Fv": "pp", "S": "s", "B": "b"}
    for P in range(wl.n_pairs):
        t = full_pair_inputs(wl, P, eps)
        for n, key in where.items():
            o = lay["off_" + key][P]
            v = t[n].ravel()
            buf[n][o:o + v.size] = v
    return buf, lay
