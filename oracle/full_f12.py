"""FP64 CPU oracle of the complete pair-specific F12 energy E_(2)F12
(Kumar, Neese, Valeev, arXiv 2008.03237, Sec. "The PNO-based
CCSD(T)F12bar Method").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  The CUDA path
shares no code with it.

Per pair P = (i, j), plain numpy/LAPACK steps in the paper's order:

  1. local density fitting with the pair's Coulomb metric (Sec. "F12 integral
     transformations"), for the densities of i and j with every function of
     the pair's orbital basis (the PAOs and the occupied i, j) and of the
     Fock-transformed occupied orbitals i_F, j_F (Eq. XAppr):
         C_x = A^g_x J_g^{-1}
  2. robust (Dunlap) fits of the two pair kernels, same coefficients:
         K_V  = A^f_i C_j^T + C_i A^f_j^T - C_i J_f C_j^T   (V kernel, Eq. V)
         K_R  = A^r_i C_j^T + C_i A^r_j^T - C_i J_r C_j^T   (geminal R)
         K_RjF, K_RiF: K_R with j (i) replaced by j_F (i_F)
  3. the Q_ij projector (Eq. Qij) removes the PNO x PNO block of the geminal:
         R_pno = Q^T K_R Q,   R_Q = K_R - Q R_pno Q^T
     and from V the part that passes through PNO pairs:
         Vh[p, q] = (Q_x^T K_V Q_x)[p, q] - sum_cd R_pno[c, d] (c p|d q)
     with Q_x = blockdiag(Q, I_2) (PNOs, then i, then j) and (c p|d q) from
     the PNO-pair factors.
  4. Vtilde (Eq. Vtilde), spatial direct and exchange forms:
         Vt_d = 1/2 (Vh[i, j] + <Vh, T> + Vh[i, s_j] + Vh[s_i, j]) + <C, T>
         Vt_x = 1/2 (Vh[j, i] + <Vh, T^T> + Vh[j, s_i] + Vh[s_j, i]) + <C, T^T>
     with C = Ft^T K_R Q + Q^T K_R Ft (Eq. C), Ft = (1 - Q Q^T) F_v Q the
     Fock coupling of the PNOs to the rest of the virtual space.
  5. B~ (Eqs. B, X, Btilde, XAppr):
         B_dd = tr(R_Q F_v R_Q^T) + tr(R_Q^T F_v R_Q),  B_dx = 2 tr(R_Q F_v R_Q)
         X_dd(jF) = <K_RjF, R_Q>, X_dx(jF) = <K_RjF, R_Q^T>, the same for iF
         B~_dd = B_dd - X_dd(jF) - X_dd(iF),  B~_dx = B_dx - X_dx(jF) - X_dx(iF)
  6. spin adaptation (Eqs. F12energy_sf*, the ROHF occupation rules):
         e_ab = n_ab (3/4 Vt_d + 1/4 Vt_x + (10 B~_dd + 6 B~_dx) / 64)
         e_aa = n_aa (1/2 (Vt_d - Vt_x) + (B~_dd - B~_dx) / 16),  e_bb likewise

Readings of the paper that these steps fix (the paper gives canonical
spin-orbital equations and describes the pair-local evaluation in prose):
the pair's PAO domain, treated as orthonormal, stands in for the complete
virtual space (OBS virtuals + CABS) of the sums in Eqs. C, B, X; V^{ij}_{pq}
(spin-free) = 1/2 Vh[p, q] with the 1/2 of Eq. V, while C, B and X carry the
geminal without it; the singles amplitudes enter through their projection
onto the pair's PNOs; the spatial direct/exchange combinations and the
prefactors follow from the spin-orbital sums with the SP-ansatz projectors,
which tests/spin_orbital_bruteforce_full.py enumerates explicitly.
"""
import numpy as np

from .pairf12 import local_fit, robust_kernel, spin_multiplicities

TERM_NAMES = ("vocc_d", "vocc_x", "d", "x", "s_d", "s_x", "c_d", "c_x",
              "b_dd", "b_dx", "xj_dd", "xj_dx", "xi_dd", "xi_dx")


# ---------------------------------------------------------------- steps 1-2


def fits(t):
    """Steps 1-2: the four robust-fit kernels of the pair.  K_V over the p + 2
    rows (PAOs, i, j); K_R, K_RjF, K_RiF over the p PAOs."""
    p = t["Q"].shape[0]
    C_i, C_j = local_fit(t["Agi"], t["Agj"], t["Jg"])
    C_iF, C_jF = local_fit(t["AgiF"][:p], t["AgjF"][:p], t["Jg"])
    K_V = robust_kernel(t["Afi"], t["Afj"], C_i, C_j, t["Jf"])
    Ci, Cj = C_i[:p], C_j[:p]
    K_R = robust_kernel(t["Ari"][:p], t["Arj"][:p], Ci, Cj, t["Jr"])
    K_RjF = robust_kernel(t["Ari"][:p], t["ArjF"][:p], Ci, C_jF, t["Jr"])
    K_RiF = robust_kernel(t["AriF"][:p], t["Arj"][:p], C_iF, Cj, t["Jr"])
    return {"K_V": K_V, "K_R": K_R, "K_RjF": K_RjF, "K_RiF": K_RiF}


# ---------------------------------------------------------------- step 3


def extended_pnos(Q):
    """Q_x = blockdiag(Q, I_2): the pair's orbital basis as PNOs, then i, then j."""
    p, k = Q.shape
    Qx = np.zeros((p + 2, k + 2))
    Qx[:p, :k] = Q
    Qx[p:, k:] = np.eye(2)
    return Qx


def projector_term(R_pno, B):
    """sum_cd R_pno[c, d] (c p|d q), (c p|d q) = sum_X B[c, X, p] B[d, X, q]."""
    return np.einsum("cd,cXp,dXq->pq", R_pno, B, B)


def projected(K, t):
    """Step 3: R_pno, R_Q and the projected V kernel Vh over the extended basis."""
    Q = t["Q"]
    R_pno = Q.T @ K["K_R"] @ Q
    R_Q = K["K_R"] - Q @ R_pno @ Q.T
    Qx = extended_pnos(Q)
    Vh = Qx.T @ K["K_V"] @ Qx - projector_term(R_pno, t["B"])
    return R_pno, R_Q, Vh


# ---------------------------------------------------------------- steps 4-5


def fock_coupling(Fv, Q):
    """Ft = (1 - Q Q^T) F_v Q: the Fock coupling of the PNOs to the rest of
    the pair's virtual space (the alpha sum of Eq. C with the PNO part removed
    by the projector of R)."""
    FQ = Fv @ Q
    return FQ - Q @ (Q.T @ FQ)


def pair_terms(t):
    """Every spatial term of the pair (TERM_NAMES) after steps 1-5."""
    Q, T, S = t["Q"], t["T"], t["S"]
    k = Q.shape[1]
    K = fits(t)
    R_pno, R_Q, Vh = projected(K, t)
    io, jo = k, k + 1
    V = Vh[:k, :k]
    si, sj = S[0], S[1]
    Ft = fock_coupling(t["Fv"], Q)
    Cm = Ft.T @ K["K_R"] @ Q + Q.T @ K["K_R"] @ Ft
    Fv = t["Fv"]
    out = {
        "vocc_d": Vh[io, jo], "vocc_x": Vh[jo, io],
        "d": float(np.sum(V * T)), "x": float(np.sum(V * T.T)),
        "s_d": float(Vh[io, :k] @ sj + si @ Vh[:k, jo]),
        "s_x": float(Vh[jo, :k] @ si + sj @ Vh[:k, io]),
        "c_d": float(np.sum(Cm * T)), "c_x": float(np.sum(Cm * T.T)),
        "b_dd": float(np.trace(R_Q @ Fv @ R_Q.T) + np.trace(R_Q.T @ Fv @ R_Q)),
        "b_dx": float(2.0 * np.trace(R_Q @ Fv @ R_Q)),
        "xj_dd": float(np.sum(K["K_RjF"] * R_Q)), "xj_dx": float(np.sum(K["K_RjF"] * R_Q.T)),
        "xi_dd": float(np.sum(K["K_RiF"] * R_Q)), "xi_dx": float(np.sum(K["K_RiF"] * R_Q.T)),
    }
    return {n: float(out[n]) for n in TERM_NAMES}, {"K": K, "R_Q": R_Q, "Vh": Vh, "C": Cm}


def vtilde(tm):
    """Spatial direct and exchange Vtilde of Eq. Vtilde."""
    vd = 0.5 * (tm["vocc_d"] + tm["d"] + tm["s_d"]) + tm["c_d"]
    vx = 0.5 * (tm["vocc_x"] + tm["x"] + tm["s_x"]) + tm["c_x"]
    return vd, vx


def btilde(tm):
    """Spatial B~ of Eqs. Btilde and XAppr: (B~_dd, B~_dx)."""
    return (tm["b_dd"] - tm["xj_dd"] - tm["xi_dd"], tm["b_dx"] - tm["xj_dx"] - tm["xi_dx"])


# ---------------------------------------------------------------- step 6


def spin_case_energies(tm, mult):
    """(e_ab, e_aa, e_bb) of the pair (Eqs. F12energy_sf*)."""
    n_ab, n_aa, n_bb = mult
    vd, vx = vtilde(tm)
    bd, bx = btilde(tm)
    e_os = 0.75 * vd + 0.25 * vx + (10.0 * bd + 6.0 * bx) / 64.0
    e_ss = 0.5 * (vd - vx) + (bd - bx) / 16.0
    return (n_ab * e_os, n_aa * e_ss, n_bb * e_ss)


def run(wl, pairs=None, inputs=None, want_terms=True):
    """Evaluate pairs of workload wl (all when pairs is None) in full.
    inputs: optional callable P -> tensors (default: synthetic.full inputs).
    Returns e_pair (n x 3), terms (n x len(TERM_NAMES)), E (pair-order sum)."""
    from synthetic.full import full_pair_inputs, orbital_energies
    eps = orbital_energies(wl)
    get = inputs or (lambda P: full_pair_inputs(wl, P, eps))
    idx = list(range(wl.n_pairs) if pairs is None else pairs)
    e_pair = np.zeros((len(idx), 3))
    terms = np.zeros((len(idx), len(TERM_NAMES)))
    for n, P in enumerate(idx):
        t = get(P)
        i, j = int(wl.pi[P]), int(wl.pj[P])
        tm, _ = pair_terms(t)
        mult = spin_multiplicities(int(wl.orb_kind[i]), int(wl.orb_kind[j]), i == j)
        e_pair[n] = spin_case_energies(tm, mult)
        terms[n] = [tm[x] for x in TERM_NAMES]
    E = 0.0
    for n in range(len(idx)):
        E += e_pair[n, 0] + e_pair[n, 1] + e_pair[n, 2]
    return {"pairs": idx, "e_pair": e_pair, "terms": terms, "E": E,
            "sum_abs": float(np.abs(e_pair.sum(axis=1)).sum())}
