"""Brute-force spin-orbital evaluation of the complete F12 pair energy for tiny
inputs: Eq. F12 energy with Vtilde (Eq. Vtilde: occupied block, amplitude,
C and singles terms), Eqs. V, C, B, X, Btilde and the decoupled Fock term of
Eq. XAppr, and the PNO projector of Eq. Qij.

Independent of oracle/: the spatial kernels are built with a Gauss-Jordan
inverse of J_g and explicit einsum contractions, the Q_ij projector is applied
as an explicit (p^2 x p^2) operator, the PNO-projector correction is summed
over PNO pairs (c, d) with the two-electron integrals written out, and every
spin-orbital quantity is formed and antisymmetrised explicitly over the
complete virtual spin orbitals (the pair's PAO domain, both spins), the PNO
spin orbitals and the occupied spin orbitals of the ROHF determinant.  It then
sums, for every pair P < R of occupied spin orbitals on the pair's orbitals,

    2 Vt^{PR}_{PR} + B~^{PR}_{PR}
    Vt^{PR}_{PR} = V^{PR}_{PR} + 1/2 (V + C)^{PR}_{AB} t^{AB}_{PR}
                   + V^{PR}_{PA} t^A_R + V^{PR}_{AR} t^A_P
    V^{PR}_{XY}  = 1/2 Vbar (the kernel with the SP spin projector, antisymmetrised)
    C^{PR}_{AB}  = F_{A G} Rbar^{PR}_{G B} + F_{B G} Rbar^{PR}_{A G}
    B~^{PR}_{PR} = Rbar_{XY} F_{Y G} Rbar_{X G} - X^{P R_F} - X^{P_F R}
    X^{P R_F}    = 1/2 Rbar^{P R_F}_{XY} Rbar^{PR}_{XY}

with unrestricted sums over the spin-orbital indices A, B (PNOs), G, X, Y
(complete virtual space).
"""
import numpy as np

from spin_orbital_bruteforce import ALPHA, BETA, gauss_jordan_inverse, spin_projector_weights


def _robust(Ao_i, Ao_j, Jinv, Ag_i, Ag_j, Jo):
    Ci = np.einsum("uX,XY->uY", Ag_i, Jinv)
    Cj = np.einsum("uX,XY->uY", Ag_j, Jinv)
    return (np.einsum("uX,vX->uv", Ao_i, Cj) + np.einsum("uX,vX->uv", Ci, Ao_j)
            - np.einsum("uX,XY,vY->uv", Ci, Jo, Cj))


def spatial_full_kernels(t):
    """Spatial kernels of one pair from its full-energy inputs (explicit loops
    and einsum): Vh over PNOs + (i, j), R_Q, and the two Fock-transformed
    geminal kernels (PAO x PAO), for electron 1 on the pair's first orbital."""
    p, k = t["Q"].shape
    Jinv = gauss_jordan_inverse(t["Jg"])
    K_V = _robust(t["Afi"], t["Afj"], Jinv, t["Agi"], t["Agj"], t["Jf"])
    K_R = _robust(t["Ari"][:p], t["Arj"][:p], Jinv, t["Agi"][:p], t["Agj"][:p], t["Jr"])
    K_jF = _robust(t["Ari"][:p], t["ArjF"][:p], Jinv, t["Agi"][:p], t["AgjF"][:p], t["Jr"])
    K_iF = _robust(t["AriF"][:p], t["Arj"][:p], Jinv, t["AgiF"][:p], t["Agj"][:p], t["Jr"])
    # Q_ij = 1 - sum_{cd in PNO} |cd><cd| as an explicit p^2 x p^2 operator
    Pno = np.zeros((p * p, p * p))
    for c in range(k):
        for d in range(k):
            v = np.einsum("u,v->uv", t["Q"][:, c], t["Q"][:, d]).ravel()
            Pno += np.outer(v, v)
    R_Q = ((np.eye(p * p) - Pno) @ K_R.ravel()).reshape(p, p)
    # V over the extended basis (PNOs, i, j), minus the PNO-pair part of the geminal
    X = np.zeros((p + 2, k + 2))
    X[:p, :k] = t["Q"]
    X[p, k] = X[p + 1, k + 1] = 1.0
    Vh = np.einsum("ua,uv,vb->ab", X, K_V, X)
    R_pno = np.einsum("uc,uv,vd->cd", t["Q"], K_R, t["Q"])
    for a in range(k + 2):
        for b in range(k + 2):
            g = 0.0
            for c in range(k):
                for d in range(k):
                    g += R_pno[c, d] * float(np.dot(t["B"][c, :, a], t["B"][d, :, b]))
            Vh[a, b] -= g
    return {"Vh": Vh, "R_Q": R_Q, "K_jF": K_jF, "K_iF": K_iF}


def _pair_term(kern, t, o1_first, s1, s2, W):
    """2 Vt^{PR}_{PR} + B~^{PR}_{PR} for electron 1 in spin s1 on the pair's
    first orbital (o1_first) or second, electron 2 in spin s2 on the other."""
    p, k = t["Q"].shape
    Vh, R_Q, K_jF, K_iF = kern["Vh"], kern["R_Q"], kern["K_jF"], kern["K_iF"]
    T, S = t["T"], t["S"]
    if o1_first:
        iP, iR = k, k + 1                 # extended index of P's and R's orbitals
        sP_amp, sR_amp = S[0], S[1]
        K_RF, K_PF = K_jF, K_iF           # R_F: electron 2's orbital transformed
    else:                                 # electron 1 on j: every kernel transposed
        Vh, R_Q, T = Vh.T, R_Q.T, T.T
        iP, iR = k + 1, k
        sP_amp, sR_amp = S[1], S[0]
        K_RF, K_PF = K_iF.T, K_jF.T
    w = lambda sa, sb: W[2 * sa + sb, 2 * s1 + s2]     # SP projector weight  # noqa: E731
    spins = (ALPHA, BETA)
    # ---- Vbar over extended spin orbitals (PNOs and occupied i, j, both spins)
    ne = k + 2
    Vso = np.zeros((2 * ne, 2 * ne))
    for sa in spins:
        for sb in spins:
            for a in range(ne):
                for b in range(ne):
                    Vso[sa * ne + a, sb * ne + b] = 0.5 * (Vh[a, b] * w(sa, sb) - Vh[b, a] * w(sb, sa))
    P_so, R_so = s1 * ne + iP, s2 * ne + iR
    vt = Vso[P_so, R_so]                                            # V^{PR}_{PR}
    # ---- geminal Rbar over the complete virtual spin orbitals (PAO domain)
    def rbar(K):
        out = np.zeros((2 * p, 2 * p))
        for sa in spins:
            for sb in spins:
                out[sa * p:(sa + 1) * p, sb * p:(sb + 1) * p] = K * w(sa, sb) - K.T * w(sb, sa)
        return out
    Rb = rbar(R_Q)
    Fso = np.kron(np.eye(2), t["Fv"])                 # spin-diagonal Fock operator
    Qso = np.kron(np.eye(2), t["Q"])                  # PNO spin orbitals in the PAO basis
    # C^{PR}_{AB} over PNO spin orbitals
    Cso = Qso.T @ Fso @ Rb @ Qso + Qso.T @ Rb @ Fso @ Qso
    # amplitudes t^{AB}_{PR} and the amplitude + C term
    tso = np.zeros((2 * k, 2 * k))
    for sa in spins:
        for sb in spins:
            for a in range(k):
                for b in range(k):
                    tso[sa * k + a, sb * k + b] = (T[a, b] * (sa == s1) * (sb == s2)
                                                   - T[b, a] * (sb == s1) * (sa == s2))
    Vpno = np.zeros((2 * k, 2 * k))
    for sa in spins:
        for sb in spins:
            Vpno[sa * k:(sa + 1) * k, sb * k:(sb + 1) * k] = Vso[sa * ne:sa * ne + k, sb * ne:sb * ne + k]
    vt += 0.5 * float(np.sum((Vpno + Cso) * tso))
    # singles: V^{PR}_{PA} t^A_R + V^{PR}_{AR} t^A_P (t^A_X only for A in X's spin)
    for a in range(k):
        vt += Vso[P_so, s2 * ne + a] * sR_amp[a]
        vt += Vso[s1 * ne + a, R_so] * sP_amp[a]
    # ---- B~
    B = float(np.einsum("xy,yg,xg->", Rb, Fso, Rb))
    X_RF = 0.5 * float(np.sum(rbar(K_RF) * Rb))
    X_PF = 0.5 * float(np.sum(rbar(K_PF) * Rb))
    return 2.0 * vt + B - X_RF - X_PF


def bruteforce_full_pair_energies(wl, inputs_of_pair):
    """Per pair of the list, the (alpha-beta, alpha-alpha, beta-beta) sums of
    2 Vt + B~ over every occupied spin-orbital pair P < R on its two orbitals."""
    W = spin_projector_weights()
    occ = [(o, ALPHA) for o in range(wl.n_orb)]
    occ += [(o, BETA) for o in range(wl.n_orb) if int(wl.orb_kind[o]) == 0]
    index = {(int(i), int(j)): P for P, (i, j) in enumerate(zip(wl.pi, wl.pj))}
    cache = {}
    e = np.zeros((wl.n_pairs, 3))
    for u in range(len(occ)):
        for v in range(u + 1, len(occ)):
            (oP, sP), (oR, sR) = occ[u], occ[v]
            key = (min(oP, oR), max(oP, oR))
            if key not in index:
                continue
            Pr = index[key]
            if Pr not in cache:
                t = inputs_of_pair(Pr)
                cache[Pr] = (t, spatial_full_kernels(t))
            t, kern = cache[Pr]
            val = _pair_term(kern, t, oP <= oR, sP, sR, W)
            case = 0 if sP != sR else (1 if sP == ALPHA else 2)
            e[Pr, case] += val
    return e
