"""Brute-force spin-orbital evaluation of the F12 amplitude term for tiny inputs.

Independent of oracle/: it inverts J_g by textbook Gauss-Jordan elimination,
forms every contraction with explicit einsum index strings, builds the spin
projectors of the SP ansatz from the spin functions of Eqs. P0, P1, singlet and
triplet, antisymmetrises spin-orbital quantities explicitly, enumerates the
occupied spin orbitals of the ROHF determinant (DOMO: alpha and beta, SOMO:
alpha only; Sec. "The PNO-based CCSD(T)F12bar Method", ROHF paragraph) and sums

    E = sum_{P<R} 2 Vt^{PR}_{PR},  Vt^{PR}_{PR} = 1/2 V^{PR}_{AB} t^{AB}_{PR}
                                                       (Eqs. F12 energy, Vtilde)
    V^{PR}_{AB} = 1/2 Rbar^{PR}_{AB} (geminal already contracted with g, Eq. V)
    R^{PR}_{AB} = <AB| O (1/2 P0 + 1/4 P1) |PR>            (Eq. ExpCorrWfnRspin)

over every pair of distinct occupied spin orbitals P, R, with O the spatial
pair operator whose matrix element <ab|O|ij> is the fitted PNO-basis
intermediate of the pair.
"""
import numpy as np

ALPHA, BETA = 0, 1


def gauss_jordan_inverse(A):
    """Textbook Gauss-Jordan inversion with partial pivoting (no LAPACK)."""
    n = A.shape[0]
    M = np.hstack([np.array(A, dtype=np.float64), np.eye(n)])
    for c in range(n):
        piv = c + int(np.argmax(np.abs(M[c:, c])))
        if piv != c:
            M[[c, piv]] = M[[piv, c]]
        M[c] = M[c] / M[c, c]
        for r in range(n):
            if r != c and M[r, c] != 0.0:
                M[r] = M[r] - M[r, c] * M[c]
    return M[:, n:]


def spatial_pair_intermediate(t, n_somo=0):
    """V_ab = <ab|O|ij> for one pair from its inputs, by explicit index contractions.

    n_somo > 0: the factors carry the SOMO rows last and the virtual space is
    the PNOs followed by the SOMOs themselves (Sec. "SOMO handling"), i.e. the
    transformation sends PAO row u < p through Q and SOMO row p + s to virtual
    k + s unchanged."""
    if n_somo:
        p, k = t["Q"].shape
        Q = np.zeros((p + n_somo, k + n_somo))
        for u in range(p):
            for a in range(k):
                Q[u, a] = t["Q"][u, a]
        for q in range(n_somo):
            Q[p + q, k + q] = 1.0
        t = dict(t, Q=Q)
    Jinv = gauss_jordan_inverse(t["Jg"])
    C_i = np.einsum("uX,XY->uY", t["Agi"], Jinv)
    C_j = np.einsum("uX,XY->uY", t["Agj"], Jinv)
    K = (np.einsum("uX,vX->uv", t["Afi"], C_j)
         + np.einsum("uX,vX->uv", C_i, t["Afj"])
         - np.einsum("uX,XY,vY->uv", C_i, t["Jf"], C_j))
    return np.einsum("ua,uv,vb->ab", t["Q"], K, t["Q"])


def spin_projector_weights():
    """4x4 matrix <s_A s_B| (1/2 P0 + 1/4 P1) |s_P s_R> in the basis
    |aa>, |ab>, |ba>, |bb> (first letter = electron 1)."""
    def ket(s1, s2):
        v = np.zeros(4)
        v[2 * s1 + s2] = 1.0
        return v
    singlet = (ket(ALPHA, BETA) - ket(BETA, ALPHA)) / np.sqrt(2.0)
    triplet0 = (ket(ALPHA, BETA) + ket(BETA, ALPHA)) / np.sqrt(2.0)
    P0 = np.outer(singlet, singlet)
    P1 = (np.outer(ket(BETA, BETA), ket(BETA, BETA)) + np.outer(triplet0, triplet0)
          + np.outer(ket(ALPHA, ALPHA), ket(ALPHA, ALPHA)))
    return 0.5 * P0 + 0.25 * P1


def _spin_orbital_pair_energy(Vs, Ts, sP, sR, W, n_alpha_virt=None):
    """2 Vt^{PR}_{PR} for electron 1 in spin sP, electron 2 in spin sR, given the
    spatial V^{oP oR} (Vs) and T^{oP oR} (Ts) of the ordered orbital pair.

    The virtual spin orbitals are (a, beta) for every spatial virtual a and
    (a, alpha) for a < n_alpha_virt only (default: all): in the SOMO-augmented
    space the trailing virtuals are SOMOs, which are alpha-occupied."""
    k = Vs.shape[0]
    na = k if n_alpha_virt is None else n_alpha_virt
    spin = np.array([ALPHA] * na + [BETA] * k)
    orb = np.array(list(range(na)) + list(range(k)))
    n = len(orb)
    O = np.zeros((n, n))
    t = np.zeros((n, n))
    for A in range(n):
        for B in range(n):
            a, b = orb[A], orb[B]
            O[A, B] = Vs[a, b] * W[2 * spin[A] + spin[B], 2 * sP + sR]
            t[A, B] = (Ts[a, b] * (spin[A] == sP) * (spin[B] == sR)
                       - Ts[b, a] * (spin[B] == sP) * (spin[A] == sR))
    Rbar = O - O.T                       # antisymmetrise the bra pair
    V = 0.5 * Rbar
    Vt = 0.5 * np.einsum("AB,AB->", V, t)
    return 2.0 * Vt


def bruteforce_pair_energies(wl, V_of_pair, T_of_pair, n_alpha_virt_of_pair=None):
    """Per pair of the list, the (alpha-beta, alpha-alpha, beta-beta) sums of
    2 Vt^{PR}_{PR} over all occupied spin-orbital pairs P < R on that pair's
    two orbitals.  n_alpha_virt_of_pair(P), when given, limits the alpha
    virtual spin orbitals of pair P to its leading spatial virtuals."""
    W = spin_projector_weights()
    occ = [(o, ALPHA) for o in range(wl.n_orb)]
    occ += [(o, BETA) for o in range(wl.n_orb) if int(wl.orb_kind[o]) == 0]
    index = {(int(i), int(j)): P for P, (i, j) in enumerate(zip(wl.pi, wl.pj))}
    e = np.zeros((wl.n_pairs, 3))
    for u in range(len(occ)):
        for w in range(u + 1, len(occ)):
            (oP, sP), (oR, sR) = occ[u], occ[w]
            key = (min(oP, oR), max(oP, oR))
            if key not in index:
                continue
            P = index[key]
            V, T = V_of_pair(P), T_of_pair(P)
            if oP > oR:                      # electron 1 sits on the pair's j orbital
                V, T = V.T, T.T
            na = None if n_alpha_virt_of_pair is None else n_alpha_virt_of_pair(P)
            val = _spin_orbital_pair_energy(V, T, sP, sR, W, na)
            case = 0 if sP != sR else (1 if sP == ALPHA else 2)
            e[P, case] += val
    return e
