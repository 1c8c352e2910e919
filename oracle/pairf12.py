"""FP64 CPU oracle for the pair-F12 path (Kumar, Neese, Valeev, arXiv 2008.03237).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  The CUDA path
shares no code with it.

It is the plain definition, pair by pair, in float64 with numpy/LAPACK
primitives and no blocking, fusion or reordering:

  1. local density fitting with the pair's auxiliary metric
     (Sec. "F12 integral transformations": the integrals of i and j are sieved
     onto the pair domain and recombined through local density fitting):
         J_g = L L^T,   C_x = A^g_x J_g^{-1},  x in {i, j}
  2. robust (Dunlap) fit of the F12-operator pair integral in the PAO domain:
         K = A^f_i C_j^T + C_i (A^f_j)^T - C_i J_f C_j^T
  3. transformation to the spin-independent PNO basis
     (Sec. "Pair-natural orbitals", "SOMO handling"):
         V = Q^T K Q
  4. the amplitude term 1/2 V^{ij}_{ab} t^{ab}_{ij} of Eq. Vtilde, with
     t^{ab}_{ji} = t^{ba}_{ij}:
         d = sum_ab V_ab T_ab,   x = sum_ab V_ab T_ba
  5. spin adaptation (Eqs. F12energy_sf*, the ROHF spin-case rules that follow):
         e_ab = n_ab (3 d + x) / 8,  e_aa = n_aa (d - x) / 4,  e_bb = n_bb (d - x) / 4
  6. E = sum over pairs, FP64, in pair-list order.

With SOMO augmentation (Sec. "SOMO handling"), every PAO domain also holds
the n_s SOMOs and the PAO-to-PNO matrix is extended by an n_s x n_s identity:
Q_aug = blockdiag(Q, I).  The factors then have p + n_s rows and V, T are
(k + n_s) x (k + n_s).  A SOMO is alpha-occupied and beta-unoccupied, so the
alpha virtual space of a pair is its PNOs and the beta virtual space its PNOs
and the SOMOs; each spin case sums only over its own virtual pairs
(spin_case_energies).

Readings of the paper that these steps fix (the paper gives the spin-orbital
equations only): the direct and exchange amplitude terms of one pair are
Vt_dir = d / 2 and Vt_exch = x / 2 (the factor 1/2 of Eq. Vtilde), the
same-spin term is (d - x) / 2, and the multiplicities n_ab, n_aa, n_bb follow
from the occupation rules (DOMO: alpha and beta occupied; SOMO: alpha only).
"""
import numpy as np
from scipy.linalg import solve_triangular

DOMO, SOMO = 0, 1


# ---------------------------------------------------------------- steps 1-4


def local_fit(Ag_i, Ag_j, Jg):
    """Step 1: C_x = A^g_x J_g^{-1} through the Cholesky factor of J_g.

    C J = A  <=>  J C^T = A^T (J symmetric)  <=>  L (L^T C^T) = A^T, solved by
    one forward and one backward triangular solve.  Raises
    numpy.linalg.LinAlgError when J_g is not positive definite."""
    L = np.linalg.cholesky(Jg)

    def solve(A):
        Y = solve_triangular(L, A.T, lower=True)
        return solve_triangular(L.T, Y, lower=False).T
    return solve(Ag_i), solve(Ag_j)


def robust_kernel(Af_i, Af_j, C_i, C_j, Jf):
    """Step 2: Dunlap's robust fit K = A^f_i C_j^T + C_i A^f_j^T - C_i J_f C_j^T."""
    return Af_i @ C_j.T + C_i @ Af_j.T - C_i @ Jf @ C_j.T


def pno_transform(K, Q):
    """Step 3: V = Q^T K Q."""
    return Q.T @ K @ Q


def amplitude_contractions(V, T):
    """Step 4: d = <V, T>, x = <V, T^T>."""
    return float(np.sum(V * T)), float(np.sum(V * T.T))


# ---------------------------------------------------------------- step 5


def spin_multiplicities(kind_i, kind_j, same_orbital):
    """(n_ab, n_aa, n_bb): how many spin-orbital pairs of each case pair (i, j) holds.

    ROHF occupations: a DOMO is occupied in alpha and beta, a SOMO in alpha
    only.  Opposite-spin pairs count every (alpha orbital, beta orbital) choice
    with distinct spin orbitals; same-spin pairs need two distinct orbitals."""
    a_i, b_i = 1, (1 if kind_i == DOMO else 0)
    a_j, b_j = 1, (1 if kind_j == DOMO else 0)
    if same_orbital:
        return (a_i * b_i, 0, 0)
    return (a_i * b_j + a_j * b_i, a_i * a_j, b_i * b_j)


def pair_energies(d, x, mult):
    n_ab, n_aa, n_bb = mult
    return (n_ab * (3.0 * d + x) / 8.0,
            n_aa * (d - x) / 4.0,
            n_bb * (d - x) / 4.0)


# ---------------------------------------------------------------- SOMO augmentation


def augment_pno(Q, n_s):
    """Sec. "SOMO handling": the PAO-to-PNO matrix extended by an n_s x n_s
    identity for the SOMOs that every PAO domain holds: blockdiag(Q, I)."""
    p, k = Q.shape
    Qa = np.zeros((p + n_s, k + n_s))
    Qa[:p, :k] = Q
    Qa[p:, k:] = np.eye(n_s)
    return Qa


def virtual_spaces(k, n_s):
    """Boolean masks over the k + n_s virtuals of an augmented pair: alpha
    virtuals are the PNOs (the SOMOs are alpha-occupied), beta virtuals are the
    PNOs and the SOMOs (beta-unoccupied)."""
    va = np.zeros(k + n_s, bool)
    va[:k] = True
    vb = np.ones(k + n_s, bool)
    return va, vb


def opposite_spin_orientations(kind_i, kind_j, same_orbital):
    """(c1, c2): whether the opposite-spin pair (i alpha, j beta) and the pair
    (j alpha, i beta) are occupied spin-orbital pairs; c1 + c2 = n_ab."""
    c1 = 1 if kind_j == DOMO else 0
    c2 = 1 if (kind_i == DOMO and not same_orbital) else 0
    return c1, c2


def spin_case_weights(kind_i, kind_j, same_orbital, va, vb):
    """Weight matrices Wd, Wx with E_P = sum_ab Wd_ab V_ab T_ab + Wx_ab V_ab T_ba.

    Spin case by spin case (alpha electron of the opposite-spin pair first):
      (i alpha, j beta):  3/8 sum_{a in va, b in vb} V_ab T_ab + 1/8 sum_{a in vb, b in va} V_ab T_ba
      (j alpha, i beta):  the same with V, T transposed (electron 1 on j)
      same spin sigma:    1/4 sum_{a, b in v_sigma} V_ab (T_ab - T_ba)
    which with va = vb = all virtuals is n_ab (3d + x)/8 + (n_aa + n_bb)(d - x)/4."""
    c1, c2 = opposite_spin_orientations(kind_i, kind_j, same_orbital)
    _, n_aa, n_bb = spin_multiplicities(kind_i, kind_j, same_orbital)
    ab = np.outer(va, vb).astype(float)
    ba = np.outer(vb, va).astype(float)
    aa = np.outer(va, va).astype(float)
    bb = np.outer(vb, vb).astype(float)
    Wd = 3.0 / 8.0 * (c1 * ab + c2 * ba) + (n_aa * aa + n_bb * bb) / 4.0
    Wx = 1.0 / 8.0 * (c1 * ba + c2 * ab) - (n_aa * aa + n_bb * bb) / 4.0
    return Wd, Wx


def spin_case_energies(V, T, kind_i, kind_j, same_orbital, va, vb):
    """(e_ab, e_aa, e_bb) with each spin case restricted to its own virtuals."""
    c1, c2 = opposite_spin_orientations(kind_i, kind_j, same_orbital)
    _, n_aa, n_bb = spin_multiplicities(kind_i, kind_j, same_orbital)

    def opposite(Vo, To):
        return (3.0 / 8.0 * float(np.sum((Vo * To)[np.ix_(va, vb)]))
                + 1.0 / 8.0 * float(np.sum((Vo * To.T)[np.ix_(vb, va)])))

    def same(v):
        blk = np.ix_(v, v)
        return 0.25 * float(np.sum((V * T)[blk]) - np.sum((V * T.T)[blk]))
    return (c1 * opposite(V, T) + c2 * opposite(V.T, T.T), n_aa * same(va), n_bb * same(vb))


# ---------------------------------------------------------------- per pair


def pair_forward(t, kind_i, kind_j, same_orbital, n_somo_aug=0):
    """All intermediates of one pair (t: dict of the pair's input tensors).

    n_somo_aug > 0: SOMO-augmented pair; t's factors have p + n_somo_aug rows
    (the SOMOs last), Q is p x k and T is (k + n_somo_aug) square."""
    C_i, C_j = local_fit(t["Agi"], t["Agj"], t["Jg"])
    K = robust_kernel(t["Afi"], t["Afj"], C_i, C_j, t["Jf"])
    Q = augment_pno(t["Q"], n_somo_aug) if n_somo_aug else t["Q"]
    V = pno_transform(K, Q)
    d, x = amplitude_contractions(V, t["T"])
    mult = spin_multiplicities(kind_i, kind_j, same_orbital)
    out = {"C_i": C_i, "C_j": C_j, "K": K, "V": V, "d": d, "x": x, "mult": mult}
    if n_somo_aug:
        va, vb = virtual_spaces(t["Q"].shape[1], n_somo_aug)
        out["e"] = spin_case_energies(V, t["T"], kind_i, kind_j, same_orbital, va, vb)
        out["W"] = spin_case_weights(kind_i, kind_j, same_orbital, va, vb)
        out["Q_aug"] = Q
    else:
        out["e"] = pair_energies(d, x, mult)
    return out


def energy_weights(mult):
    """E_P = alpha d + beta x for the multiplicities of the pair."""
    n_ab, n_aa, n_bb = mult
    return (3.0 * n_ab / 8.0 + (n_aa + n_bb) / 4.0,
            n_ab / 8.0 - (n_aa + n_bb) / 4.0)


def pair_gradient(t, fwd, dE=1.0):
    """Gradient of dE * E_P with respect to A^g_i, A^g_j, A^f_i, A^f_j, Q, T
    (J_g and J_f are constants).  Chain rule through steps 1-5:

        G_V = alpha T + beta T^T,      dT = alpha V + beta V^T
        Gb  = Q G_V Q^T,               dQ = K Q G_V^T + K^T Q G_V
        dA^f_i = Gb C_j,               dA^f_j = Gb^T C_i
        dC_i = Gb (A^f_j - C_j J_f),   dC_j = Gb^T (A^f_i - C_i J_f)
        dA^g_x = dC_x J_g^{-1}
    """
    T, V, K = t["T"], fwd["V"], fwd["K"]
    C_i, C_j = fwd["C_i"], fwd["C_j"]
    if "W" in fwd:     # SOMO-augmented: per-element weights, Q_aug = blockdiag(Q, I)
        Wd, Wx = fwd["W"]
        Q = fwd["Q_aug"]
        G_V = dE * (Wd * T + Wx * T.T)
        g = {"T": dE * (Wd * V + (Wx * V).T)}
    else:
        alpha, beta = energy_weights(fwd["mult"])
        Q = t["Q"]
        G_V = dE * (alpha * T + beta * T.T)
        g = {"T": dE * (alpha * V + beta * V.T)}
    Gb = Q @ G_V @ Q.T
    # only the PNO block of Q_aug is an input (the identity block is fixed)
    p, k = t["Q"].shape
    g["Q"] = (K @ Q @ G_V.T + K.T @ Q @ G_V)[:p, :k]
    g["Afi"] = Gb @ C_j
    g["Afj"] = Gb.T @ C_i
    dC_i = Gb @ (t["Afj"] - C_j @ t["Jf"])
    dC_j = Gb.T @ (t["Afi"] - C_i @ t["Jf"])
    Jinv_i, Jinv_j = local_fit(dC_i, dC_j, t["Jg"])   # dC J_g^{-1}, J_g symmetric
    g["Agi"] = Jinv_i
    g["Agj"] = Jinv_j
    return g


# ---------------------------------------------------------------- whole list


def run(wl, pairs=None, inputs=None, want_V=False, want_grad=False, dE=1.0):
    """Evaluate pairs of workload wl (all when pairs is None).

    inputs: optional callable P -> tensors (default: synthetic.pair_inputs).
    Returns dict with e_pair (n x 3), d, x, E (pair-order sum), and optionally
    V (list) and grads (list of dicts)."""
    from synthetic.workloads import pair_inputs
    get = inputs or (lambda P: pair_inputs(wl, P))
    idx = range(wl.n_pairs) if pairs is None else pairs
    idx = list(idx)
    e_pair = np.zeros((len(idx), 3))
    dd = np.zeros(len(idx))
    xx = np.zeros(len(idx))
    Vs, grads = [], []
    for n, P in enumerate(idx):
        t = get(P)
        i, j = int(wl.pi[P]), int(wl.pj[P])
        f = pair_forward(t, int(wl.orb_kind[i]), int(wl.orb_kind[j]), i == j,
                         int(getattr(wl, "somo_aug", 0)))
        e_pair[n] = f["e"]
        dd[n], xx[n] = f["d"], f["x"]
        if want_V:
            Vs.append(f["V"])
        if want_grad:
            grads.append(pair_gradient(t, f, dE))
    E = 0.0
    for n in range(len(idx)):
        E += e_pair[n, 0] + e_pair[n, 1] + e_pair[n, 2]
    out = {"pairs": idx, "e_pair": e_pair, "d": dd, "x": xx, "E": E,
           "E_kahan": kahan_total(e_pair), "sum_abs": float(np.abs(e_pair.sum(axis=1)).sum())}
    if want_V:
        out["V"] = Vs
    if want_grad:
        out["grads"] = grads
    return out


def kahan_total(e_pair):
    """Compensated sum of all pair energies (bounds the summation error of E)."""
    s, c = 0.0, 0.0
    for v in np.asarray(e_pair).ravel():
        y = v - c
        tt = s + y
        c = (tt - s) - y
        s = tt
    return s
