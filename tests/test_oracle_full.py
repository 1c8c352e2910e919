"""Pins of the FP64 oracle of the complete pair F12 energy (oracle/full_f12.py)
against what the paper and the mathematics fix, independently of its code:

* brute-force spin-orbital sums of Eqs. F12 energy, Vtilde, V, C, B, X,
  Btilde and XAppr with the SP-ansatz spin projectors (tests/
  spin_orbital_bruteforce_full.py);
* the closed-shell reduction (no SOMO): the spin-free Hylleraas form with
  geminal amplitudes 3/8 and 1/8 (Sec. "Pair-natural orbitals": spin-
  independent PNOs reproduce the closed-shell formalism exactly);
* the canonical limit: with a diagonal virtual Fock operator and i_F = eps_i i
  the coupling term C vanishes and B~ = (2 f_v - eps_i - eps_j) X, the
  textbook canonical-orbital form of Eq. Btilde;
* the complete PNO space (k = p): Q_ij projects out the whole geminal, so C,
  B and X vanish;
* the PNO-projector term of Eq. Qij equals the PNO x PNO part of the complete
  resolution sum R g over the pair's virtual space, written out over PAOs;
* C of Eq. C is the derivative of the PNO-projected geminal along the
  Fock-coupled PNOs (central differences, exact for a quadratic);
* pair-swap symmetry: (j, i) with every input swapped gives the same energies.

A planted-mistake test monkeypatches plausible slips into the oracle and
checks that one of these pins catches each.
"""
import numpy as np
import pytest

import oracle.full_f12 as F
import synthetic as S
from spin_orbital_bruteforce import gauss_jordan_inverse
from spin_orbital_bruteforce_full import bruteforce_full_pair_energies
from synthetic.full import full_pair_inputs, orbital_energies


def _wl_open():
    return S.custom(3, 2, None, (6, 9), ("uniform", 2, 5), (8, 16), name="full-open")


def _inputs(wl):
    eps = orbital_energies(wl)
    return lambda P: full_pair_inputs(wl, P, eps)


def check_bruteforce(wl):
    r = F.run(wl)
    bf = bruteforce_full_pair_energies(wl, _inputs(wl))
    return np.abs(r["e_pair"] - bf).max() <= 1e-12 * np.abs(bf).max()


def test_bruteforce_spin_orbitals():
    """Every pair (DOMO-DOMO, SOMO-DOMO, SOMO-SOMO, diagonal) and spin case."""
    assert check_bruteforce(_wl_open())


def check_closed_shell(wl):
    r = F.run(wl)
    e_cs = 0.0
    for P in range(wl.n_pairs):
        tm = dict(zip(F.TERM_NAMES, r["terms"][P]))
        vd, vx = F.vtilde(tm)
        bd, bx = F.btilde(tm)
        ordered = 1 if wl.pi[P] == wl.pj[P] else 2
        # sum_{kl} (2 c_kl - c_lk) Vt + sum c (2 c - c') B~ with c = 3/8, c' = 1/8
        e_cs += ordered * (2.0 * (5.0 / 8.0 * vd - 1.0 / 8.0 * vx)
                           + (14.0 * bd + 2.0 * bx) / 64.0)
    return abs(r["e_pair"].sum() - e_cs) <= 1e-12 * abs(e_cs)


def test_closed_shell_reduction():
    assert check_closed_shell(S.custom(4, 0, None, (6, 10), ("uniform", 2, 5), (8, 14),
                                       name="full-closed"))


def _explicit_kernels(t):
    """K_R (PAO x PAO) and its projection, written out with a Gauss-Jordan
    inverse and the projector as an explicit p^2 x p^2 matrix."""
    p, k = t["Q"].shape
    Jinv = gauss_jordan_inverse(t["Jg"])
    Ci = t["Agi"][:p] @ Jinv
    Cj = t["Agj"][:p] @ Jinv
    K = t["Ari"][:p] @ Cj.T + Ci @ t["Arj"][:p].T - Ci @ t["Jr"] @ Cj.T
    Pp = t["Q"] @ t["Q"].T
    R_Q = ((np.eye(p * p) - np.kron(Pp, Pp)) @ K.ravel()).reshape(p, p)
    return K, R_Q


def check_canonical(wl):
    wl.meta["canonical"] = True
    eps = orbital_energies(wl)
    r = F.run(wl)
    ok = True
    for P in range(wl.n_pairs):
        tm = dict(zip(F.TERM_NAMES, r["terms"][P]))
        t = full_pair_inputs(wl, P, eps)
        _, R_Q = _explicit_kernels(t)
        de = 2 * 1.5 - eps[wl.pi[P]] - eps[wl.pj[P]]
        bd, bx = F.btilde(tm)
        nd, nx = float(np.sum(R_Q * R_Q)), float(np.sum(R_Q * R_Q.T))
        ok &= abs(bd - de * nd) <= 1e-11 * abs(de * nd)
        ok &= abs(bx - de * nx) <= 1e-11 * max(abs(de * nd), 1e-300)
        scale = abs(tm["d"]) + abs(tm["x"]) + 1e-300
        ok &= abs(tm["c_d"]) <= 1e-12 * scale and abs(tm["c_x"]) <= 1e-12 * scale
    return ok


def test_canonical_limit():
    assert check_canonical(_wl_open())


def test_complete_pno_space():
    """k = p: Q square orthogonal, Q_ij removes the whole geminal."""
    wl = S.custom(3, 1, None, (6, 6), ("uniform", 6, 6), (10, 14), name="full-k=p")
    r = F.run(wl)
    t = r["terms"]
    names = list(F.TERM_NAMES)
    scale = np.abs(t[:, names.index("d")]).max()
    for n in ("c_d", "c_x", "b_dd", "b_dx", "xj_dd", "xj_dx", "xi_dd", "xi_dx"):
        assert np.abs(t[:, names.index(n)]).max() <= 1e-12 * scale, n


def test_projector_term_is_the_pno_part_of_the_complete_sum():
    """With PNO-pair factors built from PAO-level ones, B[c, X, q] =
    sum_{uv} Q[u, c] Qx[v, q] L[u, v, X], the projector term equals the full
    resolution sum over the PAO domain minus the same sum with the projected
    geminal R_Q: sum_{ab in PAO} (K_R - R_Q)[a, b] (a q|b q')."""
    rng = np.random.default_rng(3)
    p, k, m = 7, 4, 9
    Q, _ = np.linalg.qr(rng.standard_normal((p, k)))
    Qx = F.extended_pnos(Q)
    L = rng.standard_normal((p, p + 2, m))
    K = rng.standard_normal((p, p))
    B = np.einsum("uc,vq,uvX->cXq", Q, Qx, L)
    G = F.projector_term(Q.T @ K @ Q, B)
    Pp = Q @ Q.T
    R_Q = ((np.eye(p * p) - np.kron(Pp, Pp)) @ K.ravel()).reshape(p, p)
    want = np.zeros((k + 2, k + 2))
    for a in range(p):
        for b in range(p):
            g = np.einsum("vX,wX->vw", L[a], L[b])          # (a v|b w) over the rows
            want += (K - R_Q)[a, b] * (Qx.T @ g @ Qx)
    assert np.abs(G - want).max() <= 1e-12 * np.abs(want).max()


def test_c_is_the_fock_derivative_of_the_projected_geminal():
    """C = d/dl (Q + l Ft)^T K_R (Q + l Ft) at l = 0 (central difference, exact
    for this quadratic), Ft = (1 - Q Q^T) F_v Q."""
    wl = _wl_open()
    eps = orbital_energies(wl)
    for P in (1, 4, 9):
        t = full_pair_inputs(wl, P, eps)
        _, aux = F.pair_terms(t)
        K, _ = _explicit_kernels(t)
        Ft = F.fock_coupling(t["Fv"], t["Q"])
        h = 0.5
        Qp, Qm = t["Q"] + h * Ft, t["Q"] - h * Ft
        fd = (Qp.T @ K @ Qp - Qm.T @ K @ Qm) / (2 * h)
        assert np.abs(aux["C"] - fd).max() <= 1e-12 * np.abs(fd).max()


def _swap_inputs(t):
    """Inputs of the pair (j, i): the i and j roles exchanged everywhere."""
    p, k = t["Q"].shape
    s = {}
    for x in ("g", "f"):
        Ai, Aj = t["A%si" % x].copy(), t["A%sj" % x].copy()
        Ai[[p, p + 1]] = Ai[[p + 1, p]]      # rows (j j), (j i) -> first orbital first
        Aj[[p, p + 1]] = Aj[[p + 1, p]]
        s["A%si" % x], s["A%sj" % x] = Aj, Ai
    for a, b in (("Ari", "Arj"), ("AgiF", "AgjF"), ("AriF", "ArjF")):
        s[a], s[b] = t[b], t[a]
    for n in ("Jg", "Jf", "Jr", "Q", "Fv"):
        s[n] = t[n]
    s["T"] = t["T"].T.copy()
    s["S"] = t["S"][::-1].copy()
    B = t["B"].copy()
    B[:, :, [k, k + 1]] = B[:, :, [k + 1, k]]
    s["B"] = B
    return s


def test_pair_swap_symmetry():
    wl = _wl_open()
    eps = orbital_energies(wl)
    for P in range(wl.n_pairs):
        t = full_pair_inputs(wl, P, eps)
        a, _ = F.pair_terms(t)
        b, _ = F.pair_terms(_swap_inputs(t))
        ea = F.spin_case_energies(a, (1, 1, 1))
        eb = F.spin_case_energies(b, (1, 1, 1))
        assert np.allclose(ea, eb, rtol=1e-12, atol=0), P


# ------------------------------------------------------------ planted mistakes


def _plants():
    def v_no_half(tm):
        vd, vx = ORIG["vtilde"](tm)
        return vd + 0.5 * tm["vocc_d"], vx
    def singles_swapped(t):
        out, aux = ORIG["pair_terms"](dict(t, S=t["S"][::-1].copy()))
        return out, aux
    def c_one_sided(Fv, Q):
        return Fv @ Q                         # drops the complement projector
    def b_no_x(tm):
        return tm["b_dd"] - tm["xj_dd"], tm["b_dx"] - tm["xj_dx"]
    def proj_with_RQ(R_pno, B):
        return 2.0 * ORIG["projector_term"](R_pno, B)
    def spin_ss_prefactor(tm, mult):
        e = list(ORIG["spin_case_energies"](tm, mult))
        bd, bx = F.btilde(tm)
        e[1] += mult[1] * (bd - bx) / 16.0
        return tuple(e)
    return {"vtilde": v_no_half, "pair_terms": singles_swapped, "fock_coupling": c_one_sided,
            "btilde": b_no_x, "projector_term": proj_with_RQ,
            "spin_case_energies": spin_ss_prefactor}


ORIG = {n: getattr(F, n) for n in ("vtilde", "pair_terms", "fock_coupling", "btilde",
                                   "projector_term", "spin_case_energies")}


@pytest.mark.parametrize("name", sorted(ORIG))
def test_planted_mistakes_are_caught(monkeypatch, name):
    monkeypatch.setattr(F, name, _plants()[name])
    wl_open = S.custom(3, 2, None, (6, 9), ("uniform", 2, 5), (8, 16), name="plant")
    caught = not check_bruteforce(wl_open)
    if not caught:
        caught = not check_closed_shell(S.custom(4, 0, None, (6, 10), ("uniform", 2, 5),
                                                 (8, 14), name="plant-cs"))
    if not caught:
        caught = not check_canonical(S.custom(3, 2, None, (6, 9), ("uniform", 2, 5), (8, 16),
                                              name="plant-canon"))
    assert caught, name
