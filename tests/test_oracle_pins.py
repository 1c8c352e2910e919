"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term of
the robust fit, a transposed Q, a wrong spin multiplicity or prefactor, a swapped
direct/exchange contraction) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from synthetic.philox import philox4x32
from spin_orbital_bruteforce import (bruteforce_pair_energies, gauss_jordan_inverse,
                                     spatial_pair_intermediate)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ generator


def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors of the Random123 distribution (SC'11)."""
    cases = [((0, 0, 0, 0, 0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
             ((0xffffffff,) * 6, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
             ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344, 0xa4093822, 0x299f31d0),
              (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for inp, want in cases:
        got = tuple(int(v) for v in philox4x32(*inp))
        assert got == want


@pytest.mark.parametrize("name,count", [("tiny", 36), ("c40h81", 2821), ("c160h321", 14446),
                                        ("lattice703", 29226)])
def test_pair_counts(name, count):
    wl = S.WORKLOADS[name]()
    assert wl.n_pairs == count
    assert np.all(wl.pi <= wl.pj)
    assert np.all(wl.n_pno <= wl.n_pao)


def test_generator_properties():
    wl = S.tiny()
    for P in (0, 5, 35):
        t = S.pair_inputs(wl, P)
        p, k, m = int(wl.n_pao[P]), int(wl.n_pno[P]), int(wl.n_aux[P])
        assert t["Agi"].shape == (p, m) and t["Jg"].shape == (m, m) and t["Q"].shape == (p, k)
        for J in (t["Jg"], t["Jf"]):
            assert np.array_equal(J, J.T)
            assert np.linalg.eigvalsh(J).min() > 0.09
        assert np.allclose(t["Q"].T @ t["Q"], np.eye(k), atol=1e-13)
        if wl.pi[P] == wl.pj[P]:
            assert np.array_equal(t["T"], t["T"].T)
            assert np.array_equal(t["Agi"], t["Agj"])
    # the decay s_P = exp(-0.3 |i - j|)
    assert np.allclose(wl.decay, np.exp(-0.3 * np.abs(wl.pj - wl.pi)), rtol=1e-14)


# ------------------------------------------------------------------ P1


def test_closed_shell_reduction():
    """No SOMO: the open-shell spin-case sum equals the closed-shell SP-ansatz
    energy sum_{ordered ij} 2 (5/8 Vt_dir - 1/8 Vt_exch) (geminal amplitudes 3/8
    and 1/8), the paper's statement that spin-independent PNOs reproduce the
    closed-shell formalism exactly (Sec. "Pair-natural orbitals")."""
    wl = S.custom(6, 0, None, (12, 20), ("uniform", 4, 9), (20, 40), name="closed-shell")
    r = O.run(wl)
    e_open = r["e_pair"].sum()
    e_cs = 0.0
    for P in range(wl.n_pairs):
        d, x = r["d"][P], r["x"][P]
        vt_d, vt_x = d / 2.0, x / 2.0
        ordered = 1 if wl.pi[P] == wl.pj[P] else 2      # (i,j) and (j,i) give equal terms
        e_cs += ordered * 2.0 * (5.0 / 8.0 * vt_d - 1.0 / 8.0 * vt_x)
    assert abs(e_open - e_cs) <= 1e-12 * abs(e_cs)


# ------------------------------------------------------------------ P2


def test_bruteforce_spin_orbitals():
    """Tiny doublet (7 DOMO + 1 SOMO): per pair and spin case, the oracle equals the
    brute-force spin-orbital enumeration built from the SP projectors."""
    wl = S.tiny()
    r = O.run(wl)
    cache = {}

    def inputs(P):
        if P not in cache:
            cache[P] = S.pair_inputs(wl, P)
        return cache[P]
    e_bf = bruteforce_pair_energies(wl, lambda P: spatial_pair_intermediate(inputs(P)),
                                    lambda P: inputs(P)["T"])
    scale = np.abs(r["e_pair"]).max()
    assert np.abs(e_bf - r["e_pair"]).max() <= 1e-11 * scale
    # spin-case structure: 3 cases for DOMO-DOMO, 2 for SOMO-DOMO, 1 for SOMO-SOMO
    for P in range(wl.n_pairs):
        i, j = int(wl.pi[P]), int(wl.pj[P])
        nz = tuple(int(v != 0.0) for v in e_bf[P])
        kinds = (int(wl.orb_kind[i]), int(wl.orb_kind[j]))
        if i == j:
            assert nz[1:] == (0, 0)
        elif kinds == (0, 0):
            assert nz == (1, 1, 1)
        elif 1 in kinds and 0 in kinds:
            assert nz == (1, 1, 0)
    assert abs(e_bf.sum() - r["E"]) <= 1e-11 * np.abs(r["e_pair"]).sum()


# ------------------------------------------------------------------ P3


def test_untruncated_pno_space():
    """k = p with square orthogonal Q: the PNO-basis contraction equals the
    PAO-basis one, sum_ab V_ab T_ab = sum_cd K_cd (Q T Q^T)_cd."""
    rng = np.random.default_rng(3)
    p, m = 9, 17
    X = rng.standard_normal((m, m)) / np.sqrt(m)
    t = {n: rng.standard_normal((p, m)) for n in ("Agi", "Agj", "Afi", "Afj")}
    t["Jg"] = X @ X.T + 0.1 * np.eye(m)
    Y = rng.standard_normal((m, m)) / np.sqrt(m)
    t["Jf"] = Y @ Y.T + 0.1 * np.eye(m)
    t["Q"], _ = np.linalg.qr(rng.standard_normal((p, p)))
    t["T"] = 1e-2 * rng.standard_normal((p, p))
    f = O.pair_forward(t, O.DOMO, O.DOMO, False)
    Tpao = t["Q"] @ t["T"] @ t["Q"].T
    assert math.isclose(f["d"], float(np.sum(f["K"] * Tpao)), rel_tol=1e-12)
    assert math.isclose(f["x"], float(np.sum(f["K"] * Tpao.T)), rel_tol=1e-12)


# ------------------------------------------------------------------ P4


def _fittable_pair(rng, p, m, k):
    X = rng.standard_normal((m, m)) / np.sqrt(m)
    Jg = X @ X.T + 0.1 * np.eye(m)
    Y = rng.standard_normal((m, m)) / np.sqrt(m)
    Jf = Y @ Y.T + 0.1 * np.eye(m)
    B_i, B_j = rng.standard_normal((p, m)), rng.standard_normal((p, m))
    Q, _ = np.linalg.qr(rng.standard_normal((p, k)))
    t = {"Agi": B_i @ Jg, "Agj": B_j @ Jg, "Afi": B_i @ Jf, "Afj": B_j @ Jf,
         "Jg": Jg, "Jf": Jf, "Q": Q, "T": 1e-2 * rng.standard_normal((k, k))}
    return t, B_i, B_j


def test_complete_aux_exact_and_robust_order():
    """Exactly fittable factors (A^g = B J_g, A^f = B J_f): K = B_i J_f B_j^T.
    Perturbing A^g by eps E leaves an O(eps^2) error in the robust (Dunlap)
    K but an O(eps) error in the one-sided fit A^f_i C_j^T."""
    rng = np.random.default_rng(11)
    t, B_i, B_j = _fittable_pair(rng, 8, 15, 5)
    K_exact = B_i @ t["Jf"] @ B_j.T
    f = O.pair_forward(t, O.DOMO, O.DOMO, False)
    assert np.abs(f["K"] - K_exact).max() <= 1e-10 * np.abs(K_exact).max()
    E_i, E_j = rng.standard_normal(B_i.shape), rng.standard_normal(B_j.shape)
    eps = np.array([1e-2, 1e-3, 1e-4, 1e-5])
    err_r, err_1 = [], []
    for e in eps:
        tt = dict(t, Agi=t["Agi"] + e * E_i, Agj=t["Agj"] + e * E_j)
        C_i, C_j = O.local_fit(tt["Agi"], tt["Agj"], tt["Jg"])
        K = O.robust_kernel(tt["Afi"], tt["Afj"], C_i, C_j, tt["Jf"])
        err_r.append(np.abs(K - K_exact).max())
        err_1.append(np.abs(tt["Afi"] @ C_j.T - K_exact).max())
    slope_r = np.polyfit(np.log(eps), np.log(err_r), 1)[0]
    slope_1 = np.polyfit(np.log(eps), np.log(err_1), 1)[0]
    assert abs(slope_r - 2.0) < 0.05, slope_r
    assert abs(slope_1 - 1.0) < 0.05, slope_1


# ------------------------------------------------------------------ P5


def test_pair_swap_symmetry():
    """(j, i) with swapped factors and T^T gives V^T and identical energies."""
    wl = S.tiny()
    for P in (3, 20, 34):
        t = S.pair_inputs(wl, P)
        i, j = int(wl.pi[P]), int(wl.pj[P])
        ki, kj = int(wl.orb_kind[i]), int(wl.orb_kind[j])
        f = O.pair_forward(t, ki, kj, i == j)
        s = dict(t, Agi=t["Agj"], Agj=t["Agi"], Afi=t["Afj"], Afj=t["Afi"], T=t["T"].T)
        g = O.pair_forward(s, kj, ki, i == j)
        assert np.allclose(g["V"], f["V"].T, rtol=0, atol=1e-12 * np.abs(f["V"]).max())
        for a, b in zip(f["e"], g["e"]):
            assert math.isclose(a, b, rel_tol=1e-12, abs_tol=1e-14)


# ------------------------------------------------------------------ P6


def test_special_cases():
    wl = S.custom(2, 2, None, (10, 14), ("uniform", 3, 6), (16, 24), name="special")
    r = O.run(wl)
    for P in range(wl.n_pairs):
        i, j = int(wl.pi[P]), int(wl.pj[P])
        ki, kj = int(wl.orb_kind[i]), int(wl.orb_kind[j])
        if ki == kj == O.SOMO and i == j:
            assert tuple(r["e_pair"][P]) == (0.0, 0.0, 0.0)
        if i == j:
            # V and T symmetric: direct and exchange agree, same-spin vanishes
            assert math.isclose(r["d"][P], r["x"][P], rel_tol=1e-12)
            assert r["e_pair"][P][1] == 0.0 and r["e_pair"][P][2] == 0.0
        if ki == kj == O.SOMO and i != j:
            assert r["e_pair"][P][0] == 0.0 and r["e_pair"][P][2] == 0.0


def test_cholesky_solve_matches_gauss_jordan():
    wl = S.tiny()
    t = S.pair_inputs(wl, 9)
    C_i, C_j = O.local_fit(t["Agi"], t["Agj"], t["Jg"])
    Jinv = gauss_jordan_inverse(t["Jg"])
    for C, A in ((C_i, t["Agi"]), (C_j, t["Agj"])):
        ref = A @ Jinv
        assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


def test_not_spd_is_an_error():
    t = S.pair_inputs(S.tiny(), 1)
    t["Jg"] = t["Jg"] - 10.0 * np.eye(t["Jg"].shape[0])
    with pytest.raises(np.linalg.LinAlgError):
        O.local_fit(t["Agi"], t["Agj"], t["Jg"])


# ------------------------------------------------------------------ gradient


def _pair_energy(t, kinds, same):
    return sum(O.pair_forward(t, kinds[0], kinds[1], same)["e"])


@pytest.mark.parametrize("P", [0, 4, 15, 34])
def test_gradient_central_differences(P):
    """Central differences, h = 1e-5, along 20 random unit directions per tensor
    group, against the analytic oracle gradient (relative agreement <= 1e-7)."""
    wl = S.custom(4, 1, None, (10, 16), ("uniform", 4, 8), (14, 22), name="grad")
    P = P % wl.n_pairs
    t = S.pair_inputs(wl, P)
    i, j = int(wl.pi[P]), int(wl.pj[P])
    kinds = (int(wl.orb_kind[i]), int(wl.orb_kind[j]))
    f = O.pair_forward(t, kinds[0], kinds[1], i == j)
    g = O.pair_gradient(t, f)
    rng = np.random.default_rng(100 + P)
    h = 1e-5
    for name in ("Agi", "Agj", "Afi", "Afj", "Q", "T"):
        for _ in range(20):
            dvec = rng.standard_normal(t[name].shape)
            dvec /= np.linalg.norm(dvec)
            tp = dict(t, **{name: t[name] + h * dvec})
            tm = dict(t, **{name: t[name] - h * dvec})
            fd = (_pair_energy(tp, kinds, i == j) - _pair_energy(tm, kinds, i == j)) / (2 * h)
            an = float(np.sum(g[name] * dvec))
            scale = max(abs(an), np.linalg.norm(g[name]) * 1e-3)
            assert abs(fd - an) <= 1e-7 * scale + 1e-12, (name, fd, an)


# ------------------------------------------------------------------ regression


def test_tiny_matches_stored_oracle_values():
    """Stored by tests/golden/make_golden.py (oracle/ and synthetic/ only):
    guards the oracle and the generator against silent drift."""
    with open(os.path.join(GOLDEN, "tiny_oracle.json")) as fh:
        ref = json.load(fh)
    r = O.run(S.tiny())
    assert np.allclose(r["e_pair"], np.array(ref["e_pair"]), rtol=1e-12, atol=1e-13)
    assert math.isclose(r["E"], ref["E"], rel_tol=1e-12)
