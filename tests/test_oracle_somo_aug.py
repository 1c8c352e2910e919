"""Pins of the oracle's SOMO-augmented PNO space (Sec. "SOMO handling").

Every PAO domain holds the SOMOs and the PAO-to-PNO matrix is extended by an
identity block, so a pair's virtual space is its PNOs followed by the SOMOs.
A SOMO is alpha-occupied, so only the beta spin case may excite into it.  The
pins below are independent of the oracle's closed forms:
- brute-force spin-orbital enumeration with the alpha virtual spin orbitals
  restricted to the PNOs;
- reduction to the plain PNO space when the SOMO amplitudes vanish;
- invariance under rotations within the SOMO space (Sec. "Pair-natural
  orbitals": the pair energies are invariant to unitary transformations within
  the SOMO space);
- central finite differences of the augmented gradient.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from spin_orbital_bruteforce import bruteforce_pair_energies, spatial_pair_intermediate


def _three_somo():
    return S.custom(4, 3, None, (10, 16), ("uniform", 4, 8), (14, 22), name="aug3")


@pytest.mark.parametrize("make", [S.tiny, _three_somo], ids=["tiny-1somo", "custom-3somo"])
def test_bruteforce_augmented(make):
    wl = make().augmented()
    ns = wl.somo_aug
    assert ns == wl.n_somo > 0
    r = O.run(wl)
    cache = {}

    def inputs(P):
        if P not in cache:
            cache[P] = S.pair_inputs(wl, P)
        return cache[P]
    e_bf = bruteforce_pair_energies(wl, lambda P: spatial_pair_intermediate(inputs(P), ns),
                                    lambda P: inputs(P)["T"],
                                    lambda P: int(wl.n_pno[P]))
    scale = np.abs(r["e_pair"]).max()
    assert np.abs(e_bf - r["e_pair"]).max() <= 1e-11 * scale
    # the restriction matters: without it the brute force gives other values
    e_free = bruteforce_pair_energies(wl, lambda P: spatial_pair_intermediate(inputs(P), ns),
                                      lambda P: inputs(P)["T"])
    assert np.abs(e_free - r["e_pair"]).max() > 1e-6 * scale


def test_augmented_reduces_without_somo_amplitudes():
    """Zero amplitudes into the SOMO virtuals: every spin case equals the plain
    PNO-space energy of the first p factor rows (the SOMO rows drop out)."""
    wl = S.tiny().augmented()
    ns = wl.somo_aug
    for P in range(wl.n_pairs):
        t = S.pair_inputs(wl, P)
        p, k = t["Q"].shape
        T = t["T"].copy()
        T[k:, :] = 0.0
        T[:, k:] = 0.0
        i, j = int(wl.pi[P]), int(wl.pj[P])
        kinds = (int(wl.orb_kind[i]), int(wl.orb_kind[j]))
        aug = O.pair_forward(dict(t, T=T), kinds[0], kinds[1], i == j, ns)
        plain = dict(t, T=T[:k, :k], **{x: t[x][:p] for x in ("Agi", "Agj", "Afi", "Afj")})
        ref = O.pair_forward(plain, kinds[0], kinds[1], i == j)
        assert np.allclose(aug["e"], ref["e"], rtol=1e-12, atol=1e-15), P
        assert np.allclose(aug["V"][:k, :k], ref["V"], rtol=1e-12, atol=1e-14), P


def test_somo_rotation_invariance():
    """Rotating the three SOMOs among themselves (their factor rows, and the
    SOMO rows and columns of T) leaves every pair energy unchanged."""
    wl = _three_somo().augmented()
    ns = wl.somo_aug
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((ns, ns)))
    for P in range(wl.n_pairs):
        t = S.pair_inputs(wl, P)
        p, k = t["Q"].shape
        i, j = int(wl.pi[P]), int(wl.pj[P])
        kinds = (int(wl.orb_kind[i]), int(wl.orb_kind[j]))
        ref = O.pair_forward(t, kinds[0], kinds[1], i == j, ns)
        rot = dict(t)
        for x in ("Agi", "Agj", "Afi", "Afj"):
            a = t[x].copy()
            a[p:] = U.T @ t[x][p:]
            rot[x] = a
        Ua = np.eye(k + ns)
        Ua[k:, k:] = U
        rot["T"] = Ua.T @ t["T"] @ Ua
        got = O.pair_forward(rot, kinds[0], kinds[1], i == j, ns)
        assert np.allclose(got["e"], ref["e"], rtol=1e-11, atol=1e-15), P


def _energy(t, kinds, same, ns):
    return sum(O.pair_forward(t, kinds[0], kinds[1], same, ns)["e"])


@pytest.mark.parametrize("P", [0, 3, 9, 14, 20, 27])
def test_augmented_gradient_central_differences(P):
    """Augmented gradient (Q only through its PNO block) against central
    differences, h = 1e-5, 12 random unit directions per tensor group."""
    wl = _three_somo().augmented()
    ns = wl.somo_aug
    P = P % wl.n_pairs
    t = S.pair_inputs(wl, P)
    i, j = int(wl.pi[P]), int(wl.pj[P])
    kinds = (int(wl.orb_kind[i]), int(wl.orb_kind[j]))
    f = O.pair_forward(t, kinds[0], kinds[1], i == j, ns)
    g = O.pair_gradient(t, f)
    for name in ("Agi", "Agj", "Afi", "Afj", "Q", "T"):
        assert g[name].shape == t[name].shape, name
    rng = np.random.default_rng(300 + P)
    h = 1e-5
    for name in ("Agi", "Agj", "Afi", "Afj", "Q", "T"):
        for _ in range(12):
            dvec = rng.standard_normal(t[name].shape)
            dvec /= np.linalg.norm(dvec)
            tp = dict(t, **{name: t[name] + h * dvec})
            tm = dict(t, **{name: t[name] - h * dvec})
            fd = (_energy(tp, kinds, i == j, ns) - _energy(tm, kinds, i == j, ns)) / (2 * h)
            an = float(np.sum(g[name] * dvec))
            scale = max(abs(an), np.linalg.norm(g[name]) * 1e-3)
            assert abs(fd - an) <= 1e-7 * scale + 1e-12, (name, fd, an)


def test_augmented_tiny_matches_stored_oracle_values():
    """Stored by tests/golden/make_golden.py (oracle/ and synthetic/ only):
    guards the augmented oracle and generator against silent drift."""
    import json
    import math
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_aug_oracle.json")
    with open(path) as fh:
        ref = json.load(fh)
    r = O.run(S.tiny().augmented())
    assert np.allclose(r["e_pair"], np.array(ref["e_pair"]), rtol=1e-12, atol=1e-13)
    assert math.isclose(r["E"], ref["E"], rel_tol=1e-12)
