"""Gather-mode generator: sieving a pair's rows and columns out of the
per-orbital blocks gives exactly the pair's factors drawn from global indices,
and every pair domain lies inside both orbitals' extended domains."""
import numpy as np

import synthetic as S
from synthetic import gather as G


def test_sieve_reproduces_pair_factors():
    gw = G.make_gather(S.custom(5, 1, 3, (10, 20), ("uniform", 3, 8), (10, 20)))
    blocks, (P, M, ld, off, _) = G.orbital_blocks(gw)
    mp, ma, op, oa = G.pair_maps(gw)
    wl = gw.base
    for q in range(wl.n_pairs):
        t = G.pair_inputs(gw, q)
        p, m = int(wl.n_pao[q]), int(wl.n_aux[q])
        for side, o in enumerate((int(wl.pi[q]), int(wl.pj[q]))):
            rows = mp[op[q] + side * p: op[q] + (side + 1) * p]
            cols = ma[oa[q] + side * m: oa[q] + (side + 1) * m]
            assert np.all(np.diff(rows) > 0) and np.all(np.diff(cols) > 0)
            for name, key in (("Bg", "Agi" if side == 0 else "Agj"), ("Bf", "Afi" if side == 0 else "Afj")):
                B = blocks[name][off[o]:off[o] + P[o] * ld[o]].reshape(P[o], ld[o])
                assert np.array_equal(B[np.ix_(rows, cols)], t[key])
        assert set(gw.pao_atoms[q]) <= set(gw.ext_pao_atoms[int(wl.pi[q])])
        assert set(gw.aux_atoms[q]) <= set(gw.ext_aux_atoms[int(wl.pj[q])])
