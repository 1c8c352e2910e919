"""Gather mode: per-orbital pair-extended blocks sieved on the device.

The sieved path must reproduce the packed path bit for bit on the same values,
match the oracle, and return per-orbital gradients equal to the oracle's
per-pair gradients scatter-added in pair order."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from synthetic import gather as G
from gpu_helpers import run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _gather_workload(n_domo=6, n_somo=1, cutoff=3):
    base = S.custom(n_domo, n_somo, cutoff, (10, 20), ("uniform", 2, 40), (10, 20), name="gather-mini")
    return G.make_gather(base)


def _upload_gather(gw, precision, variant=None, sieve_plain=False):
    import paper_2008_03237_gb300 as pf
    wl = gw.base
    blocks, (P, M, ld, off, tot) = G.orbital_blocks(gw)
    mp, ma, op, oa = G.pair_maps(gw)
    host, lay = S.packed_inputs(wl)   # J, Q, T of the pair sizes (A's unused)
    dev = {n: torch.from_numpy(host[n]).cuda() for n in ("Jg", "Jf", "Q", "T")}
    bl = {n: torch.from_numpy(v).cuda() for n, v in blocks.items()}
    eng = pf.PairF12(precision, variant=variant, sieve_plain=sieve_plain)
    eng.upload_pairs_gather(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, bl,
                            dict(off_orb=off, ext_pao=P, ext_aux=M, ext_ld=ld),
                            dict(map_pao=mp, map_aux=ma, off_map_pao=op, off_map_aux=oa), dev, lay)
    return eng, bl, (P, M, ld, off, tot), lay


def _packed_from_gather(gw):
    """The same pair inputs in packed layout (oracle view of every pair)."""
    wl = gw.base
    lay = S.packed_offsets(wl)
    buf = {n: np.zeros(max(lay["len_pm"], 2)) for n in ("Agi", "Agj", "Afi", "Afj")}
    buf.update({n: np.zeros(max(lay["len_mm"], 2)) for n in ("Jg", "Jf")})
    buf["Q"] = np.zeros(max(lay["len_pk"], 2))
    buf["T"] = np.zeros(max(lay["len_kk"], 2))
    for P in range(wl.n_pairs):
        t = G.pair_inputs(gw, P)
        for n, key in (("Agi", "pm"), ("Agj", "pm"), ("Afi", "pm"), ("Afj", "pm"), ("Jg", "mm"),
                       ("Jf", "mm"), ("Q", "pk"), ("T", "kk")):
            o = lay["off_" + key][P]
            buf[n][o:o + t[n].size] = t[n].ravel()
    return buf, lay


@pytest.mark.parametrize("sieve_plain", [False, True])
@pytest.mark.parametrize("precision,variant", [("fp64", 0), ("fp64", 1), ("mixed_fp32", 1),
                                               ("mixed_fp32", 2)])
def test_gather_equals_packed_and_oracle(built, precision, variant, sieve_plain):
    """TMA tile::gather4 sieve and plain-load sieve alike."""
    gw = _gather_workload()
    wl = gw.base
    eng, *_ = _upload_gather(gw, precision, variant, sieve_plain)
    eng.fit()
    assert eng.stats()["sieve_tma"] == (0 if sieve_plain else 1)
    E, e = eng.energy()
    e = e.cpu().numpy()
    from gpu_helpers import upload_host
    t, lay = upload_host(wl, _packed_from_gather(gw))
    ref_gpu = run(wl, precision, t=t, lay=lay, want_V=False, variant=variant)
    assert np.array_equal(e, ref_gpu["e_pair"])          # same values, same arithmetic
    ref = O.run(wl, inputs=lambda P: G.pair_inputs(gw, P))
    tol = 1e-10 if precision == "fp64" else 1e-5 * np.abs(ref["e_pair"]).max()
    assert np.abs(e - ref["e_pair"]).max() <= tol


@pytest.mark.parametrize("sieve_plain", [False, True])
def test_gather_backward_scatters_in_pair_order(built, sieve_plain):
    gw = _gather_workload(5, 2, 4)
    wl = gw.base
    eng, bl, (P, M, ld, off, tot), lay = _upload_gather(gw, "fp64", sieve_plain=sieve_plain)
    eng.fit()
    eng.energy()
    outs = []
    for _ in range(2):
        g = {"Bg": torch.zeros_like(bl["Bg"]), "Bf": torch.zeros_like(bl["Bf"]),
             "Q": torch.zeros(max(lay["len_pk"], 2), dtype=torch.float64, device="cuda"),
             "T": torch.zeros(max(lay["len_kk"], 2), dtype=torch.float64, device="cuda")}
        eng.backward_gather(0.5, g)
        torch.cuda.synchronize()
        outs.append({n: v.cpu().numpy() for n, v in g.items()})
    for n in outs[0]:
        assert np.array_equal(outs[0][n], outs[1][n]), n    # deterministic
    ref = O.run(wl, inputs=lambda q: G.pair_inputs(gw, q), want_grad=True, dE=0.5)
    mp, ma, op, oa = G.pair_maps(gw)
    want = {"Bg": np.zeros_like(outs[0]["Bg"]), "Bf": np.zeros_like(outs[0]["Bf"])}
    for q in range(wl.n_pairs):
        p_, m_ = int(wl.n_pao[q]), int(wl.n_aux[q])
        for side, o in enumerate((int(wl.pi[q]), int(wl.pj[q]))):
            rows = mp[op[q] + side * p_: op[q] + (side + 1) * p_]
            cols = ma[oa[q] + side * m_: oa[q] + (side + 1) * m_]
            for name, key in (("Bg", "Agi" if side == 0 else "Agj"), ("Bf", "Afi" if side == 0 else "Afj")):
                blk = want[name][off[o]:off[o] + P[o] * ld[o]].reshape(P[o], ld[o])
                blk[np.ix_(rows, cols)] += ref["grads"][q][key]
    for name in ("Bg", "Bf"):
        scale = np.abs(want[name]).max()
        assert np.abs(outs[0][name] - want[name]).max() <= 1e-9 * scale, name
    for q in range(wl.n_pairs):
        k_ = int(wl.n_pno[q])
        o = lay["off_kk"][q]
        assert np.abs(outs[0]["T"][o:o + k_ * k_].reshape(k_, k_) - ref["grads"][q]["T"]).max() <= \
            1e-9 * np.abs(ref["grads"][q]["T"]).max()


def test_gather_rejects_bad_maps(built):
    import paper_2008_03237_gb300 as pf
    gw = _gather_workload()
    wl = gw.base
    blocks, (P, M, ld, off, tot) = G.orbital_blocks(gw)
    mp, ma, op, oa = G.pair_maps(gw)
    host, lay = S.packed_inputs(wl)
    dev = {n: torch.from_numpy(host[n]).cuda() for n in ("Jg", "Jf", "Q", "T")}
    bl = {n: torch.from_numpy(v).cuda() for n, v in blocks.items()}
    eng = pf.PairF12("fp64")
    for bad in (mp[::-1].copy(), mp + 10**6):
        with pytest.raises(pf.Pf12Error) as ei:
            eng.upload_pairs_gather(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno,
                                    wl.n_aux, bl, dict(off_orb=off, ext_pao=P, ext_aux=M, ext_ld=ld),
                                    dict(map_pao=bad, map_aux=ma, off_map_pao=op, off_map_aux=oa),
                                    dev, lay)
        assert ei.value.code == -1
