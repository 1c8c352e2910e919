"""Parity of the SOMO-augmented PNO space (Sec. "SOMO handling") through the C
ABI with the FP64 CPU oracle: factor blocks with the SOMO rows last, Q_aug =
blockdiag(Q, I), alpha virtuals = PNOs, beta virtuals = PNOs + SOMOs.

Bars as for the plain space: FP64 within 1e-10 Eh per pair and V within 1e-11
relative; mixed within 1e-5 per pair (relative) and 1 uEh normalised total;
gradients within 1e-9 (FP64) and 2e-5 (mixed) of the largest entry per block.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_helpers import normalised_error, sized_workload, upload_host

pytestmark = pytest.mark.gpu

# ragged sizes across tile and panel edges, k = 1 and k = p, with 3 SOMOs
EDGE_SIZES = [(1, 1, 1), (7, 7, 3), (5, 2, 33), (65, 61, 65), (130, 70, 129), (200, 1, 257),
              (33, 33, 31), (90, 41, 190), (64, 61, 64), (128, 96, 300)]
GRADS = ("Agi", "Agj", "Afi", "Afj", "Q", "T")


def _tiny():
    return S.tiny().augmented()


def _three_somo():
    return S.custom(5, 3, None, (40, 150), ("uniform", 1, 90), (30, 230),
                    name="mini-3somo").augmented()


def _edge():
    return sized_workload(EDGE_SIZES, kinds=[0] * 8 + [1] * 3, diag_every=3,
                          name="edge-sizes").augmented()


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _run(wl, precision, variant=None, want_grad=False, t=None, lay=None):
    import paper_2008_03237_gb300 as pf
    if t is None:
        t, lay = upload_host(wl)
    eng = pf.PairF12(precision, variant=variant, augment_somo=True)
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    E, e = eng.energy()
    out = {"E": E, "e_pair": e.cpu().numpy(), "status": eng.pair_status()}
    V = eng.build_v().cpu().numpy()
    out["V"] = [S.unpack(V, lay["off_kk"], P, int(wl.n_virt[P]), int(wl.n_virt[P]))
                for P in range(wl.n_pairs)]
    if want_grad:
        g = {n: torch.zeros_like(t[n]) for n in GRADS}
        eng.backward(1.0, g)
        out["grads"] = {n: v.cpu().numpy() for n, v in g.items()}
    torch.cuda.synchronize()
    eng.close()
    return out, lay


def _blocks(wl, lay, g, P):
    r, p, k, v, m = (int(wl.n_rows[P]), int(wl.n_pao[P]), int(wl.n_pno[P]), int(wl.n_virt[P]),
                     int(wl.n_aux[P]))
    out = {n: S.unpack(g[n], lay["off_pm"], P, r, m) for n in ("Agi", "Agj", "Afi", "Afj")}
    out["Q"] = S.unpack(g["Q"], lay["off_pk"], P, p, k)
    out["T"] = S.unpack(g["T"], lay["off_kk"], P, v, v)
    return out


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("make", [_tiny, _three_somo, _edge])
def test_augmented_forward_fp64(built, make, variant):
    wl = make()
    ref = O.run(wl, want_V=True)
    r, _ = _run(wl, "fp64", variant)
    assert (r["status"] == 0).all()
    assert np.abs(r["e_pair"] - ref["e_pair"]).max() <= 1e-10
    for P in range(wl.n_pairs):
        scale = max(np.abs(ref["V"][P]).max(), 1e-300)
        assert np.abs(r["V"][P] - ref["V"][P]).max() <= 1e-11 * scale, P
    assert abs(r["E"] - ref["E"]) <= 1e-10 * max(1.0, abs(ref["E"]))


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("make", [_tiny, _three_somo, _edge])
def test_augmented_forward_mixed(built, make, variant):
    wl = make()
    ref = O.run(wl)
    r, _ = _run(wl, "mixed_fp32", variant)
    rel = np.abs(r["e_pair"] - ref["e_pair"]).max() / np.abs(ref["e_pair"]).max()
    assert rel <= 1e-5, rel
    assert normalised_error(r["E"] - ref["E"], ref["sum_abs"], wl.n_orb) <= 1e-6


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("mixed_fp32", 2e-5)])
@pytest.mark.parametrize("make", [_tiny, _edge])
def test_augmented_gradients(built, make, precision, bar):
    wl = make()
    ref = O.run(wl, want_grad=True)
    r, lay = _run(wl, precision, want_grad=True)
    for P in range(wl.n_pairs):
        got = _blocks(wl, lay, r["grads"], P)
        for name, w in ref["grads"][P].items():
            assert got[name].shape == w.shape, (P, name)
            scale = max(np.abs(w).max(), 1e-300)
            assert np.abs(got[name] - w).max() <= bar * scale, (P, name)


def test_augment_flag_without_somos_is_the_plain_path(built):
    """augment_somo on a closed-shell list (n_s = 0) gives bitwise the plain result."""
    import paper_2008_03237_gb300 as pf
    wl = S.custom(6, 0, None, (40, 120), ("uniform", 4, 40), (30, 160), name="closed")
    t, lay = upload_host(wl)
    res = []
    for aug in (False, True):
        eng = pf.PairF12("fp64", augment_somo=aug)
        eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
        eng.fit()
        E, e = eng.energy()
        res.append((E, e.cpu().numpy()))
        eng.close()
    assert res[0][0] == res[1][0] and np.array_equal(res[0][1], res[1][1])


def test_augmented_gather_mode_unsupported(built):
    import paper_2008_03237_gb300 as pf
    from synthetic import gather as G
    gw = G.make_gather(S.custom(4, 1, 2, (10, 20), ("uniform", 2, 10), (10, 20), name="g"))
    wl = gw.base
    blocks, (P, M, ld, off, _) = G.orbital_blocks(gw)
    mp, ma, op, oa = G.pair_maps(gw)
    host, lay = S.packed_inputs(wl)
    dev = {n: torch.from_numpy(host[n]).cuda() for n in ("Jg", "Jf", "Q", "T")}
    bl = {n: torch.from_numpy(v).cuda() for n, v in blocks.items()}
    eng = pf.PairF12("fp64", augment_somo=True)
    with pytest.raises(pf.Pf12Error) as ex:
        eng.upload_pairs_gather(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno,
                                wl.n_aux, bl, dict(off_orb=off, ext_pao=P, ext_aux=M, ext_ld=ld),
                                dict(map_pao=mp, map_aux=ma, off_map_pao=op, off_map_aux=oa),
                                dev, lay)
    assert ex.value.code == -7          # PF12_ERR_UNSUPPORTED
    eng.close()


def test_c40h81_augmented_sampled(built):
    """The C40H81 list in the augmented space, device-drawn inputs, one launch;
    sampled pairs (largest domains, SOMO pairs, random) against the oracle."""
    from synthetic import device
    wl = S.c40h81().augmented()
    t, lay = device.allocate(wl)
    device.fill(wl, t, lay)
    r, _ = _run(wl, "fp64", t=t, lay=lay)
    rm, _ = _run(wl, "mixed_fp32", t=t, lay=lay)
    assert (r["status"] == 0).all() and (rm["status"] == 0).all()
    somo = np.nonzero(wl.orb_kind == 1)[0]
    with_somo = np.nonzero(np.isin(wl.pi, somo) | np.isin(wl.pj, somo))[0]
    rng = np.random.default_rng(11)
    pairs = sorted({int(np.argmax(wl.n_aux)), int(np.argmax(wl.n_pno)), *map(int, with_somo[:4]),
                    *map(int, rng.choice(wl.n_pairs, 6, replace=False))})
    ref = O.run(wl, pairs=pairs)
    for n, P in enumerate(pairs):
        assert np.abs(r["e_pair"][P] - ref["e_pair"][n]).max() <= 1e-10, P
    sum_abs = float(np.abs(r["e_pair"].sum(axis=1)).sum())
    assert normalised_error(rm["E"] - r["E"], sum_abs, wl.n_orb) <= 1e-6
