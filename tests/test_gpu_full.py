"""Parity of the complete pair-energy kernel (pf12_upload_full / pf12_fit /
pf12_energy / pf12_full_terms, through the C ABI) with the FP64 oracle of
oracle/full_f12.py: every spatial term and every spin-case pair energy.

Bars: FP64 mode within 1e-10 Eh per pair energy, each term within 1e-11 of its
largest magnitude over the list; mixed mode within 1 uEh in total after the
chemical-scale normalisation (reading G1) and 1e-5 relative per pair (the
error model of the FP32 products, as in the amplitude-only path).
"""
import numpy as np
import pytest
import torch

import oracle.full_f12 as F
import synthetic as S
from gpu_helpers import normalised_error, sized_workload
from synthetic import full as FU

pytestmark = pytest.mark.gpu

EDGE_SIZES = [(1, 1, 1), (7, 7, 3), (5, 2, 33), (65, 64, 65), (130, 70, 129), (33, 33, 31),
              (90, 41, 190), (64, 64, 64), (40, 9, 300)]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _mini():
    return S.custom(5, 2, None, (40, 150), ("uniform", 1, 90), (30, 230), name="mini-ragged")


def _edge():
    return sized_workload(EDGE_SIZES, kinds=[0] * 7 + [1] * 3, diag_every=3, name="edge-sizes")


def _upload(wl, host=None):
    buf, lay = host if host is not None else FU.full_packed_inputs(wl)
    t = {n: torch.from_numpy(v).cuda() for n, v in buf.items()}
    return t, lay


def run_full(wl, precision, t=None, lay=None, variant=None):
    import paper_2008_03237_gb300 as pf
    if t is None:
        t, lay = _upload(wl)
    eng = pf.PairF12(precision, variant=variant)
    eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    E, e = eng.energy()
    terms = eng.full_terms().cpu().numpy()
    st = eng.pair_status()
    eng.close()
    return E, e.cpu().numpy(), terms, st


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("make", [S.tiny, _mini, _edge])
def test_full_fp64(built, make, variant):
    wl = make()
    ref = F.run(wl)
    E, e, terms, st = run_full(wl, "fp64", variant=variant)
    assert (st == 0).all()
    assert np.abs(e - ref["e_pair"]).max() <= 1e-10, np.abs(e - ref["e_pair"]).max()
    for q, name in enumerate(F.TERM_NAMES):
        scale = max(np.abs(ref["terms"][:, q]).max(), 1e-300)
        assert np.abs(terms[:, q] - ref["terms"][:, q]).max() <= 1e-11 * scale, name
    assert abs(E - ref["E"]) <= 1e-10 * max(1.0, abs(ref["E"]))


@pytest.mark.parametrize("make", [S.tiny, _mini, _edge])
def test_full_mixed(built, make):
    wl = make()
    ref = F.run(wl)
    E, e, terms, st = run_full(wl, "mixed_fp32")
    assert (st == 0).all()
    rel = np.abs(e - ref["e_pair"]).max() / np.abs(ref["e_pair"]).max()
    assert rel <= 1e-5, rel
    assert normalised_error(E - ref["E"], ref["sum_abs"], wl.n_orb) <= 1e-6


def test_full_canonical_limit(built):
    """The canonical inputs through the kernel: C vanishes and B~ follows the
    oracle (which a CPU pin ties to (2 f_v - eps_i - eps_j) X)."""
    wl = _mini()
    wl.meta["canonical"] = True
    ref = F.run(wl)
    _, e, terms, _ = run_full(wl, "fp64")
    assert np.abs(e - ref["e_pair"]).max() <= 1e-10
    names = list(F.TERM_NAMES)
    d = np.abs(terms[:, names.index("d")]).max()
    assert np.abs(terms[:, names.index("c_d")]).max() <= 1e-12 * d


def test_full_device_generator_bitwise(built):
    from synthetic import device
    for make in (_edge, _mini):
        wl = make()
        host, lay = FU.full_packed_inputs(wl)
        t, lay2 = device.allocate_full(wl)
        device.fill_full(wl, t, lay2)
        for n, v in host.items():
            assert np.array_equal(t[n].cpu().numpy()[:v.size], v), (wl.name, n)


def test_full_not_spd_pair_is_reported(built):
    import paper_2008_03237_gb300 as pf
    wl = S.tiny()
    host, lay = FU.full_packed_inputs(wl)
    bad = 5
    m = int(wl.n_aux[bad])
    o = lay["off_mm"][bad]
    host["Jg"][o:o + m * m].reshape(m, m)[...] -= 20.0 * np.eye(m)
    t, lay = _upload(wl, (host, lay))
    eng = pf.PairF12("fp64")
    eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    with pytest.raises(pf.Pf12Error) as ei:
        eng.energy()
    assert ei.value.code == -2
    st = eng.pair_status()
    assert st[bad] == 1 and (np.delete(st, bad) == 0).all()
    _, e = eng.energy(check=False)
    e = e.cpu().numpy()
    keep = [P for P in range(wl.n_pairs) if P != bad]
    ref = F.run(wl, pairs=keep)
    assert np.isnan(e[bad]).all()
    assert np.abs(np.delete(e, bad, axis=0) - ref["e_pair"]).max() <= 1e-10


def test_full_mode_refuses_what_it_does_not_offer(built):
    import paper_2008_03237_gb300 as pf
    wl = S.tiny()
    t, lay = _upload(wl)
    eng = pf.PairF12("fp64")
    eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    for call in (lambda: eng.build_v(), lambda: eng.backward(1.0, {})):
        with pytest.raises(pf.Pf12Error) as ei:
            call()
        assert ei.value.code == -7
    eng.close()
    eng = pf.PairF12("fp64", metric_packed=True)
    with pytest.raises(pf.Pf12Error) as ei:
        eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    assert ei.value.code == -7


def test_full_graph_replay_is_deterministic(built):
    import paper_2008_03237_gb300 as pf
    wl = _mini()
    t, lay = _upload(wl)
    eng = pf.PairF12("mixed_fp32")
    eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    E1, e1 = eng.energy()
    e1 = e1.cpu().numpy().copy()
    for _ in range(2):
        eng.fit()
        E2, e2 = eng.energy()
        assert E2 == E1 and np.array_equal(e2.cpu().numpy(), e1)
    assert eng.stats()["graph_used"] == 1


def test_full_c40h81_list_sampled_against_the_oracle(built):
    """The complete pair energy at the size bench.py times (the whole C40H81
    chain, device-drawn inputs, one persistent launch, mixed and FP64): sampled
    pairs one by one against the oracle (the largest and smallest domains,
    diagonal, SOMO and random pairs), properties over every pair, and the
    mixed total against FP64 on the chemical scale."""
    import paper_2008_03237_gb300 as pf
    from synthetic import device
    wl = S.c40h81()
    t, lay = device.allocate_full(wl)
    device.fill_full(wl, t, lay)
    out = {}
    for prec in ("fp64", "mixed_fp32"):
        eng = pf.PairF12(prec)
        eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
        eng.fit()
        E, e = eng.energy()
        out[prec] = (E, e.cpu().numpy(), eng.full_terms().cpu().numpy(), eng.pair_status())
        eng.close()
    del t
    E64, e64, tm64, st64 = out["fp64"]
    Emx, emx, _, stmx = out["mixed_fp32"]
    assert (st64 == 0).all() and (stmx == 0).all()
    assert np.isfinite(e64).all() and np.isfinite(emx).all()
    diag = wl.pi == wl.pj
    assert (e64[diag, 1:] == 0.0).all()
    somo = wl.orb_kind == 1
    ss = somo[wl.pi] & somo[wl.pj]
    assert (e64[ss, 0] == 0.0).all() and (e64[ss, 2] == 0.0).all()
    sd = somo[wl.pi] ^ somo[wl.pj]
    assert (e64[sd, 2] == 0.0).all()
    picks = {int(np.argmax(wl.n_aux)), int(np.argmin(wl.n_aux)), int(np.argmax(wl.n_pao)),
             int(np.argmax(wl.n_pno)), int(np.nonzero(diag)[0][7])}
    picks.update(int(x) for x in np.nonzero(somo[wl.pi] | somo[wl.pj])[0][:2])
    picks.update(int(x) for x in np.random.default_rng(5).choice(wl.n_pairs, 5, replace=False))
    picks = sorted(picks)
    ref = F.run(wl, pairs=picks)
    for q, P in enumerate(picks):
        assert np.abs(e64[P] - ref["e_pair"][q]).max() <= 1e-10, P
        scale = np.abs(ref["terms"][q]).max()
        assert np.abs(tm64[P] - ref["terms"][q]).max() <= 1e-11 * scale, P
        assert np.abs(emx[P] - ref["e_pair"][q]).max() <= 1e-5 * np.abs(ref["e_pair"][q]).max(), P
    sum_abs = float(np.abs(e64.sum(axis=1)).sum())
    assert normalised_error(Emx - E64, sum_abs, wl.n_orb) <= 1e-6


def test_full_streamed_batches_equal_single_pass(built, tmp_path):
    """The complete pair energy through the pair-streamed executor (batches
    drawn on a side stream while the previous one is evaluated): the same pair
    energies, bit for bit, as one resident launch."""
    from paper_2008_03237_gb300.stream import StreamedPairF12, full_input_bytes
    from synthetic import device
    wl = S.custom(6, 2, 4, (30, 90), ("uniform", 3, 40), (40, 160), name="full-stream-mini")
    t, lay = device.allocate_full(wl)
    device.fill_full(wl, t, lay)
    E1, e1, _, _ = run_full(wl, "fp64", t=t, lay=lay, variant=0)

    def produce(b, e, tb, lb):
        device.fill_full(wl.subset(np.arange(b, e)), tb, lb)
    budget = full_input_bytes(wl.n_pao, wl.n_pno, wl.n_aux).sum() / 4.5
    sp = StreamedPairF12("fp64", budget_bytes=budget, tuner_cache=str(tmp_path / "t.txt"),
                         full=True)
    E, e, st = sp.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, produce)
    assert len(sp.batches) >= 4 and (st == 0).all()
    assert np.array_equal(e.cpu().numpy(), e1)
    assert abs(E - E1) <= 1e-12 * np.abs(e1).sum()
