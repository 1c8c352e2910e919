"""Streamed inputs (pf12_set_arrival / HostStreamer): one persistent launch
whose CTAs wait for each group's arrival flag while the host-to-device copies
of later groups are still running.

- Results equal the resident path bit for bit (each pair's arithmetic does not
  depend on the queue order; the total is summed in list order), on three
  calls in a row with different data, so stale device buffers would show; with
  groups spread over three copy streams they may also land out of order.
- A flag that nothing writes makes the bounded wait expire: status 3 and
  PF12_ERR_TIMEOUT, and the context works again after a new upload.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_helpers import run, upload_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _pinned(wl):
    buf, lay = S.packed_inputs(wl)
    host = {}
    for x, v in buf.items():
        h = torch.empty(max(v.size, 2), dtype=torch.float64, pin_memory=True)
        h[:v.size].copy_(torch.from_numpy(v))
        host[x] = h
    return host, lay


def _lists():
    """Two lists with the same sizes and different drawn values."""
    import dataclasses
    a = S.custom(7, 2, 5, (30, 120), ("uniform", 3, 40), (40, 220), name="arrival-a")
    b = dataclasses.replace(a, seed=a.seed + 77, name="arrival-b")
    return a, b


@pytest.mark.parametrize("precision,variant,streams", [("fp64", 1, 1), ("mixed_fp32", None, 1),
                                                       ("mixed_fp32", 2, 1), ("fp64", 0, 3)])
def test_streamed_equals_resident(built, precision, variant, streams):
    import paper_2008_03237_gb300 as pf
    from paper_2008_03237_gb300.stream import HostStreamer, arrival_groups
    wla, wlb = _lists()
    assert np.array_equal(wla.n_pao, wlb.n_pao) and not np.array_equal(
        S.pair_inputs(wla, 3)["Agi"], S.pair_inputs(wlb, 3)["Agi"])
    eng = pf.PairF12(precision, variant=variant)
    # small groups: many waits inside one launch
    hs = HostStreamer(eng, first_bytes=0.5e6, max_group_bytes=3e6, copy_streams=streams)
    ends = arrival_groups(wla.n_pao, wla.n_pno, wla.n_aux, 0.5e6, 3e6)
    assert len(ends) >= 8
    for wl in (wla, wlb, wla):
        host, lay = _pinned(wl)
        ref = run(wl, precision, want_V=False, variant=variant)
        E, e, st, ng = hs.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux,
                              host, lay)
        assert ng == len(ends)
        assert (st == 0).all()
        assert np.array_equal(e.cpu().numpy(), ref["e_pair"]), wl.name
        assert E == ref["E"], wl.name
    eng.close()


def test_streamed_augmented(built):
    import paper_2008_03237_gb300 as pf
    from paper_2008_03237_gb300.stream import HostStreamer
    wl = _lists()[0].augmented()
    host, lay = _pinned(wl)
    t, _ = upload_host(wl)
    ref_eng = pf.PairF12("fp64", augment_somo=True)
    ref_eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    ref_eng.fit()
    E_ref, e_ref = ref_eng.energy()
    eng = pf.PairF12("fp64", augment_somo=True)
    E, e, st, ng = HostStreamer(eng, 0.5e6, 3e6).run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao,
                                                   wl.n_pno, wl.n_aux, host, lay)
    assert ng >= 8 and (st == 0).all()
    assert np.array_equal(e.cpu().numpy(), e_ref.cpu().numpy()) and E == E_ref


def test_arrival_wait_expires_and_context_recovers(built):
    import paper_2008_03237_gb300 as pf
    wl = _lists()[0]
    t, lay = upload_host(wl)
    eng = pf.PairF12("fp64", variant=1, debug_wait_timeout=True)
    args = (wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.upload_pairs(*args)
    ready = torch.zeros(2, dtype=torch.int32, device="cuda")   # nothing ever writes these
    eng.set_arrival([wl.n_pairs // 2, wl.n_pairs], ready, 5)
    eng.fit()
    with pytest.raises(pf.Pf12Error) as ex:
        eng.energy()
    assert ex.value.code == -5                                  # PF12_ERR_TIMEOUT
    assert (eng.pair_status() == 3).any()
    # a new upload clears the stop flag and the arrival setting
    eng.upload_pairs(*args)
    eng.fit()
    E, e = eng.energy()
    ref = run(wl, "fp64", want_V=False, variant=1)
    assert np.array_equal(e.cpu().numpy(), ref["e_pair"]) and E == ref["E"]
    eng.close()


def test_set_arrival_rejects_bad_groups(built):
    import paper_2008_03237_gb300 as pf
    wl = _lists()[0]
    t, lay = upload_host(wl)
    eng = pf.PairF12("fp64")
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    ready = torch.zeros(4, dtype=torch.int32, device="cuda")
    n = wl.n_pairs
    for ends in ([n // 2, n // 2, n], [n // 2], [0, n], [n // 2, n + 1]):
        with pytest.raises(pf.Pf12Error) as ex:
            eng.set_arrival(ends, ready, 1)
        assert ex.value.code == -1, ends
    # turning streaming on and off again leaves a normal fit
    eng.set_arrival([n // 3, n], ready, 1)
    eng.set_arrival([], ready, 0)
    eng.fit()
    E, e = eng.energy()
    ref = run(wl, "fp64", want_V=False)
    assert np.array_equal(e.cpu().numpy(), ref["e_pair"])
    eng.close()
