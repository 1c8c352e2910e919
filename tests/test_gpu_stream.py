"""Pair-streamed execution: batches through reused device buffers.

The lattice quartet (703 orbitals, 29,226 pairs, ~819 GB of FP64 inputs) runs
mixed forward plus adjoint inside a 180 GB device budget."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_helpers import run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _producer(wl):
    from synthetic import device

    def produce(b, e, t, lay):
        device.fill(wl.subset(np.arange(b, e)), t, lay)
    return produce


def test_streamed_batches_equal_single_pass(built, tmp_path):
    from paper_2008_03237_gb300.stream import StreamedPairF12, input_bytes
    wl = S.custom(6, 2, 4, (30, 90), ("uniform", 3, 40), (40, 160), name="stream-mini")
    one = run(wl, "fp64", want_V=False)
    budget = input_bytes(wl.n_pao, wl.n_pno, wl.n_aux).sum() / 4.5
    sp = StreamedPairF12("fp64", budget_bytes=budget, tuner_cache=str(tmp_path / "tune.txt"))
    E, e, st = sp.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, _producer(wl))
    assert len(sp.batches) >= 4
    assert (st == 0).all()
    assert np.array_equal(e.cpu().numpy(), one["e_pair"])
    assert abs(E - one["E"]) <= 1e-12 * np.abs(one["e_pair"]).sum()


def test_lattice_quartet_streamed_mixed_with_backward(built, tmp_path):
    from paper_2008_03237_gb300.stream import StreamedPairF12
    wl = S.lattice_quartet()
    somo = np.nonzero(wl.orb_kind == 1)[0]
    rng = np.random.default_rng(4)
    picks = sorted({int(np.argmax(wl.n_aux)), int(np.argmax(wl.n_pno)),
                    int(np.nonzero(np.isin(wl.pi, somo) & np.isin(wl.pj, somo))[0][0]),
                    *[int(x) for x in rng.choice(wl.n_pairs, 3, replace=False)]})
    kept = {}
    torch.cuda.synchronize()
    torch.cuda.empty_cache()          # memory cached by earlier tests is not this run's
    free0, total = torch.cuda.mem_get_info()
    base = total - free0
    peak = [0]

    def consume(b, e, g, lay):
        peak[0] = max(peak[0], total - torch.cuda.mem_get_info()[0])
        for P in picks:
            if b <= P < e:
                q = P - b
                p_, k_, m_ = int(wl.n_pao[P]), int(wl.n_pno[P]), int(wl.n_aux[P])
                blk = {}
                for n in ("Agi", "Agj", "Afi", "Afj"):
                    o = int(lay["off_pm"][q])
                    blk[n] = g[n][o:o + p_ * m_].cpu().numpy().reshape(p_, m_)
                o = int(lay["off_pk"][q])
                blk["Q"] = g["Q"][o:o + p_ * k_].cpu().numpy().reshape(p_, k_)
                o = int(lay["off_kk"][q])
                blk["T"] = g["T"][o:o + k_ * k_].cpu().numpy().reshape(k_, k_)
                kept[P] = blk
    sp = StreamedPairF12("mixed_fp32", budget_bytes=40e9, tuner_cache=str(tmp_path / "tune.txt"))
    E, e, st = sp.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux,
                      _producer(wl), backward=True, grad_consumer=consume)
    assert (st == 0).all()
    assert peak[0] - base <= 180e9, (peak[0], base)
    e = e.cpu().numpy()
    assert np.isfinite(e).all()
    ref = O.run(wl, pairs=picks, want_grad=True)
    for n, P in enumerate(picks):
        assert np.abs(e[P] - ref["e_pair"][n]).max() <= 1e-5 * np.abs(ref["e_pair"][n]).max(), P
        for name, want in ref["grads"][n].items():
            assert np.abs(kept[P][name] - want).max() <= 2e-5 * np.abs(want).max(), (P, name)


def test_host_pipelined_equals_resident(built, tmp_path):
    """Inputs in pinned host memory, copied batch by batch on a second stream
    while the previous batch is fitted: same pair energies as the resident run."""
    import paper_2008_03237_gb300 as pf
    from paper_2008_03237_gb300.stream import input_bytes, run_from_host
    wl = S.custom(6, 2, 4, (30, 90), ("uniform", 3, 40), (40, 160), name="e2e-mini")
    host, lay = S.packed_inputs(wl)
    one = run(wl, "fp64", want_V=False)
    pinned = {n: torch.from_numpy(v).pin_memory() for n, v in host.items()}
    budget = input_bytes(wl.n_pao, wl.n_pno, wl.n_aux).sum() / 3.5
    E, e, st, nb = run_from_host(pf.PairF12("fp64", tuner_cache=str(tmp_path / "t.txt")),
                                 wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux,
                                 pinned, lay, budget)
    assert nb >= 3 and (st == 0).all()
    assert np.array_equal(e.cpu().numpy(), one["e_pair"])
    assert abs(E - one["E"]) <= 1e-12 * np.abs(one["e_pair"]).sum()


def test_streamed_run_resumes_after_a_failed_batch(built, tmp_path):
    """Failure injected on the host: the producer of the third batch raises.
    The resume record keeps the finished batches; a second run with the same
    record produces and evaluates only the rest and returns the uninterrupted
    result bit for bit."""
    from paper_2008_03237_gb300.stream import StreamedPairF12, input_bytes
    wl = S.custom(6, 2, 4, (30, 90), ("uniform", 3, 40), (40, 160), name="stream-resume")
    budget = input_bytes(wl.n_pao, wl.n_pno, wl.n_aux).sum() / 4.5
    args = (wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux)
    ref = StreamedPairF12("fp64", budget_bytes=budget)
    E_ref, e_ref, _ = ref.run(*args, _producer(wl))
    e_ref = e_ref.cpu().numpy().copy()
    ck = str(tmp_path / "resume.npz")
    good = _producer(wl)
    calls = []

    def failing(b, e, t, lay):
        if len(calls) == 2:
            raise RuntimeError("injected producer failure")
        calls.append((b, e))
        good(b, e, t, lay)
    sp = StreamedPairF12("fp64", budget_bytes=budget)
    with pytest.raises(RuntimeError, match="injected"):
        sp.run(*args, failing, checkpoint=ck)
    again = []

    def counting(b, e, t, lay):
        again.append((b, e))
        good(b, e, t, lay)
    sp2 = StreamedPairF12("fp64", budget_bytes=budget)
    E, e, st = sp2.run(*args, counting, checkpoint=ck)
    assert sp2.resumed == 2 and len(again) == len(sp2.batches) - 2
    assert (st == 0).all()
    assert np.array_equal(e.cpu().numpy(), e_ref) and E == E_ref
