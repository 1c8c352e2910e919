"""Metrics as packed lower triangles (pf12_opts.metric_packed): the Cholesky
reads the same lower triangle and the J_f product the same values, so results
equal the full-block path bit for bit, forward and adjoint, in every variant."""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_helpers import sized_workload

pytestmark = pytest.mark.gpu

EDGE = [(1, 1, 1), (7, 7, 3), (5, 2, 33), (65, 64, 65), (130, 70, 129), (33, 33, 31),
        (90, 41, 190), (64, 64, 64), (128, 96, 300)]


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _lists():
    return [S.tiny(),
            S.custom(5, 2, None, (40, 150), ("uniform", 1, 90), (30, 230), name="mini"),
            sized_workload(EDGE, kinds=[0] * 7 + [1] * 3, diag_every=3, name="edge"),
            S.tiny().augmented()]


def _run(wl, precision, variant, packed, grads):
    import paper_2008_03237_gb300 as pf
    buf, lay = S.packed_inputs(wl, metric_packed=packed)
    t = {n: torch.from_numpy(np.concatenate([v, np.zeros(2)])).cuda() for n, v in buf.items()}
    eng = pf.PairF12(precision, variant=variant, metric_packed=packed,
                     augment_somo=bool(wl.somo_aug))
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    E, e = eng.energy()
    out = {"E": E, "e": e.cpu().numpy(), "V": eng.build_v().cpu().numpy()}
    if grads:
        g = {n: torch.zeros_like(t[n]) for n in ("Agi", "Agj", "Afi", "Afj", "Q", "T")}
        eng.backward(0.5, g)
        out["g"] = {n: v.cpu().numpy() for n, v in g.items()}
    torch.cuda.synchronize()
    eng.close()
    return out


@pytest.mark.parametrize("precision,variant", [("fp64", 0), ("fp64", 1), ("mixed_fp32", 1),
                                               ("mixed_fp32", 2)])
@pytest.mark.parametrize("idx", [0, 1, 2, 3], ids=["tiny", "mini", "edge", "tiny-aug"])
def test_packed_metrics_equal_full(built, precision, variant, idx):
    wl = _lists()[idx]
    grads = variant != 2
    full = _run(wl, precision, variant, False, grads)
    tri = _run(wl, precision, variant, True, grads)
    assert np.array_equal(full["e"], tri["e"]) and full["E"] == tri["E"]
    assert np.array_equal(full["V"], tri["V"])
    if grads:
        for n in full["g"]:
            assert np.array_equal(full["g"][n], tri["g"][n]), n


def test_packed_metrics_streamed(built):
    import paper_2008_03237_gb300 as pf
    from paper_2008_03237_gb300.stream import HostStreamer
    wl = _lists()[1]
    ref = _run(wl, "mixed_fp32", 1, False, False)
    buf, lay = S.packed_inputs(wl, metric_packed=True)
    host = {}
    for x, v in buf.items():
        h = torch.empty(max(v.size, 2), dtype=torch.float64, pin_memory=True)
        h[:v.size].copy_(torch.from_numpy(v))
        host[x] = h
    eng = pf.PairF12("mixed_fp32", variant=1, metric_packed=True)
    hs = HostStreamer(eng, 0.3e6, 2e6)
    for _ in range(2):
        E, e, st, ng = hs.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux,
                              host, lay)
        assert ng >= 4 and (st == 0).all()
        assert np.array_equal(e.cpu().numpy(), ref["e"]) and E == ref["E"]
    eng.close()
