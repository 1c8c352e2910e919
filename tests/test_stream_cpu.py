"""Host logic of the pair-streamed executor: packed layout and batch plan."""
import numpy as np
import pytest

import synthetic as S
from paper_2008_03237_gb300.stream import input_bytes, packed_layout, plan_batches


def test_packed_layout_matches_generator_layout():
    wl = S.custom(6, 1, 3, (10, 50), ("uniform", 2, 9), (5, 70))
    a = packed_layout(wl.n_pao, wl.n_pno, wl.n_aux)
    b = S.packed_offsets(wl)
    for key in a:
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
    assert all(int(o) % 32 == 0 for key in ("off_pm", "off_mm", "off_pk", "off_kk") for o in a[key])


def test_plan_batches_covers_list_within_budget():
    wl = S.lattice_quartet()
    per = input_bytes(wl.n_pao, wl.n_pno, wl.n_aux)
    budget = 40e9
    batches = plan_batches(wl.n_pao, wl.n_pno, wl.n_aux, budget)
    assert batches[0][0] == 0 and batches[-1][1] == wl.n_pairs
    for (b0, e0), (b1, _) in zip(batches, batches[1:]):
        assert e0 == b1
    for b, e in batches:
        assert per[b:e].sum() <= budget
    assert per.sum() > 800e9 and len(batches) >= 20
    with pytest.raises(ValueError):
        plan_batches(wl.n_pao, wl.n_pno, wl.n_aux, per.max() / 2)


def test_arrival_groups_cover_the_list_and_grow():
    from paper_2008_03237_gb300.stream import arrival_groups
    wl = S.c160h321()
    per = input_bytes(wl.n_pao, wl.n_pno, wl.n_aux)
    ends = arrival_groups(wl.n_pao, wl.n_pno, wl.n_aux, 0.5e9, 4e9)
    assert ends[-1] == wl.n_pairs and (np.diff(ends) > 0).all() and ends[0] > 0
    starts = np.concatenate([[0], ends[:-1]])
    sizes = np.array([per[b:e].sum() for b, e in zip(starts, ends)])
    assert sizes[0] <= 0.5e9 + per.max()
    assert sizes[:-1].max() <= 4e9 + per.max()
    # doubling until the cap: few groups for 178 GB
    assert 40 <= len(ends) <= 60
    assert arrival_groups([], [], [], 1e9, 4e9).size == 0
    one = arrival_groups(wl.n_pao[:1], wl.n_pno[:1], wl.n_aux[:1], 1.0, 1.0)
    assert list(one) == [1]


def test_packed_metric_layout():
    """Metrics as packed lower triangles: block sizes m (m + 1) / 2 and row r of
    the triangle at r (r + 1) / 2."""
    wl = S.custom(3, 1, None, (5, 9), ("uniform", 2, 4), (4, 11))
    full, lay_f = S.packed_inputs(wl)
    tri, lay_t = S.packed_inputs(wl, metric_packed=True)
    for P in range(wl.n_pairs):
        m = int(wl.n_aux[P])
        J = S.unpack(full["Jg"], lay_f["off_mm"], P, m, m)
        o = int(lay_t["off_mm"][P])
        for r in range(m):
            row = tri["Jg"][o + r * (r + 1) // 2: o + r * (r + 1) // 2 + r + 1]
            assert np.array_equal(row, J[r, :r + 1])
        assert lay_t["off_mm"][P] % 32 == 0
    m = wl.n_aux.astype(np.int64)
    assert lay_t["len_mm"] == int(((m * (m + 1) // 2 + 31) // 32 * 32).sum())
    for key in ("off_pm", "off_pk", "off_kk"):
        assert np.array_equal(lay_t[key], lay_f[key])


def test_resume_record_round_trip_and_plan_check(tmp_path):
    """The batch-level resume record (the checkpoint of a streamed run): what a
    run commits is what the next run reads back, and a record of another batch
    plan is ignored."""
    from paper_2008_03237_gb300.stream import ResumeRecord
    path = str(tmp_path / "rec.npz")
    batches = [(0, 3), (3, 7), (7, 10)]
    rec = ResumeRecord.open(path, batches, 10)
    assert not rec.done.any()
    rng = np.random.default_rng(1)
    e1 = rng.standard_normal((4, 3))
    rec.commit(1, 2.5, e1, np.array([0, 0, 1, 0], np.int32))
    back = ResumeRecord.open(path, batches, 10)
    assert list(back.done) == [False, True, False]
    assert back.totals[1] == 2.5 and np.array_equal(back.e_pair[3:7], e1)
    assert list(back.status[3:7]) == [0, 0, 1, 0]
    other = ResumeRecord.open(path, [(0, 5), (5, 10)], 10)     # another plan: start afresh
    assert not other.done.any()
    assert not ResumeRecord.open(path, batches, 11).done.any()


def test_full_layout_matches_the_generator_layout():
    """The executor's complete-pair-energy layout is the generator's (and the
    C ABI's pf12_full_tensors layout)."""
    from paper_2008_03237_gb300.stream import full_input_bytes, full_packed_layout
    from synthetic.full import full_offsets
    wl = S.custom(6, 1, 3, (10, 50), ("uniform", 2, 9), (5, 70))
    a = full_packed_layout(wl.n_pao, wl.n_pno, wl.n_aux)
    b = full_offsets(wl)
    for key in b:
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
    p, k, m = (wl.n_pao.astype(float), wl.n_pno.astype(float), wl.n_aux.astype(float))
    lens = 8.0 * (10 * (p + 2) * m + 3 * m * m + p * k + k * k + p * p + 2 * k + k * m * (k + 2))
    assert np.allclose(full_input_bytes(wl.n_pao, wl.n_pno, wl.n_aux), lens)
