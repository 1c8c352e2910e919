"""Parity at the full workload sizes, in the launch configuration bench.py times
(device-drawn inputs, one persistent launch over the whole pair list).

The oracle evaluates a deterministic sample of pairs one by one (the largest
and smallest domains, diagonal, SOMO and random pairs); the rest is checked
through properties that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_helpers import grad_blocks, normalised_error

pytestmark = pytest.mark.gpu
GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden(name):
    """Oracle values of every pair, written by tests/golden/make_fullsize_oracle.py."""
    import os
    path = os.path.join(GOLDEN, f"{name}_oracle.npz")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    return np.load(path)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def _sample(wl, n_random, seed):
    somo = np.nonzero(wl.orb_kind == 1)[0]
    picks = {int(np.argmax(wl.n_aux)), int(np.argmin(wl.n_aux)), int(np.argmax(wl.n_pno)),
             int(np.argmin(wl.n_pno)), int(np.argmax(wl.n_pao)), int(np.argmin(wl.n_pao))}
    diag = np.nonzero(wl.pi == wl.pj)[0]
    picks.add(int(diag[len(diag) // 2]))
    with_somo = np.nonzero(np.isin(wl.pi, somo) | np.isin(wl.pj, somo))[0]
    picks.update(int(x) for x in with_somo[:3])
    rng = np.random.default_rng(seed)
    picks.update(int(x) for x in rng.choice(wl.n_pairs, n_random, replace=False))
    return sorted(picks)


def _device_inputs(wl):
    from synthetic import device
    t, lay = device.allocate(wl)
    device.fill(wl, t, lay)
    return t, lay


def _engine(wl, t, lay, precision):
    import paper_2008_03237_gb300 as pf
    eng = pf.PairF12(precision)
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    return eng


def _properties(wl, e_pair, E, status):
    assert (status == 0).all()
    assert np.isfinite(e_pair).all()
    # the fixed-order device total agrees with a compensated host sum
    assert abs(E - O.kahan_total(e_pair)) <= 1e-12 * np.abs(e_pair).sum()
    diag = wl.pi == wl.pj
    assert (e_pair[diag, 1:] == 0.0).all()          # no same-spin term on (ii)
    somo = wl.orb_kind == 1
    ss = somo[wl.pi] & somo[wl.pj]
    assert (e_pair[ss, 0] == 0.0).all() and (e_pair[ss, 2] == 0.0).all()
    sd = somo[wl.pi] ^ somo[wl.pj]
    assert (e_pair[sd, 2] == 0.0).all()


def test_c40h81_fp64_full_list(built):
    wl = S.c40h81()
    t, lay = _device_inputs(wl)
    eng = _engine(wl, t, lay, "fp64")
    E, e = eng.energy()
    e = e.cpu().numpy()
    _properties(wl, e, E, eng.pair_status())
    ref_all = _golden("c40h81")
    assert np.abs(e - ref_all["e_pair"]).max() <= 1e-10           # every pair against the oracle
    assert abs(E - float(ref_all["E"])) <= 1e-9
    V = eng.build_v().cpu().numpy()
    pairs = _sample(wl, 14, 1)
    ref = O.run(wl, pairs=pairs, want_V=True)
    for n, P in enumerate(pairs):
        assert np.abs(e[P] - ref["e_pair"][n]).max() <= 1e-10, P
        k = int(wl.n_pno[P])
        got = S.unpack(V, lay["off_kk"], P, k, k)
        assert np.abs(got - ref["V"][n]).max() <= 1e-11 * np.abs(ref["V"][n]).max(), P


def test_c40h81_backward_full_list(built):
    """Adjoint over the whole C40H81 list (FP64 and mixed), sampled pairs against
    the oracle gradient, mixed against FP64 everywhere."""
    wl = S.c40h81()
    t, lay = _device_inputs(wl)
    names = ("Agi", "Agj", "Afi", "Afj", "Q", "T")
    grads = {}
    for prec in ("fp64", "mixed_fp32"):
        eng = _engine(wl, t, lay, prec)
        g = {n: torch.zeros_like(t[n]) for n in names}
        eng.backward(1.0, g)
        torch.cuda.synchronize()
        assert (eng.pair_status() == 0).all()
        grads[prec] = {n: v.cpu().numpy() for n, v in g.items()}
        eng.close()
        del g
    pairs = _sample(wl, 6, 2)
    ref = O.run(wl, pairs=pairs, want_grad=True)
    for n, P in enumerate(pairs):
        got = grad_blocks(wl, lay, grads["fp64"], P)
        for name, want in ref["grads"][n].items():
            assert np.abs(got[name] - want).max() <= 1e-10 * np.abs(want).max(), (P, name)
    for name in names:
        a, b = grads["mixed_fp32"][name], grads["fp64"][name]
        assert np.abs(a - b).max() <= 2e-5 * np.abs(b).max(), name


def test_c160h321_mixed_full_list(built):
    """The bench workload: mixed precision over all 14,446 pairs; sampled pairs
    against the oracle; the normalised total error against the FP64 path."""
    wl = S.c160h321()
    t, lay = _device_inputs(wl)
    eng = _engine(wl, t, lay, "mixed_fp32")
    E, e = eng.energy()
    e = e.cpu().numpy()
    _properties(wl, e, E, eng.pair_status())
    eng.close()
    eng64 = _engine(wl, t, lay, "fp64")
    E64, e64 = eng64.energy()
    e64 = e64.cpu().numpy()
    eng64.close()
    pairs = _sample(wl, 6, 3)
    ref = O.run(wl, pairs=pairs)
    for n, P in enumerate(pairs):
        assert np.abs(e64[P] - ref["e_pair"][n]).max() <= 1e-10, P
        scale = np.abs(ref["e_pair"][n]).max()
        assert np.abs(e[P] - ref["e_pair"][n]).max() <= 1e-5 * scale, P
    sum_abs = float(np.abs(e64.sum(axis=1)).sum())
    assert normalised_error(E - E64, sum_abs, wl.n_orb) <= 1e-6
    ref_all = _golden("c160h321")
    assert np.abs(e64 - ref_all["e_pair"]).max() <= 1e-10         # FP64 path, every pair
    assert normalised_error(E - float(ref_all["E"]), float(ref_all["sum_abs"]), wl.n_orb) <= 1e-6
