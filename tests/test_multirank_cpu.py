"""Multi-rank path on CPU: world-size-2 gloo ranks shard the pair list by LPT,
evaluate their shards (the oracle stands in for the per-rank device work) and
gather; the total must equal the single-rank total bit for bit."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle as O
import synthetic as S
from paper_2008_03237_gb300.shard import lpt_partition, pair_costs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2008_03237_gb300.shard import gather_pair_energies
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = S.tiny()
    shards = lpt_partition(pair_costs(wl.n_pao, wl.n_pno, wl.n_aux), world)
    mine = shards[rank]
    r = O.run(wl, pairs=list(mine))
    full, total = gather_pair_energies(r["e_pair"], mine, wl.n_pairs)
    out[rank] = (full.tolist(), total)
    dist.destroy_process_group()


def test_lpt_partition_properties():
    costs = np.array([5.0, 1.0, 4.0, 4.0, 2.0, 9.0, 3.0])
    shards = lpt_partition(costs, 3)
    flat = np.sort(np.concatenate(shards))
    assert np.array_equal(flat, np.arange(len(costs)))
    loads = [costs[s].sum() for s in shards]
    assert max(loads) - min(loads) <= costs.max()
    assert [list(s) for s in lpt_partition(costs, 3)] == [list(s) for s in shards]


def test_two_gloo_ranks_match_single_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    ref = O.run(S.tiny())
    for r in range(2):
        full, total = out[r]
        assert np.array_equal(np.array(full), ref["e_pair"])
        assert total == ref["E"]


def _scatter_orbital(gw, pairs, grads, layout, maps):
    """Host scatter-add of per-pair factor gradients into orbital blocks, pair order."""
    P_o, M_o, ld, off, total = layout
    mp, ma, op, oa = maps
    wl = gw.base
    out = np.zeros((2, max(total, 2)))
    for q, g in zip(pairs, grads):
        p_, m_ = int(wl.n_pao[q]), int(wl.n_aux[q])
        for side, o in enumerate((int(wl.pi[q]), int(wl.pj[q]))):
            rows = mp[op[q] + side * p_: op[q] + (side + 1) * p_]
            cols = ma[oa[q] + side * m_: oa[q] + (side + 1) * m_]
            for b, key in enumerate(("Agi", "Afi") if side == 0 else ("Agj", "Afj")):
                blk = out[b][off[o]:off[o] + P_o[o] * ld[o]].reshape(P_o[o], ld[o])
                blk[np.ix_(rows, cols)] += g[key]
    return out


def _rank_grad(rank, world, port, out):
    import torch.distributed as dist
    from synthetic import gather as G
    from paper_2008_03237_gb300.shard import reduce_orbital_gradients
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    gw = G.make_gather(S.custom(4, 1, 2, (10, 20), ("uniform", 2, 10), (10, 20), name="mr-gather"))
    wl = gw.base
    shards = lpt_partition(pair_costs(wl.n_pao, wl.n_pno, wl.n_aux), world)
    mine = list(shards[rank])
    r = O.run(wl, pairs=mine, inputs=lambda q: G.pair_inputs(gw, q), want_grad=True)
    local = _scatter_orbital(gw, mine, r["grads"], G.orbital_layout(gw), G.pair_maps(gw))
    out[rank] = reduce_orbital_gradients(local).tolist()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_orbital_gradients():
    """Gather-mode adjoint across ranks: per-orbital gradient blocks of two
    shards summed in rank order equal the single-rank blocks (to rounding) and
    are identical on both ranks."""
    from synthetic import gather as G
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_grad, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    gw = G.make_gather(S.custom(4, 1, 2, (10, 20), ("uniform", 2, 10), (10, 20), name="mr-gather"))
    allp = list(range(gw.n_pairs))
    ref = O.run(gw.base, pairs=allp, inputs=lambda q: G.pair_inputs(gw, q), want_grad=True)
    want = _scatter_orbital(gw, allp, ref["grads"], G.orbital_layout(gw), G.pair_maps(gw))
    a, b = np.array(out[0]), np.array(out[1])
    assert np.array_equal(a, b)
    assert np.abs(a - want).max() <= 1e-12 * np.abs(want).max()
