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
