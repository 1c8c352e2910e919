"""The LPT shard path of the multi-GPU design on one GPU: the list is split
with shard.lpt_partition, each shard is evaluated through the library on its
own inputs (as one rank would), and the parts are assembled in pair-list
order.  The ranks' kernels never wait on one another, so running them one
after the other on one GPU is the same device work as on several GPUs; the
NCCL exchange itself is covered by the gloo test on CPU."""
import numpy as np
import pytest

import synthetic as S
from paper_2008_03237_gb300.shard import assemble, evaluate_shard, lpt_partition, pair_costs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("world", [2, 3])
def test_lpt_shards_reassemble_the_single_gpu_result(built, world):
    from synthetic import device
    full = S.c40h81()
    wl = full.subset(np.arange(0, full.n_pairs, 5), name="C40H81-chain[every 5th pair]")
    t, lay = device.allocate(wl)
    device.fill(wl, t, lay)
    e_one = evaluate_shard(wl, np.arange(wl.n_pairs), t, lay, "mixed_fp32", variant=1)
    del t
    shards = lpt_partition(pair_costs(wl.n_pao, wl.n_pno, wl.n_aux), world)
    parts = []
    for mine in shards:
        sub = wl.subset(mine)
        ts, ls = device.allocate(sub)          # a rank holds its shard's inputs only
        device.fill(sub, ts, ls)
        parts.append((evaluate_shard(wl, mine, ts, ls, "mixed_fp32", variant=1), mine))
        del ts
    e_full, total = assemble(parts, wl.n_pairs)
    assert np.array_equal(e_full, e_one)       # pair by pair, bit for bit
    _, total_one = assemble([(e_one, np.arange(wl.n_pairs))], wl.n_pairs)
    assert total == total_one
