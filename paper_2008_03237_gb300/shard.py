"""Pair-list sharding across ranks (host logic of the multi-GPU path).

Pairs are independent, so ranks share no data: each rank evaluates its shard
and the pair energies meet once at the end.  Shards are built by longest-
processing-time assignment on the FP64 cost model m^3/3 + 4 k m^2 plus the
mixable part.  After the gather, every rank holds the full pair-energy array
in pair-list order and sums it on the host in that order (assemble), so that
total is bitwise the same for every number of ranks and every partition.  It
is not bitwise the total pf12_energy returns on one GPU, which adds the same
pair energies in a fixed tree order on the device; the two agree to rounding.
"""
import heapq

import numpy as np


def pair_costs(n_pao, n_pno, n_aux):
    p, k, m = (np.asarray(a, np.float64) for a in (n_pao, n_pno, n_aux))
    return m ** 3 / 3.0 + 4.0 * k * m * m + (8.0 * p * k * m + 2.0 * k * m * m + 4.0 * k * k * m) / 8.0


def lpt_partition(costs, n_ranks):
    """Deterministic LPT: pairs by decreasing cost (ties: list order) go to the
    least-loaded rank (ties: lowest rank).  Returns one sorted index array per rank."""
    order = np.argsort(-np.asarray(costs, np.float64), kind="stable")
    heap = [(0.0, r) for r in range(n_ranks)]
    out = [[] for _ in range(n_ranks)]
    for P in order:
        load, r = heapq.heappop(heap)
        out[r].append(int(P))
        heapq.heappush(heap, (load + float(costs[P]), r))
    return [np.array(sorted(s), np.int64) for s in out]


def evaluate_shard(wl, shard, tensors, offsets, precision="mixed_fp32", variant=None):
    """Device work of one rank: the pairs `shard` (indices into wl's list) of
    workload wl through the library, their inputs given as packed CUDA tensors
    of the shard alone (offsets: the shard's packed layout).  Returns the
    (len(shard) x 3) pair energies as a host array, in shard order."""
    from . import PairF12
    sub = wl.subset(shard)
    eng = PairF12(precision, variant=variant)
    try:
        eng.upload_pairs(sub.n_orb, sub.orb_kind, sub.pi, sub.pj, sub.n_pao, sub.n_pno, sub.n_aux,
                         tensors, offsets)
        eng.fit()
        _, e = eng.energy()
        return e.cpu().numpy()
    finally:
        eng.close()


def assemble(parts, n_pairs):
    """Full (n_pairs x 3) pair energies from (e_local, shard) parts, and their
    FP64 total summed on the host in pair-list order."""
    full = np.full((n_pairs, 3), np.nan)
    for e, idx in parts:
        full[np.asarray(idx, np.int64)] = np.asarray(e, np.float64).reshape(-1, 3)
    total = 0.0
    for P in range(n_pairs):
        total += full[P, 0] + full[P, 1] + full[P, 2]
    return full, total


def gather_pair_energies(e_local, shard, n_pairs, group=None):
    """All-gather every rank's (n_local x 3) pair energies into the full
    (n_pairs x 3) array in pair-list order, then the FP64 total summed in that
    order (assemble).  Works on the process group's backend: with NCCL the
    exchanged tensors live on the current CUDA device, with gloo on the host."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    e_local = torch.as_tensor(np.asarray(e_local, np.float64)).reshape(-1, 3)
    idx_local = torch.as_tensor(np.asarray(shard, np.int64))
    sizes = [None] * world
    dist.all_gather_object(sizes, int(idx_local.numel()), group=group)
    nmax = max(sizes)
    pad_e = torch.zeros((nmax, 3), dtype=torch.float64, device=dev)
    pad_i = torch.full((nmax,), -1, dtype=torch.int64, device=dev)
    pad_e[:e_local.shape[0]] = e_local.to(dev)
    pad_i[:idx_local.numel()] = idx_local.to(dev)
    all_e = [torch.zeros_like(pad_e) for _ in range(world)]
    all_i = [torch.zeros_like(pad_i) for _ in range(world)]
    dist.all_gather(all_e, pad_e, group=group)
    dist.all_gather(all_i, pad_i, group=group)
    parts = [(e[:n].cpu().numpy(), i[:n].cpu().numpy()) for e, i, n in zip(all_e, all_i, sizes)]
    return assemble(parts, n_pairs)


def reduce_orbital_gradients(blocks, group=None):
    """Sum every rank's per-orbital gradient blocks (gather-mode adjoint: each
    rank scatter-adds the pairs of its shard) and return the total on every
    rank.  The ranks' contributions are added in rank order after an
    all-gather, so the result is the same on every rank and reproducible for a
    given world size and partition."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    local = torch.as_tensor(np.ascontiguousarray(blocks, dtype=np.float64))
    parts = [torch.zeros_like(local) for _ in range(world)]
    dist.all_gather(parts, local, group=group)
    total = parts[0].clone()
    for r in range(1, world):
        total += parts[r]
    return total.numpy()
