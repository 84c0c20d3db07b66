"""Host-side multi-GPU logic (one process per GPU).

The predicates have no exchange step: ciphertexts (and instances) are
independent, so ranks share nothing on their data path.  The one exchange is
an aggregate (COUNT / SUM) over a column split across ranks: each rank reduces
its share to one partial aggregate ciphertext, the partials are all-gathered,
and every rank adds them with the library's ciphertext sum (collectives have
no sum mod q).  Two layouts:
  * weak scaling: every rank processes its own batch of the same size (the
    benchmark; inputs drawn from a per-rank seed);
  * strong scaling of one batch: ciphertext range [start, end) per rank.
Timing takes the maximum over ranks (the job is done when the slowest rank is).
"""
from __future__ import annotations


def ct_shard(n_ct: int, world: int, rank: int):
    """Contiguous ciphertext range of `rank` when n_ct ciphertexts are split over
    `world` ranks as evenly as possible (the first n_ct % world ranks get one more)."""
    if world <= 0 or not 0 <= rank < world or n_ct < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_ct, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's own inputs under weak scaling (distinct per rank)."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allgather_partials(part, dist):
    """All ranks' partial aggregate ciphertexts in rank order, [world, *part.shape]
    (the part itself without a process group).  The caller adds them mod Q."""
    import torch

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return part.unsqueeze(0)
    parts = [torch.empty_like(part) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, part.contiguous())
    return torch.stack(parts)
