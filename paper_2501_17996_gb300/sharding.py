"""Multi-rank pieces of the path (host side).

1. Replicas (what ``bench.py --gpus N`` runs): every rank solves its own instance; the job's
   rate is (units processed on all ranks) / (slowest rank's time), a MAX all-reduce.

2. Destination-row sharding of one instance (the decomposition a multi-GPU solve of a single
   large instance would use). Rows i of F, Y, T and W are split across ranks: Y A and
   F A^T act row by row, so the edge gather and the node prox stay local; the only coupling
   is the capped-simplex projection of each edge column (Sec. 2.3), whose multiplier mu_l
   depends on all n destinations. The Newton iteration on
   phi(mu) = sum_i (q_il - mu)_+ - c_l needs, per step, the column sums of q over the active
   set and their counts: one SUM all-reduce of 2m values per step. This module implements
   that protocol with torch.distributed on tensors (gloo on the CPU in the tests); each
   rank ends with exactly the unsharded multipliers because every rank applies the same
   arithmetic to the same all-reduced sums.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def aggregate_rate(units_local: float, seconds_local: float, world: int, device=None) -> tuple:
    """Returns (job rate, slowest time): sum of units over ranks / max of times."""
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def row_shard(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous destination rows [lo, hi) of this rank."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def sharded_mu(q_local: torch.Tensor, c: torch.Tensor, max_steps: int = 64) -> torch.Tensor:
    """Multipliers of the capped-simplex projection of the m columns of Q, whose rows are
    split across the ranks (q_local: this rank's rows, shape [rows, m], float64).

    Newton from the left on phi(mu) (mu starts at 0): mu <- (S - c)/C with S, C the sums and
    counts over {q > mu}, all-reduced; a column is finished once its count stops changing
    (the active set is fixed, so mu is exact), or mu = 0 when sum (q)_+ <= c."""
    m = q_local.shape[1]
    mu = torch.zeros(m, dtype=q_local.dtype)
    active = torch.ones(m, dtype=torch.bool)
    prev_cnt = torch.full((m,), -1.0, dtype=q_local.dtype)
    for _ in range(max_steps):
        mask = q_local > mu.unsqueeze(0)
        sc = torch.stack([(q_local * mask).sum(dim=0), mask.sum(dim=0).to(q_local.dtype)])
        if dist.is_initialized() and dist.get_world_size() > 1:
            dist.all_reduce(sc, op=dist.ReduceOp.SUM)
        s, cnt = sc[0], sc[1]
        first = prev_cnt < 0
        # mu = 0 columns: sum of positive parts within capacity
        zero = first & (s <= c)
        active &= ~zero
        done = (~first) & (cnt == prev_cnt)
        active &= ~done
        if not bool(active.any()):
            break
        new_mu = torch.where(active & (cnt > 0), (s - c) / torch.clamp(cnt, min=1.0), mu)
        mu = torch.where(active, torch.maximum(new_mu, mu), mu)
        prev_cnt = torch.where(active, cnt, prev_cnt)
    return mu
