"""Categorical (bounded non-negative integer) decision variables (Sec. 2).

The paper notes that its method applies unchanged to x_ij in {0, 1, ..., u_j}:
the objective and every constraint are linear in x_ij and the local
constraints count it, so x_ij is the sum of u_j binary copies of item j, each
with the profit p_ij and the consumption b_ijk of the original and each in the
local sets that hold j.  Copies of an item tie in every reduced cost, and
Algorithm 1 breaks ties by the lower index, so the greedy takes the copies in
order.  This module builds that binary instance (a change of layout, no step
of the method) and folds binary decisions back into integer ones; the library
then solves the expanded instance as any other.
"""
from __future__ import annotations

from typing import Sequence

import torch

from .gen import Instance


def expand_categorical(inst: Instance, ubound: Sequence[int]) -> Instance:
    """Binary instance of `inst` with item j repeated ubound[j] >= 1 times (copies
    of one item consecutive, items in order); sum(ubound) <= 64."""
    u = [int(v) for v in ubound]
    if len(u) != inst.M or min(u) < 1:
        raise ValueError("ubound needs one bound >= 1 per item")
    M2 = sum(u)
    if M2 > 64:
        raise ValueError("the expanded instance has more than 64 items")
    dev = inst.p.device
    src = torch.repeat_interleave(torch.arange(inst.M, device=dev), torch.tensor(u, device=dev))  # [M2]
    N, M, K = inst.N, inst.M, inst.K
    p2 = inst.p.view(N, M)[:, src].contiguous().view(-1)
    first = [sum(u[:j]) for j in range(M)]
    S2 = []
    for s in inst.S:
        m = 0
        for j in range(M):
            if (s >> j) & 1:
                m |= ((1 << u[j]) - 1) << first[j]
        S2.append(m)
    kw = dict(name=inst.name + "_categorical", N=N, M=M2, K=K, layout=inst.layout, p=p2, B=inst.B,
              S=S2, C=list(inst.C), seed=inst.seed, recipe=inst.recipe + "; categorical copies " + str(u))
    if inst.layout == "dense":
        b2 = inst.b.view(N, M, K)[:, src, :].contiguous().view(-1)
        return Instance(b=b2, **kw)
    # CSR: every copy owns its original's entries
    cnt = inst.item_nnz.view(N, M).long()
    cnt2 = cnt[:, src]                                            # [N, M2]
    start = (torch.cumsum(cnt, 1) - cnt) + inst.user_off[:N, None] - inst.user_off[0]
    start2 = start[:, src]
    tot2 = cnt2.sum(1)
    off2 = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    off2[1:] = torch.cumsum(tot2, 0)
    n2 = int(off2[-1])
    owner = torch.repeat_interleave(torch.arange(N * M2, device=dev), cnt2.reshape(-1))
    rank = torch.arange(n2, device=dev) - torch.repeat_interleave(
        torch.cumsum(cnt2.reshape(-1), 0) - cnt2.reshape(-1), cnt2.reshape(-1))
    ent = start2.reshape(-1)[owner] + rank + inst.user_off[0]
    return Instance(user_off=off2, item_nnz=cnt2.to(torch.uint8).reshape(-1).contiguous(),
                    val=inst.val[ent].contiguous(), kidx=inst.kidx[ent].contiguous(), **kw)


def fold_decisions(x2: torch.Tensor, ubound: Sequence[int]) -> torch.Tensor:
    """Integer decisions [N, M] from the expanded instance's binary decisions [N, sum(ubound)]."""
    u = torch.tensor([int(v) for v in ubound], device=x2.device)
    grp = torch.repeat_interleave(torch.arange(len(u), device=x2.device), u)
    out = torch.zeros(x2.shape[0], len(u), dtype=torch.int64, device=x2.device)
    out.index_add_(1, grp, x2.long())
    return out
