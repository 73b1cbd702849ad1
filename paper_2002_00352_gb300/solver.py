"""Iteration drivers over the C ABI: dual descent (Algorithm 2) and synchronous
coordinate descent (Algorithm 4), eager or replayed from a CUDA graph.

Each iteration is a fixed sequence of library calls on the current stream;
nothing here computes any part of the method.
"""
from __future__ import annotations

import torch

from . import kp


class IterStats:
    """Per-iteration device outputs: R [K], dual sum, primal sum (float64, on device)."""

    def __init__(self, K: int, device):
        self.R = torch.zeros(K, dtype=torch.float64, device=device)
        self.dual = torch.zeros((), dtype=torch.float64, device=device)
        self.primal = torch.zeros((), dtype=torch.float64, device=device)


def dd_step(prob, lam, alpha, lam_next, stats: IterStats = None):
    kp.kp_dd_step(prob, lam, alpha, lam_next, R=stats.R if stats else None)


def scd_step(prob, lam, lam_next, stats: IterStats = None):
    if stats is None:
        kp.kp_scd_step(prob, lam, lam_next)
    else:
        kp.kp_scd_step(prob, lam, lam_next, R=stats.R, dual_sum=stats.dual, primal_sum=stats.primal)


def scd_solve(prob, lam0: torch.Tensor, iters: int, record: bool = False):
    """Runs `iters` SCD iterations from lam0; returns the final lambda and, if
    `record`, the list of lambdas (host float64 tensors)."""
    a = lam0.clone()
    b = torch.empty_like(a)
    hist = [a.cpu()] if record else None
    for _ in range(iters):
        scd_step(prob, a, b)
        a, b = b, a
        if record:
            hist.append(a.cpu())
    return a, hist


def dd_solve(prob, lam0: torch.Tensor, alpha: float, iters: int, record: bool = False):
    a = lam0.clone()
    b = torch.empty_like(a)
    hist = [a.cpu()] if record else None
    for _ in range(iters):
        dd_step(prob, a, alpha, b)
        a, b = b, a
        if record:
            hist.append(a.cpu())
    return a, hist


def cd_solve(prob, lam0: torch.Tensor, blocks, record: bool = False):
    """Block coordinate descent (Sec. 4.3.2): one kp_bcd_step per entry of
    `blocks`, each a collection of knapsack indices updated together (cyclic CD:
    blocks = [[0], [1], ..., [K-1]] repeated; SCD: every block = all of them)."""
    a = lam0.clone()
    b = torch.empty_like(a)
    mask = torch.zeros(prob.K, dtype=torch.uint8, device=a.device)
    hist = [a.cpu()] if record else None
    for blk in blocks:
        mask.zero_()
        mask[torch.as_tensor(list(blk), dtype=torch.int64, device=a.device)] = 1
        kp.kp_bcd_step(prob, a, mask, b)
        a, b = b, a
        if record:
            hist.append(a.cpu())
    return a, hist


def cyclic_blocks(K: int, sweeps: int):
    """The blocks of cyclic CD: one multiplier at a time, k = 0..K-1, `sweeps` times."""
    return [[k] for _ in range(sweeps) for k in range(K)]


def presolve(prob, n: int, iters: int, seed: int = 0) -> torch.Tensor:
    """Sec. 5.3: lambda^0 from `iters` SCD iterations on about n users drawn
    uniformly (seeded; n draws, repeats dropped), budgets scaled by the sample's
    share of the users (kp_presolve)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    users = torch.unique(torch.randint(0, prob.N, (min(n, prob.N),), generator=g)).to("cuda")
    return kp.kp_presolve(prob, users, iters)


class ScdGraph:
    """Two SCD iterations (lambda_a -> lambda_b -> lambda_a) captured in one CUDA
    graph; replay() advances the state by two iterations with one launch."""

    def __init__(self, prob, lam0: torch.Tensor, stats: IterStats = None):
        self.prob = prob
        self.a = lam0.clone()
        self.b = torch.empty_like(self.a)
        self.stats = stats
        # kernel attributes were set when the handle was created, so capture
        # needs no warm-up launch (which would also advance the selection state)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            scd_step(prob, self.a, self.b, stats)
            scd_step(prob, self.b, self.a, stats)

    def replay(self):
        self.graph.replay()

    @property
    def lam(self):
        return self.a


class BatchScdGraph:
    """Two batched SCD iterations (every instance of a kp.Batch) captured in one CUDA
    graph; replay() advances all instances by two iterations with one launch."""

    def __init__(self, batch, lam0: torch.Tensor):
        self.batch = batch
        self.a = lam0.clone()
        self.b = torch.empty_like(self.a)
        torch.cuda.synchronize()  # kernel attributes were set when the batch was created
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            kp.kp_batch_scd_step(batch, self.a, self.b)
            kp.kp_batch_scd_step(batch, self.b, self.a)

    def replay(self):
        self.graph.replay()

    @property
    def lam(self):
        return self.a
