"""Seeded synthetic knapsack instances (inputs only; none of the method's arithmetic).

The paper's experiments use synthetic instances (Sec. 6: p_ij ~ U[0,1], b_ijk ~
U[0,1], dense or sparse global constraints, budgets scaled so that the
constraints are tight, hierarchical local constraints such as C=[2,2,3]).
The workloads below follow that recipe at the shapes this library is measured
on; every array is drawn from a torch.Generator seeded with ``seed`` on the
requested device, so the same call gives the same instance on every run.

Both the CUDA path and the CPU oracle consume what this module produces; it
contains no step of the solver itself.

Storage:
  p          float32 [N*M]                 profit p_ij, row-major by user
  dense b    float32 [N*M*K]               b_ijk with k fastest
  CSR b      user_off int64 [N+1]          first entry of user i
             item_nnz uint8  [N*M]         entries owned by item (i, j)
             val      float32 [nnz]        b_ijk of the entry
             kidx     int16   [nnz]        k of the entry, strictly increasing
                                           within an item
  B          float64 [K]                   budgets
  S, C       L item-set bitmasks and caps (hierarchical local constraints,
             shared by all users)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch


@dataclass
class Instance:
    name: str
    N: int
    M: int
    K: int
    layout: str                      # "dense" | "csr"
    p: torch.Tensor
    B: torch.Tensor
    S: List[int]
    C: List[int]
    b: Optional[torch.Tensor] = None
    user_off: Optional[torch.Tensor] = None
    item_nnz: Optional[torch.Tensor] = None
    val: Optional[torch.Tensor] = None
    kidx: Optional[torch.Tensor] = None
    seed: int = 0
    recipe: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def device(self):
        return self.p.device

    def nbytes(self) -> int:
        t = [self.p, self.b, self.user_off, self.item_nnz, self.val, self.kidx]
        return sum(x.numel() * x.element_size() for x in t if x is not None)

    def users_dense(self, idx) -> tuple:
        """(p [n, M], b [n, M, K]) as float64 numpy arrays for the given users."""
        dev = self.p.device
        idx = torch.as_tensor(np.asarray(idx, dtype=np.int64), device=dev)
        M, K = self.M, self.K
        n = idx.numel()
        p = self.p.view(self.N, M)[idx].double().cpu().numpy()
        if self.layout == "dense":
            b = self.b.view(self.N, M, K)[idx].double().cpu().numpy()
            return p, b
        # gather the users' CSR entries (layout conversion only)
        starts = self.user_off[idx]
        cnt = self.item_nnz.view(self.N, M)[idx].long()          # [n, M]
        tot = cnt.sum(1)                                          # [n]
        nent = int(tot.sum())
        b = torch.zeros(n * M, K, dtype=torch.float64, device=dev)
        if nent:
            base = torch.repeat_interleave(starts, tot)
            first = torch.repeat_interleave(torch.cumsum(tot, 0) - tot, tot)
            ent = base + (torch.arange(nent, device=dev) - first)
            owner = torch.repeat_interleave(torch.arange(n * M, device=dev), cnt.reshape(-1))
            b.index_put_((owner, self.kidx[ent].long()), self.val[ent].double(), accumulate=True)
        return p, b.view(n, M, K).cpu().numpy()

    def to_dense_numpy(self) -> tuple:
        """(p [N, M], b [N, M, K]) float64 numpy for the whole (small) instance."""
        return self.users_dense(np.arange(self.N))


def _gen(device, seed):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _groups(M, groups, caps, total_cap):
    S, C = [], []
    for (lo, hi), c in zip(groups, caps):
        S.append(sum(1 << j for j in range(lo, hi)))
        C.append(int(c))
    if total_cap is not None:
        S.append((1 << M) - 1)
        C.append(int(total_cap))
    return S, C


def _dense_budget(b, N, M, K, frac):
    # B_k = frac * sum_ij b_ijk, summed in float64 in chunks of users
    B = torch.zeros(K, dtype=torch.float64, device=b.device)
    bv = b.view(N, M * K)
    step = max(1, (1 << 24) // max(1, M * K))
    for s in range(0, N, step):
        B += bv[s:s + step].double().view(-1, M, K).sum(dim=(0, 1))
    return B * frac


def _dense_instance(name, N, M, K, seed, device, p_dist, b_bern, frac, S, C, recipe):
    g = _gen(device, seed)
    p = torch.empty(N * M, dtype=torch.float32, device=device)
    if p_dist == "uniform":
        p.uniform_(0.0, 1.0, generator=g)
    else:
        p.log_normal_(0.0, 1.0, generator=g)
    b = torch.empty(N * M * K, dtype=torch.float32, device=device)
    chunk = 1 << 26
    for s in range(0, b.numel(), chunk):
        seg = b[s:s + chunk]
        seg.uniform_(0.0, 1.0, generator=g)
        if b_bern is not None:
            keep = torch.empty_like(seg).uniform_(0.0, 1.0, generator=g) < b_bern
            seg.mul_(keep)
    B = _dense_budget(b, N, M, K, frac)
    return Instance(name=name, N=N, M=M, K=K, layout="dense", p=p, b=b, B=B, S=S, C=C,
                    seed=seed, recipe=recipe)


def small_dd_scd(N=10_000, seed=1, device="cpu") -> Instance:
    """N=1e4, M=10, K=5; p, b ~ U[0,1] FP32 dense; B_k = 0.2 sum b; one cap of 3."""
    M, K = 10, 5
    S, C = _groups(M, [], [], 3)
    return _dense_instance("dense_N1e4_M10_K5_cap3", N, M, K, seed, device, "uniform", None,
                           0.2, S, C, "p,b~U[0,1]; B=0.2*sum(b); total cap 3")


def hier_m20(N=1_000_000, seed=2, device="cpu") -> Instance:
    """N=1e6, M=20, K=20; p ~ lognormal(0,1); b ~ U[0,1]*Bernoulli(0.5) dense; B = 0.1 sum b;
    four groups of five items capped at 2 under a total cap of 5."""
    M, K = 20, 20
    S, C = _groups(M, [(0, 5), (5, 10), (10, 15), (15, 20)], [2, 2, 2, 2], 5)
    return _dense_instance("dense_N1e6_M20_K20_laminar", N, M, K, seed, device, "lognormal",
                           0.5, 0.1, S, C,
                           "p~lognormal(0,1); b~U[0,1]*Bern(0.5); B=0.1*sum(b); 4x(5 items cap 2) under cap 5")


def dense_2e7(N=20_000_000, seed=3, device="cpu") -> Instance:
    """N=2e7, M=10, K=10; p, b ~ U[0,1] dense; B = 0.05 sum b; {1..5}:2, {6..10}:2, total 3."""
    M, K = 10, 10
    S, C = _groups(M, [(0, 5), (5, 10)], [2, 2], 3)
    return _dense_instance("dense_N2e7_M10_K10_laminar", N, M, K, seed, device, "uniform", None,
                           0.05, S, C, "p,b~U[0,1]; B=0.05*sum(b); {1..5}:2,{6..10}:2, total 3")


def sparse_csr(N=100_000_000, seed=5, device="cpu", K=200, nnz_per_item=2) -> Instance:
    """N users, M=10, K=200; per item 2 distinct knapsacks drawn uniformly (int16, ascending);
    values ~ U[0,1] FP32 in CSR; p ~ lognormal(0,1); B = 0.05 sum b;
    constraints {1..5}:2, {6..10}:2 and a total cap of 3."""
    M = 10
    assert nnz_per_item == 2
    S, C = _groups(M, [(0, 5), (5, 10)], [2, 2], 3)
    g = _gen(device, seed)
    p = torch.empty(N * M, dtype=torch.float32, device=device)
    p.log_normal_(0.0, 1.0, generator=g)
    nnz = N * M * nnz_per_item
    val = torch.empty(nnz, dtype=torch.float32, device=device)
    kidx = torch.empty(nnz, dtype=torch.int16, device=device)
    B = torch.zeros(K, dtype=torch.float64, device=device)
    chunk_items = 1 << 24
    n_items = N * M
    for s in range(0, n_items, chunk_items):
        n = min(chunk_items, n_items - s)
        k1 = torch.randint(0, K, (n,), generator=g, device=device)
        k2 = torch.randint(0, K - 1, (n,), generator=g, device=device)
        k2 = k2 + (k2 >= k1).to(k2.dtype)
        lo = torch.minimum(k1, k2)
        hi = torch.maximum(k1, k2)
        ks = torch.stack([lo, hi], dim=1).reshape(-1)
        kidx[2 * s:2 * (s + n)] = ks.to(torch.int16)
        v = val[2 * s:2 * (s + n)]
        v.uniform_(0.0, 1.0, generator=g)
        B.index_add_(0, ks, v.double())
    B *= 0.05
    item_nnz = torch.full((N * M,), nnz_per_item, dtype=torch.uint8, device=device)
    user_off = torch.arange(N + 1, dtype=torch.int64, device=device) * (M * nnz_per_item)
    return Instance(name=f"csr_N{N:.0e}_M10_K{K}_nnz2".replace("+", ""), N=N, M=M, K=K,
                    layout="csr", p=p, B=B, S=S, C=C, user_off=user_off, item_nnz=item_nnz,
                    val=val, kidx=kidx, seed=seed,
                    recipe="p~lognormal(0,1); 2 distinct k per item uniform, val~U[0,1]; "
                           "B=0.05*sum(b); {1..5}:2,{6..10}:2, total 3")


def batched_specs(count=256, seed=4, n_lo=1_000, n_hi=1_000_000, m_lo=5, m_hi=50, k_lo=1, k_hi=64):
    """Shapes of the batched workload: N log-uniform in [n_lo, n_hi], M ~ U{m_lo..m_hi},
    K ~ U{k_lo..k_hi}, single total cap C ~ U{1..floor(M/2)}; one seed per instance."""
    rng = np.random.default_rng(seed)
    specs = []
    for t in range(count):
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        M = int(rng.integers(m_lo, m_hi + 1))
        K = int(rng.integers(k_lo, k_hi + 1))
        cap = int(rng.integers(1, M // 2 + 1))
        specs.append(dict(N=N, M=M, K=K, cap=cap, seed=seed * 100_003 + t))
    return specs


def batched_instance(spec, device="cpu") -> Instance:
    """One member of the batched workload: p, b ~ U[0,1] dense FP32, B = 0.1 sum b."""
    N, M, K = spec["N"], spec["M"], spec["K"]
    S, C = _groups(M, [], [], spec["cap"])
    return _dense_instance(f"batch_N{N}_M{M}_K{K}_C{spec['cap']}", N, M, K, spec["seed"], device,
                           "uniform", None, 0.1, S, C, "p,b~U[0,1]; B=0.1*sum(b); total cap C")


def random_small(N, M, K, seed, device="cpu", layout="dense", L_groups=None, total_cap=None,
                 p_dist="uniform", b_bern=None, frac=0.2) -> Instance:
    """Small instance of arbitrary shape for tests (dense, or CSR with random per-item
    entry counts in 0..min(K,3))."""
    if L_groups is None:
        L_groups = []
    S, C = _groups(M, [g[0] for g in L_groups], [g[1] for g in L_groups], total_cap)
    if layout == "dense":
        return _dense_instance(f"small_{N}_{M}_{K}", N, M, K, seed, device, p_dist, b_bern, frac,
                               S, C, "test instance")
    g = _gen(device, seed)
    p = torch.empty(N * M, dtype=torch.float32, device=device)
    if p_dist == "uniform":
        p.uniform_(0.0, 1.0, generator=g)
    else:
        p.log_normal_(0.0, 1.0, generator=g)
    maxn = min(K, 3)
    item_nnz = torch.randint(0, maxn + 1, (N * M,), generator=g, device=device).to(torch.uint8)
    cnt = item_nnz.long()
    nnz = int(cnt.sum())
    user_tot = cnt.view(N, M).sum(1)
    user_off = torch.zeros(N + 1, dtype=torch.int64, device=device)
    user_off[1:] = torch.cumsum(user_tot, 0)
    # distinct ascending k per item: take the first cnt of a random permutation, sorted
    keys = torch.rand((N * M, K), generator=g, device=device)
    perm = torch.argsort(keys, dim=1)[:, :maxn]
    perm, _ = torch.sort(perm, dim=1)
    mask = torch.arange(maxn, device=device)[None, :] < cnt[:, None]
    kidx = perm[mask].to(torch.int16)
    val = torch.empty(nnz, dtype=torch.float32, device=device).uniform_(0.0, 1.0, generator=g)
    B = torch.zeros(K, dtype=torch.float64, device=device)
    B.index_add_(0, kidx.long(), val.double())
    B = B * frac
    B = torch.clamp(B, min=1e-3)
    return Instance(name=f"small_csr_{N}_{M}_{K}", N=N, M=M, K=K, layout="csr", p=p, B=B, S=S,
                    C=C, user_off=user_off, item_nnz=item_nnz, val=val, kidx=kidx, seed=seed,
                    recipe="test instance (csr)")


def regular_csr(N, M, K, C, seed, device="cpu", frac=0.1) -> Instance:
    """CSR with exactly C distinct knapsacks per item (uniform, ascending), values
    U[0,1], p ~ lognormal(0,1), B = frac * sum b, no local constraints (callers set
    S, C).  With small K many knapsacks are shared by two or more items of a user."""
    assert 1 <= C <= K
    g = _gen(device, seed)
    p = torch.empty(N * M, dtype=torch.float32, device=device)
    p.log_normal_(0.0, 1.0, generator=g)
    keys = torch.rand((N * M, K), generator=g, device=device)
    ks, _ = torch.sort(torch.argsort(keys, dim=1)[:, :C], dim=1)
    kidx = ks.reshape(-1).to(torch.int16)
    val = torch.empty(N * M * C, dtype=torch.float32, device=device).uniform_(0.0, 1.0, generator=g)
    B = torch.zeros(K, dtype=torch.float64, device=device)
    B.index_add_(0, kidx.long(), val.double())
    B = torch.clamp(B * frac, min=1e-3)
    item_nnz = torch.full((N * M,), C, dtype=torch.uint8, device=device)
    user_off = torch.arange(N + 1, dtype=torch.int64, device=device) * (M * C)
    return Instance(name=f"regular_csr_{N}_{M}_{K}_{C}", N=N, M=M, K=K, layout="csr", p=p, B=B,
                    S=[], C=[], user_off=user_off, item_nnz=item_nnz, val=val, kidx=kidx,
                    seed=seed, recipe="test instance (regular csr)")


def one_to_one(N, K, Q, seed, device="cpu", frac=0.2) -> Instance:
    """Sec. 5.1's special case: M = K items per user, item k consuming only
    knapsack k (CSR with one entry per item, k = j), at most Q items per user.
    p, b ~ U[0,1]; B_k = frac * sum_i b_ikk."""
    g = _gen(device, seed)
    p = torch.empty(N * K, dtype=torch.float32, device=device).uniform_(0.0, 1.0, generator=g)
    val = torch.empty(N * K, dtype=torch.float32, device=device).uniform_(0.0, 1.0, generator=g)
    kidx = torch.arange(K, dtype=torch.int16, device=device).repeat(N)
    B = torch.clamp(val.view(N, K).double().sum(0) * frac, min=1e-3)
    item_nnz = torch.ones(N * K, dtype=torch.uint8, device=device)
    user_off = torch.arange(N + 1, dtype=torch.int64, device=device) * K
    S, C = _groups(K, [], [], Q)
    return Instance(name=f"one_to_one_{N}_{K}_Q{Q}", N=N, M=K, K=K, layout="csr", p=p, B=B, S=S, C=C,
                    user_off=user_off, item_nnz=item_nnz, val=val, kidx=kidx, seed=seed,
                    recipe="Sec. 5.1 special case (one item per knapsack, one cap)")


WORKLOADS = {
    "dense_N1e4_M10_K5": small_dd_scd,
    "dense_N1e6_M20_K20": hier_m20,
    "dense_N2e7_M10_K10": dense_2e7,
    "csr_N1e8_M10_K200": sparse_csr,
}
