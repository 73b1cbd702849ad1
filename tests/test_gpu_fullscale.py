"""Parity at the full size of the headline workload (N = 1e8 users, M = 10, K = 200,
CSR with 2 entries per item), in the launch configuration bench.py times.

The oracle cannot run 1e8 users, so the checks are:
  * decisions of sampled users against the oracle, one user at a time
    (Algorithm 1 at the GPU's lambda^t);
  * the consumption reduction against an independent float64 recount of
    sum_i sum_j b_ijk x_ij from the GPU's decisions (torch ops, exact up to
    float64 rounding);
  * the Reduce rule of Algorithm 4 (reading R6) as a property at any size: with
    the other multipliers at lambda^t, the k-consumption just above the
    selected lambda_k fits B_k and just below it does not.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp
from tests.gpu_util import TAU

pytestmark = pytest.mark.gpu

N = 100_000_000


@pytest.fixture(scope="module")
def big():
    if torch.cuda.get_device_properties(0).total_memory < 60e9:
        pytest.skip("needs a GPU with > 60 GB")
    inst = gen.sparse_csr(N=N, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    lam = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    nxt = torch.zeros_like(lam)
    for _ in range(4):  # the bench's warm-up part of the trajectory
        kp.kp_scd_step(prob, lam, nxt)
        lam, nxt = nxt, lam
    kp.kp_device_status(prob)
    yield inst, prob, lam
    prob.close()
    del inst
    torch.cuda.empty_cache()


def test_fullscale_decisions_and_consumption(big):
    inst, prob, lam = big
    K, M = inst.K, inst.M
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    x = torch.zeros(N, dtype=torch.int32, device="cuda")
    kp.kp_reduce_consumption(prob, lam, R=R, x_bits=x)
    torch.cuda.synchronize()
    # sampled users against the oracle
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(N, size=2000, replace=False))
    p, b = inst.users_dense(idx)
    lam_h = lam.cpu().numpy()
    xs = kp.unpack_x(x[torch.as_tensor(idx, device="cuda")], len(idx), M).cpu().numpy()
    pt = p - np.einsum("ijk,k->ij", b, lam_h)
    s = p + np.einsum("ijk,k->ij", b, lam_h)
    bad = 0
    for r in range(len(idx)):
        want = oracle.greedy(pt[r], inst.S, inst.C)
        if not np.array_equal(want, xs[r]):
            d = np.abs(pt[r][:, None] - pt[r][None, :]) <= TAU * (s[r][:, None] + s[r][None, :])
            np.fill_diagonal(d, False)
            near = (np.abs(pt[r]) <= TAU * s[r]).any() or d.any()
            assert near, (idx[r], want, xs[r], pt[r])
            bad += 1
    assert bad <= 2
    # consumption: recount sum_ij b_ijk x_ij in float64 from the decisions
    xm = kp.unpack_x(x, N, M).view(-1).bool()                 # [N*M]
    sel_items = torch.nonzero(xm).view(-1)
    ent = (sel_items * 2).repeat_interleave(2) + torch.arange(2, device="cuda").repeat(sel_items.numel())
    R_ref = torch.zeros(K, dtype=torch.float64, device="cuda")
    R_ref.index_add_(0, inst.kidx[ent].long(), inst.val[ent].double())
    assert torch.all(torch.abs(R - R_ref) <= 1e-9 * R_ref + 1e-6)


def test_fullscale_threshold_rule(big):
    inst, prob, lam = big
    nxt = torch.zeros_like(lam)
    kp.kp_scd_step(prob, lam, nxt)
    kp.kp_device_status(prob)
    lam_h, nxt_h, B = lam.cpu().numpy(), nxt.cpu().numpy(), inst.B.cpu().numpy()
    R = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    ks = rng.choice(np.nonzero(nxt_h > 0)[0], size=6, replace=False)
    eps = 1e-5
    for k in ks:
        for f, fits in ((1 + eps, True), (1 - eps, False)):
            l2 = lam_h.copy()
            l2[k] = nxt_h[k] * f
            kp.kp_reduce_consumption(prob, torch.tensor(l2, device="cuda"), R=R)
            Rk = float(R[k])
            assert (Rk <= B[k]) == fits, (k, f, Rk, B[k])
