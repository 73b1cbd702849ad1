"""Batched solving of many independent instances (one persistent launch per pass)
against the per-instance path and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp
from tests.gpu_util import compare_state, lam_close

pytestmark = pytest.mark.gpu


def _instances(count=9, seed=4, n_hi=20_000):
    specs = gen.batched_specs(count=count, seed=seed, n_lo=300, n_hi=n_hi, m_lo=2, m_hi=20, k_lo=1, k_hi=12)
    return [gen.batched_instance(sp, device="cuda") for sp in specs]


def test_batch_scd_equals_per_instance():
    insts = _instances()
    batch = kp.kp_batch_create(insts)
    probs = [kp.kp_create_from_instance(x) for x in insts]
    rng = np.random.default_rng(1)
    lam = torch.tensor(rng.uniform(0, 0.3, batch.totK), dtype=torch.float64, device="cuda")
    for step in range(4):
        nxt = torch.zeros_like(lam)
        kp.kp_batch_scd_step(batch, lam, nxt)
        kp.kp_batch_device_status(batch)
        for i, (x, pr) in enumerate(zip(insts, probs)):
            a, b = batch.koff[i], batch.koff[i + 1]
            one = torch.zeros(x.K, dtype=torch.float64, device="cuda")
            kp.kp_scd_step(pr, lam[a:b].contiguous(), one)
            assert torch.equal(one, nxt[a:b]), (step, i)
        lam = nxt


def test_batch_scd_matches_oracle_one_step():
    insts = _instances(count=5, seed=8, n_hi=3000)
    batch = kp.kp_batch_create(insts)
    rng = np.random.default_rng(2)
    lam_h = rng.uniform(0, 0.4, batch.totK)
    lam = torch.tensor(lam_h, device="cuda")
    nxt = torch.zeros_like(lam)
    kp.kp_batch_scd_step(batch, lam, nxt)
    kp.kp_batch_device_status(batch)
    got = nxt.cpu().numpy()
    for i, x in enumerate(insts):
        a, b = batch.koff[i], batch.koff[i + 1]
        p, bb = x.to_dense_numpy()
        want, _, _ = oracle.scd_step(p, bb, x.S, x.C, lam_h[a:b], x.B.cpu().numpy())
        assert np.all(lam_close(got[a:b], want)), (i, got[a:b], want)


def test_batch_consumption_and_dd():
    insts = _instances(count=7, seed=9, n_hi=5000)
    batch = kp.kp_batch_create(insts)
    rng = np.random.default_rng(3)
    lam_h = rng.uniform(0, 0.5, batch.totK)
    lam = torch.tensor(lam_h, device="cuda")
    R = torch.zeros(batch.totK, dtype=torch.float64, device="cuda")
    d = torch.zeros(batch.count, dtype=torch.float64, device="cuda")
    pr = torch.zeros(batch.count, dtype=torch.float64, device="cuda")
    x = torch.zeros(batch.xoff[-1], dtype=torch.int32, device="cuda")
    kp.kp_batch_reduce_consumption(batch, lam, R=R, dual_sum=d, primal_sum=pr, x_bits=x)
    nxt = torch.zeros_like(lam)
    kp.kp_batch_dd_step(batch, lam, 1e-3, nxt)
    torch.cuda.synchronize()
    for i, inst in enumerate(insts):
        a, b = batch.koff[i], batch.koff[i + 1]
        p, bb = inst.to_dense_numpy()
        xo, Ro, do, po = oracle.user_pass(p, bb, inst.S, inst.C, lam_h[a:b])
        xs = kp.unpack_x(x[batch.xoff[i]:batch.xoff[i + 1]], inst.N, inst.M).cpu().numpy().astype(np.int32)
        compare_state(p, bb, lam_h[a:b], xs, R[a:b].cpu().numpy(), float(d[i]), float(pr[i]), xo, Ro, do, po)
        want = oracle.dd_update(lam_h[a:b], R[a:b].cpu().numpy(), inst.B.cpu().numpy(), 1e-3)
        assert np.allclose(nxt[a:b].cpu().numpy(), want, rtol=1e-12, atol=1e-15)


def test_batch_rejects_csr():
    x = gen.random_small(100, 4, 3, seed=1, device="cuda", layout="csr")
    with pytest.raises(Exception):
        kp.kp_batch_create([x])


def test_batch_graph_replay_equals_eager():
    from paper_2002_00352_gb300.solver import BatchScdGraph
    insts = _instances(count=6, seed=21, n_hi=4000)
    batch = kp.kp_batch_create(insts)
    lam0 = torch.zeros(batch.totK, dtype=torch.float64, device="cuda")
    a = lam0.clone()
    b = torch.empty_like(a)
    for _ in range(4):
        kp.kp_batch_scd_step(batch, a, b)
        a, b = b, a
    g = BatchScdGraph(batch, lam0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(g.lam, a)


def test_batch_config_shape():
    """The batched workload's own shapes (N log-uniform up to 1e6, M 5..50, K 1..64,
    one total cap C in 1..M/2), on 24 of its instances: three SCD steps from lambda = 0
    by the batched path equal the per-instance path bit for bit; at the last
    lambda^t, sampled users' decisions of every instance against the oracle's
    greedy, and the whole step of the three smallest instances against the oracle's
    Algorithm 4 (1e-5 relative plus the local FP32 floor)."""
    from tests.gpu_util import check_scd_step, excused_users, floor_ulps
    specs = gen.batched_specs(count=256, n_hi=1_000_000)[:24]
    insts = [gen.batched_instance(sp, device="cuda") for sp in specs]
    batch = kp.kp_batch_create(insts)
    probs = [kp.kp_create_from_instance(x) for x in insts]
    lam = torch.zeros(batch.totK, dtype=torch.float64, device="cuda")
    for step in range(3):
        nxt = torch.zeros_like(lam)
        kp.kp_batch_scd_step(batch, lam, nxt)
        kp.kp_batch_device_status(batch)
        loop = torch.zeros_like(lam)
        for i, pr in enumerate(probs):
            a, b = batch.koff[i], batch.koff[i + 1]
            kp.kp_scd_step(pr, lam[a:b].contiguous(), loop[a:b])
            kp.kp_device_status(pr)
        assert torch.equal(loop, nxt), step
        if step < 2:
            lam = nxt
    lam_h = lam.cpu().numpy()
    got = nxt.cpu().numpy()
    rng = np.random.default_rng(9)
    for i, (x, pr) in enumerate(zip(insts, probs)):
        a, b = batch.koff[i], batch.koff[i + 1]
        idx = np.sort(rng.choice(x.N, size=min(300, x.N), replace=False))
        p, bb = x.users_dense(idx)
        xb = kp.kp_solve_users(pr, lam[a:b].contiguous())
        xs = kp.unpack_x(xb.view(x.N, -1)[torch.as_tensor(idx, device="cuda")].reshape(-1), len(idx), x.M).cpu().numpy()
        xo, _, _, _ = oracle.user_pass(p, bb, x.S, x.C, lam_h[a:b])
        exc = excused_users(p, bb, lam_h[a:b])
        assert np.array_equal(xs[~exc], xo[~exc]), i
    for i in np.argsort([x.N * x.M * x.K for x in insts])[:3]:
        x = insts[i]
        a, b = batch.koff[i], batch.koff[i + 1]
        p, bb = x.to_dense_numpy()
        want, _, _ = oracle.scd_step(p, bb, x.S, x.C, lam_h[a:b], x.B.cpu().numpy())
        emis = oracle.scd_map_users(p, bb, x.S, x.C, lam_h[a:b])
        check_scd_step(got[a:b], want, p, bb, lam_h[a:b], emis, floor_ulps("dense", x.K), label=f"batch inst {i}",
                       max_loose_share=1.0)


def test_batch_with_solo_instances():
    """A batch mixing instances that fill the GPU on their own (run by their own
    launches inside the batched calls) with small ones (the shared persistent launch):
    SCD steps, the consumption pass and a DD step equal the per-instance path bit for
    bit, eagerly and replayed from a CUDA graph."""
    from paper_2002_00352_gb300.solver import BatchScdGraph
    big = [gen.dense_2e7(N=400_000, device="cuda"), gen.hier_m20(N=60_000, device="cuda")]
    insts = big + _instances(count=4, seed=31, n_hi=4000)
    batch = kp.kp_batch_create(insts)
    probs = [kp.kp_create_from_instance(x) for x in insts]
    lam0 = torch.zeros(batch.totK, dtype=torch.float64, device="cuda")
    lam = lam0.clone()
    for step in range(4):
        nxt = torch.zeros_like(lam)
        kp.kp_batch_scd_step(batch, lam, nxt)
        kp.kp_batch_device_status(batch)
        for i, (x, pr) in enumerate(zip(insts, probs)):
            a, b = batch.koff[i], batch.koff[i + 1]
            one = torch.zeros(x.K, dtype=torch.float64, device="cuda")
            kp.kp_scd_step(pr, lam[a:b].contiguous(), one)
            assert torch.equal(one, nxt[a:b]), (step, i)
        lam = nxt
    R = torch.zeros(batch.totK, dtype=torch.float64, device="cuda")
    d = torch.zeros(batch.count, dtype=torch.float64, device="cuda")
    pr_ = torch.zeros(batch.count, dtype=torch.float64, device="cuda")
    kp.kp_batch_reduce_consumption(batch, lam, R=R, dual_sum=d, primal_sum=pr_)
    dd = torch.zeros_like(lam)
    kp.kp_batch_dd_step(batch, lam, 1e-3, dd)
    kp.kp_batch_device_status(batch)
    for i, (x, pr) in enumerate(zip(insts, probs)):
        a, b = batch.koff[i], batch.koff[i + 1]
        Ri = torch.zeros(x.K, dtype=torch.float64, device="cuda")
        di = torch.zeros(1, dtype=torch.float64, device="cuda")
        pi = torch.zeros(1, dtype=torch.float64, device="cuda")
        kp.kp_reduce_consumption(pr, lam[a:b].contiguous(), R=Ri, dual_sum=di, primal_sum=pi)
        assert torch.equal(Ri, R[a:b]) and torch.equal(di[0], d[i]) and torch.equal(pi[0], pr_[i]), i
        ddi = torch.zeros(x.K, dtype=torch.float64, device="cuda")
        kp.kp_dd_step(pr, lam[a:b].contiguous(), 1e-3, ddi)
        assert torch.equal(ddi, dd[a:b]), i
    g = BatchScdGraph(kp.kp_batch_create(insts), lam0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    want = lam0.clone()
    nb = kp.kp_batch_create(insts)
    tmp = torch.empty_like(want)
    for _ in range(4):
        kp.kp_batch_scd_step(nb, want, tmp)
        want, tmp = tmp, want
    assert torch.equal(g.lam, want)
