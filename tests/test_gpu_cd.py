"""Block and cyclic coordinate descent (Sec. 4.3.2) and categorical decision
variables (Sec. 2) on the GPU, against the oracle.

Cyclic CD updates one multiplier per iteration and block CD a subset of them,
each by the Reduce of Algorithm 4 at the current lambda; kp_bcd_step computes
only the breakpoints of the block's knapsacks.  Every GPU step is compared
with the oracle's step at the GPU's lambda^t: the multipliers outside the
block bit for bit, the updated ones within 1e-5 relative plus the local FP32
floor of the breakpoints next to their thresholds.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp, solver
from paper_2002_00352_gb300.categorical import expand_categorical, fold_decisions
from tests.gpu_util import check_scd_step, compare_state, cuda_state, floor_ulps
from tests.helpers import random_laminar

pytestmark = pytest.mark.gpu


def _bcd(prob, lam, block):
    lt = torch.tensor(lam, dtype=torch.float64, device="cuda")
    ln = torch.zeros_like(lt)
    kp.kp_bcd_step(prob, lt, torch.tensor(block.astype(np.uint8), device="cuda"), ln)
    kp.kp_device_status(prob)
    return ln.cpu().numpy()


def _check(prob, inst, p, b, lam, block, label):
    got = _bcd(prob, lam, block)
    want = oracle.bcd_step(p, b, inst.S, inst.C, lam, inst.B.cpu().numpy(), block)
    assert np.array_equal(got[~block], lam[~block]), label
    emis = oracle.scd_map_users(p, b, inst.S, inst.C, lam)
    keep = block[emis[1]]
    emis = tuple(a[keep] for a in emis)
    check_scd_step(got, want, p, b, lam, emis, floor_ulps(inst.layout, inst.K), label=label, max_loose_share=1.0)
    return got


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_cyclic_cd_trajectory(layout):
    """Two sweeps of cyclic CD (one multiplier at a time) from lambda = 0."""
    rng = np.random.default_rng(61)
    M, K = 8, 5
    S, C = random_laminar(M, rng, max_nodes=4)
    inst = (gen.random_small(3000, M, K, seed=61, device="cuda", layout=layout, frac=0.15)
            if layout == "dense" else gen.regular_csr(3000, M, K, 2, seed=61, device="cuda", frac=0.15))
    inst.S, inst.C = S, C
    prob = kp.kp_create_from_instance(inst)
    p, b = inst.to_dense_numpy()
    lam = np.zeros(K)
    for t, blk in enumerate(solver.cyclic_blocks(K, 2)):
        block = np.zeros(K, dtype=bool)
        block[blk] = True
        lam = _check(prob, inst, p, b, lam, block, f"cyclic {layout} t={t}")


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_block_cd_random_blocks(layout):
    """Block CD with random halves of the knapsacks, from a random lambda; the
    solver driver gives the same trajectory."""
    rng = np.random.default_rng(62)
    M, K = 10, 8
    S, C = random_laminar(M, rng, max_nodes=5)
    inst = (gen.random_small(2500, M, K, seed=62, device="cuda", layout=layout, frac=0.15)
            if layout == "dense" else gen.sparse_csr(N=20_000, K=K, device="cuda"))
    if layout == "dense":
        inst.S, inst.C = S, C
    prob = kp.kp_create_from_instance(inst)
    p, b = inst.to_dense_numpy()
    lam0 = rng.uniform(0, 0.6, size=K)
    lam = lam0.copy()
    blocks = []
    for t in range(4):
        block = rng.random(K) < 0.5
        blocks.append(np.nonzero(block)[0].tolist())
        lam = _check(prob, inst, p, b, lam, block, f"block {layout} t={t}")
    prob2 = kp.kp_create_from_instance(inst)
    got, _ = solver.cd_solve(prob2, torch.tensor(lam0, device="cuda"), blocks)
    assert np.array_equal(got.cpu().numpy(), lam)


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_categorical_variables(layout):
    """x_ij in {0..u_j} as u_j binary copies (Sec. 2): decisions, consumption and one
    SCD step of the expanded instance against the oracle, and the folded integer
    decisions within their bounds."""
    rng = np.random.default_rng(63)
    M, K = 5, 4
    u = [3, 1, 2, 4, 2]
    S, C = random_laminar(M, rng, max_nodes=3)
    inst = gen.random_small(2000, M, K, seed=63, device="cuda", layout=layout, frac=0.2)
    inst.S, inst.C = S, C
    big = expand_categorical(inst, u)
    prob = kp.kp_create_from_instance(big)
    p2, b2 = big.to_dense_numpy()
    lam = rng.uniform(0, 0.5, size=K)
    x, R, d, pr, g, xb = cuda_state(prob, torch.tensor(lam, device="cuda"))
    xo, Ro, do, po = oracle.user_pass(p2, b2, big.S, big.C, lam)
    compare_state(p2, b2, lam, x, R, d, pr, xo, Ro, do, po)
    xi = fold_decisions(torch.tensor(x), u).numpy()
    assert np.all(xi >= 0) and np.all(xi <= np.array(u))
    got = _bcd(prob, lam, np.ones(K, dtype=bool))
    want, _, _ = oracle.scd_step(p2, b2, big.S, big.C, lam, big.B.cpu().numpy())
    emis = oracle.scd_map_users(p2, b2, big.S, big.C, lam)
    check_scd_step(got, want, p2, b2, lam, emis, floor_ulps(big.layout, K), label=f"categorical {layout}",
                   max_loose_share=1.0)
