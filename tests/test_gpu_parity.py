"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every test here needs a GB300 and the built libkp.so; inputs are the seeded
generators of paper_2002_00352_gb300.gen, created on the GPU and copied to the
host for the oracle.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp
from tests.gpu_util import (REL, REL_LAMBDA, TAU, check_scd_step, compare_state, cuda_state, excused_users,
                            floor_ulps, lam_close, lam_close_local, local_floor)
from tests.helpers import random_laminar

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _problem(inst):
    return kp.kp_create_from_instance(inst)


def _dense_np(inst):
    return inst.to_dense_numpy()


# ---------------------------------------------------------------------------
# decisions, consumption, objectives at fixed lambda (Algorithm 1 + Algorithm 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("layout", ["dense", "csr"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_state_parity_random_trees(layout, seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(2, 14))
    K = int(rng.integers(1, 9))
    S, C = random_laminar(M, rng, max_nodes=6)
    N = 3001
    inst = gen.random_small(N, M, K, seed=seed, device="cuda", layout=layout)
    inst.S, inst.C = S, C
    prob = _problem(inst)
    p, b = _dense_np(inst)
    for trial in range(4):
        lam = rng.uniform(0, 0.6, size=K) * (rng.random(K) < 0.8)
        x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
        xo, Ro, do, po = oracle.user_pass(p, b, S, C, lam)
        compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)
        assert g == pytest.approx(d + float(lam @ inst.B.cpu().numpy()), rel=1e-12)


def test_state_parity_small_config():
    inst = gen.small_dd_scd(device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    rng = np.random.default_rng(0)
    for lam in [np.zeros(5), rng.uniform(0, 1, 5), np.full(5, 0.66), np.full(5, 50.0)]:
        x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
        xo, Ro, do, po = oracle.user_pass(p, b, inst.S, inst.C, lam)
        compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)


def test_state_parity_sparse_config_downscaled():
    inst = gen.sparse_csr(N=20_000, device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    rng = np.random.default_rng(5)
    lam = rng.uniform(0, 8, size=inst.K)
    x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
    xo, Ro, do, po = oracle.user_pass(p, b, inst.S, inst.C, lam)
    compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)


# ---------------------------------------------------------------------------
# one SCD iteration (Algorithms 3-4) at the same lambda^t
# ---------------------------------------------------------------------------

def _scd_gpu_state(prob, lam):
    """One SCD step; also the consumption and objectives the breakpoint pass reports."""
    lt = torch.tensor(lam, dtype=torch.float64, device="cuda")
    ln = torch.zeros_like(lt)
    R = torch.zeros_like(lt)
    d = torch.zeros((), dtype=torch.float64, device="cuda")
    pr = torch.zeros((), dtype=torch.float64, device="cuda")
    kp.kp_scd_step(prob, lt, ln, R=R, dual_sum=d, primal_sum=pr)
    kp.kp_device_status(prob)
    return ln.cpu().numpy(), R.cpu().numpy(), float(d), float(pr)


def _check_breakpoint_state(p, b, lam, R, d, pr, Ro, do, po):
    """The breakpoint pass reports R at lambda^t as the mass of the breakpoints above
    lambda_k^t (regular CSR rows): equal to the oracle's consumption up to the
    contributions of users with near-tied or near-zero reduced costs."""
    exc = excused_users(p, b, lam)
    slackR = b[exc].sum(axis=(0, 1)) if exc.any() else np.zeros(b.shape[2])
    assert np.all(np.abs(R - Ro) <= REL * np.abs(Ro) + slackR + 1e-9), (R, Ro)
    s = p + np.einsum("ijk,k->ij", b, lam)
    assert abs(d - do) <= REL * abs(do) + (2 * TAU * s[exc].sum() if exc.any() else 0.0) + 1e-9
    assert abs(pr - po) <= REL * abs(po) + (p[exc].sum() if exc.any() else 0.0) + 1e-9


def _scd_gpu(prob, lam):
    lt = torch.tensor(lam, dtype=torch.float64, device="cuda")
    ln = torch.zeros_like(lt)
    kp.kp_scd_step(prob, lt, ln)
    kp.kp_device_status(prob)
    return ln.cpu().numpy()


@pytest.mark.parametrize("K,Q,frac", [(10, 3, 0.2), (16, 1, 0.03), (8, 8, 0.2)])
def test_scd_step_one_item_per_knapsack(K, Q, frac):
    """Sec. 5.1's special case (M = K, item k consumes only knapsack k, at most Q
    items; Q = K: the cap never binds): five GPU SCD steps from lambda = 0, each
    against Algorithm 5's Map with Algorithm 4's Reduce at the GPU's lambda^t, at
    1e-5 relative plus the local FP32 floor of the breakpoints next to each
    threshold."""
    N = 20_000
    inst = gen.one_to_one(N, K, Q, seed=31 + K, device="cuda", frac=frac)
    prob = _problem(inst)
    p = inst.p.view(N, K).double().cpu().numpy()
    bd = inst.val.view(N, K).double().cpu().numpy()
    B = inst.B.cpu().numpy()
    b3 = np.zeros((N, K, K))
    for k in range(K):
        b3[:, k, k] = bd[:, k]
    lam = np.zeros(K)
    for t in range(5):
        got = _scd_gpu(prob, lam)
        want = oracle.alg5_step(p, bd, Q, lam, B)
        emis = oracle.alg5_map_users(p, bd, Q, lam)
        check_scd_step(got, want, p, b3, lam, emis, floor_ulps("csr", K), label=f"alg5 K={K} Q={Q} t={t}",
                       max_loose_share=1.0)
        lam = got


@pytest.mark.parametrize("layout", ["dense", "csr"])
@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_scd_step_parity_random(layout, seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(2, 11))
    K = int(rng.integers(1, 7))
    S, C = random_laminar(M, rng, max_nodes=5)
    inst = gen.random_small(2000, M, K, seed=seed, device="cuda", layout=layout, frac=0.15)
    inst.S, inst.C = S, C
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    for trial in range(3):
        lam = rng.uniform(0, 0.8, size=K) * (rng.random(K) < 0.8)
        got = _scd_gpu(prob, lam)
        want, _, _ = oracle.scd_step(p, b, S, C, lam, B)
        assert np.all(lam_close(got, want)), (got, want)


@pytest.mark.parametrize("M,Cn,K,seed", [(10, 2, 6, 21), (8, 2, 5, 22), (16, 2, 9, 23),
                                         (10, 1, 3, 24), (8, 1, 4, 25), (16, 1, 5, 26)])
def test_regular_csr_shared_knapsacks(M, Cn, K, seed):
    """Every item has exactly C entries and K is small, so most knapsacks of a user are
    used by two of its items (the pair sweep) or by three or more (their own kernel,
    up to all M items); random laminar families leave more fixed lines selected than
    the pair sweep keeps in order.  Decisions, consumption and one SCD step against
    the oracle."""
    rng = np.random.default_rng(seed)
    S, C = random_laminar(M, rng, max_nodes=6)
    inst = gen.regular_csr(3000, M, K, Cn, seed=seed, device="cuda", frac=0.15)
    inst.S, inst.C = S, C
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    for trial in range(3):
        lam = rng.uniform(0, 0.8, size=K) * (rng.random(K) < 0.85)
        x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
        xo, Ro, do, po = oracle.user_pass(p, b, S, C, lam)
        compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)
        got, Rb, db, pb = _scd_gpu_state(prob, lam)
        _check_breakpoint_state(p, b, lam, Rb, db, pb, Ro, do, po)
        want, _, _ = oracle.scd_step(p, b, S, C, lam, B)
        assert np.all(lam_close(got, want)), (trial, got, want)


@pytest.mark.parametrize("layout", ["csr", "dense"])
def test_scd_step_parity_wide_users(layout):
    """M = 20 and 40 items per user (beyond the register path of 16): the general
    per-user routine and its kinetic sweeps, one SCD step and the state against the
    oracle."""
    for M, K, seed in ((20, 4, 31), (40, 3, 32)):
        rng = np.random.default_rng(seed)
        S, C = random_laminar(M, rng, max_nodes=5)
        inst = gen.random_small(600, M, K, seed=seed, device="cuda", layout=layout, frac=0.15)
        inst.S, inst.C = S, C
        prob = _problem(inst)
        p, b = _dense_np(inst)
        B = inst.B.cpu().numpy()
        lam = rng.uniform(0, 0.8, size=K)
        x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
        xo, Ro, do, po = oracle.user_pass(p, b, S, C, lam)
        compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)
        got = _scd_gpu(prob, lam)
        want, _, _ = oracle.scd_step(p, b, S, C, lam, B)
        assert np.all(lam_close(got, want)), (M, got, want)


def test_scd_step_parity_largest_K():
    """K = KP_MAX_K = 2048 on regular CSR rows (M = 10, 2 entries per item): the
    per-knapsack state of the breakpoint pass is at its largest, the pass keeps one
    user tile per sweep phase; the state and one SCD step against the oracle.  With
    about 4 breakpoints per knapsack thresholds spread widely, down to 1e-5 of
    lambda_k^t, where a FP32 breakpoint has lost relative precision: its absolute
    error is a few ulps of s_j / b_jk (s_j = p_j + sum_k lambda_k b_jk, the scale
    of the reduced cost), which the local floor of the breakpoints next to each
    threshold allows on top of 1e-5 relative."""
    rng = np.random.default_rng(41)
    M, K = 10, 2048
    S, C = random_laminar(M, rng, max_nodes=4)
    inst = gen.regular_csr(400, M, K, 2, seed=41, device="cuda", frac=0.2)
    inst.S, inst.C = S, C
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    lam, _, _ = oracle.scd_step(p, b, S, C, rng.uniform(0, 0.8, size=K), B)
    x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
    xo, Ro, do, po = oracle.user_pass(p, b, S, C, lam)
    compare_state(p, b, lam, x, R, d, pr, xo, Ro, do, po)
    got, Rb, db, pb = _scd_gpu_state(prob, lam)
    _check_breakpoint_state(p, b, lam, Rb, db, pb, Ro, do, po)
    want, _, _ = oracle.scd_step(p, b, S, C, lam, B)
    # with about 4 breakpoints per knapsack one user whose reduced costs are
    # near-tied (decisions excused above) can move a threshold to its neighbour:
    # only knapsacks touched by such a user may differ beyond the local floor
    exc = excused_users(p, b, lam)
    touched = (b[exc] > 0).any(axis=(0, 1)) if exc.any() else np.zeros(K, dtype=bool)
    emis = oracle.scd_map_users(p, b, S, C, lam)
    check_scd_step(got, want, p, b, lam, emis, floor_ulps("csr", K), label="K=2048", max_loose_share=1.0,
                   excused_k=touched)
    assert touched.sum() <= 0.01 * K, touched.sum()


@pytest.mark.parametrize("which", ["dense", "csr"])
def test_presolve_matches_oracle(which):
    """Sec. 5.3: kp_presolve on a sampled quarter of the users (budgets scaled by
    n / N).  kp_presolve with t iterations is deterministic, so its results for
    t = 1, 2, 3 are the GPU's trajectory on the sample: each step against the
    oracle's step (Algorithm 4 on the same sample and budgets) at the GPU's
    lambda^t, 1e-5 relative plus the local FP32 floor."""
    inst = gen.small_dd_scd(device="cuda") if which == "dense" else gen.sparse_csr(N=20_000, device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    g = torch.Generator(device="cpu").manual_seed(11)
    users = torch.randperm(inst.N, generator=g)[: inst.N // 4].sort().values
    us = users.numpy()
    ps, bs, Bs = p[us], b[us], B * (len(us) / inst.N)
    lam = np.zeros(inst.K)
    for iters in (1, 2, 3):
        got = kp.kp_presolve(prob, users.to("cuda"), iters).cpu().numpy()
        want, _, _ = oracle.scd_step(ps, bs, inst.S, inst.C, lam, Bs)
        emis = oracle.scd_map_users(ps, bs, inst.S, inst.C, lam)
        check_scd_step(got, want, ps, bs, lam, emis, floor_ulps(inst.layout, inst.K),
                       label=f"presolve {which} t={iters}", max_loose_share=1.0)
        lam = got
    with pytest.raises(kp.KpError):
        kp.kp_presolve(prob, torch.tensor([0, inst.N], dtype=torch.int64, device="cuda"), 1)


def test_scd_trajectory_small_config():
    """N=1e4, M=10, K=5: 50 SCD iterations; each GPU step matches the oracle's step
    taken at the GPU's own lambda^t."""
    inst = gen.small_dd_scd(device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    lam = np.zeros(inst.K)
    for t in range(50):
        got = _scd_gpu(prob, lam)
        if t < 6 or t % 7 == 0:
            want, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
            assert np.all(lam_close(got, want)), (t, got, want)
        lam = got


def test_scd_step_sparse_downscaled():
    inst = gen.sparse_csr(N=20_000, device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    lam = np.zeros(inst.K)
    for t in range(4):
        got, Rb, db, pb = _scd_gpu_state(prob, lam)
        _, Ro, do, po = oracle.user_pass(p, b, inst.S, inst.C, lam, want_x=False)
        _check_breakpoint_state(p, b, lam, Rb, db, pb, Ro, do, po)
        want, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
        frac_ok = lam_close(got, want).mean()
        assert frac_ok == 1.0, (t, frac_ok, np.max(np.abs(got - want) / np.maximum(want, 1e-12)))
        lam = got


def test_dd_trajectory_small_config():
    """Eq. (14): 50 DD iterations at alpha = 1e-3 (Sec. 6.5's learning rates)."""
    inst = gen.small_dd_scd(device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    lam_t = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    nxt = torch.zeros_like(lam_t)
    R = torch.zeros_like(lam_t)
    for t in range(50):
        kp.kp_dd_step(prob, lam_t, 1e-3, nxt, R=R)
        lam = lam_t.cpu().numpy()
        _, Ro, _, _ = oracle.user_pass(p, b, inst.S, inst.C, lam, want_x=False)
        want = oracle.dd_update(lam, Ro, B, 1e-3)
        got = nxt.cpu().numpy()
        # Eq. (14) moves lambda by alpha * R: R within 1e-6 relative plus the whole
        # consumption of the users whose decisions are excused (margins below 1e-6)
        exc = excused_users(p, b, lam)
        slackR = b[exc].sum(axis=(0, 1)) if exc.any() else np.zeros(inst.K)
        tol = 1e-3 * (REL * np.abs(Ro) + slackR) + 1e-12 * np.abs(want) + 1e-12
        assert np.all(np.abs(got - want) <= tol), (t, got, want, tol)
        lam_t.copy_(nxt)


def test_golden_fixture():
    d = json.load(open(os.path.join(HERE, "golden", "oracle_tiny.json")))
    N, M, K = d["N"], d["M"], d["K"]
    p = torch.tensor(d["p"], dtype=torch.float32, device="cuda")
    b = torch.tensor(d["b"], dtype=torch.float32, device="cuda")
    B = torch.tensor(d["B"], dtype=torch.float64, device="cuda")
    prob = kp.kp_create(N, M, K, p, B, d["S"], d["C"], b_dense=b)
    lam = np.zeros(K)
    for t in range(1, len(d["scd_lambda"])):
        lam = _scd_gpu(prob, lam)
        assert np.all(lam_close(lam, d["scd_lambda"][t])), (t, lam, d["scd_lambda"][t])
    lt = torch.zeros(K, dtype=torch.float64, device="cuda")
    nx = torch.zeros_like(lt)
    for t in range(1, len(d["dd_lambda"])):
        kp.kp_dd_step(prob, lt, d["alpha"], nx)
        lt.copy_(nx)
        assert np.all(np.abs(lt.cpu().numpy() - np.array(d["dd_lambda"][t])) <= 1e-9 + 1e-6 * np.abs(d["dd_lambda"][t]))


# ---------------------------------------------------------------------------
# dual gradient (Danskin) and the autograd function
# ---------------------------------------------------------------------------

def test_dual_backward_matches_oracle_and_fd():
    """Danskin's gradient of the dual (Eq. (5)) on the N=2e7, M=10, K=10 recipe at
    N = 5e4: against the oracle's x* and R (decisions exact for every user whose
    margins exceed 1e-6, R within 1e-6 relative plus the excused users' b), and
    against central differences of the oracle's FP64 dual at h = 1e-4.  g is
    convex and piecewise linear in lambda_k with slope B_k - R_k, so its central
    difference lies between the slopes at lambda - h e_k and lambda + h e_k."""
    from paper_2002_00352_gb300.autograd import dual
    inst = gen.dense_2e7(N=50_000, device="cuda")
    prob = _problem(inst)
    p, b = _dense_np(inst)
    B = inst.B.cpu().numpy()
    rng = np.random.default_rng(3)
    inst.p.requires_grad_(True)
    inst.B.requires_grad_(True)
    h = 1e-4

    def gpu_slope(lv):
        """(B - R)(lv) from the GPU and its allowance (1e-6 R + excused users' b)."""
        _, R, _, _, _, _ = cuda_state(prob, torch.tensor(lv, device="cuda"))
        exc = excused_users(p, b, lv)
        slack = b[exc].sum(axis=(0, 1)) if exc.any() else np.zeros(inst.K)
        return B - R, REL * np.abs(R) + slack + 1e-9

    for trial in range(64):
        lam0 = rng.uniform(0.05, 0.2, size=inst.K)
        lam = torch.tensor(lam0, device="cuda", requires_grad=True)
        g = dual(lam, prob)
        (gl, gp, gB) = torch.autograd.grad(2.0 * g, [lam, inst.p, inst.B])
        gl = gl.cpu().numpy()
        if trial < 4:
            x, R, _, _ = oracle.user_pass(p, b, inst.S, inst.C, lam0)
            exc = excused_users(p, b, lam0)
            slack = b[exc].sum(axis=(0, 1)) if exc.any() else np.zeros(inst.K)
            assert np.all(np.abs(gl / 2.0 - (B - R)) <= REL * np.abs(R) + slack + 1e-9), trial
            assert np.allclose(gB.cpu().numpy(), 2.0 * lam0, rtol=1e-15, atol=0)
            xm = gp.detach().cpu().numpy().reshape(inst.N, inst.M)
            assert set(np.unique(xm)) <= {0.0, 2.0}
            assert np.array_equal(xm[~exc] / 2.0, x[~exc]), trial
        # central difference of the oracle's dual in coordinate k
        k = trial % inst.K
        e = np.zeros(inst.K)
        e[k] = h
        fd = (oracle.dual_value(p, b, inst.S, inst.C, lam0 + e, B)
              - oracle.dual_value(p, b, inst.S, inst.C, lam0 - e, B)) / (2 * h)
        lo, tlo = gpu_slope(lam0 - e)
        hi, thi = gpu_slope(lam0 + e)
        fd_noise = 1e-9 * np.abs(B[k]) / h      # FP64 rounding of the two dual values
        assert lo[k] - tlo[k] - fd_noise <= fd <= hi[k] + thi[k] + fd_noise, (trial, lo[k], fd, hi[k])
        # and the gradient at lambda itself between the two one-sided slopes
        assert lo[k] - tlo[k] <= gl[k] / 2.0 <= hi[k] + thi[k], (trial, lo[k], gl[k] / 2.0, hi[k])


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_edge_single_user_single_item():
    p = torch.tensor([0.6], dtype=torch.float32, device="cuda")
    b = torch.tensor([0.3], dtype=torch.float32, device="cuda")
    B = torch.tensor([0.1], dtype=torch.float64, device="cuda")
    prob = kp.kp_create(1, 1, 1, p, B, [], [], b_dense=b)
    got = _scd_gpu(prob, np.zeros(1))
    assert got[0] == pytest.approx(2.0, rel=1e-6)   # zero crossing p/b
    x, R, d, pr, g, _ = cuda_state(prob, torch.tensor([2.5], dtype=torch.float64, device="cuda"))
    assert x.sum() == 0 and R[0] == 0.0


def test_edge_empty_csr_rows_and_zero_entries():
    N, M, K = 5, 4, 3
    p = torch.rand(N * M, device="cuda", generator=torch.Generator(device="cuda").manual_seed(7))
    nnz = torch.tensor([0, 0, 0, 0, 1, 0, 2, 0, 0, 0, 0, 0, 3, 1, 0, 0, 0, 0, 0, 1],
                       dtype=torch.uint8, device="cuda")
    cnt = nnz.long().view(N, M).sum(1)
    off = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    off[1:] = torch.cumsum(cnt, 0)
    ks = torch.tensor([2, 0, 1, 0, 1, 2, 1, 0], dtype=torch.int16, device="cuda")
    vals = torch.tensor([0.5, 0.0, 0.7, 0.2, 0.3, 0.9, 0.4, 0.6], device="cuda")
    B = torch.tensor([0.5, 0.5, 0.5], dtype=torch.float64, device="cuda")
    prob = kp.kp_create(N, M, K, p, B, [0b1111], [2], csr_user_off=off, csr_item_nnz=nnz,
                        csr_val=vals, csr_k=ks)
    dense = oracle.densify_csr(N, M, K, off.cpu(), nnz.cpu(), vals.cpu(), ks.cpu())
    pn = p.cpu().double().numpy().reshape(N, M)
    lam = np.array([0.3, 0.0, 1.2])
    x, R, d, pr, g, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
    xo, Ro, do, po = oracle.user_pass(pn, dense, [0b1111], [2], lam)
    compare_state(pn, dense, lam, x, R, d, pr, xo, Ro, do, po)
    got = _scd_gpu(prob, lam)
    want, _, _ = oracle.scd_step(pn, dense, [0b1111], [2], lam, B.cpu().numpy())
    emis = oracle.scd_map_users(pn, dense, [0b1111], [2], lam)
    floor = local_floor(got, want, pn, dense, lam, emis, floor_ulps("csr", K))
    assert np.all(lam_close_local(got, want, floor)), (got, want, floor)


def test_errors_are_reported():
    p = torch.rand(8, device="cuda")
    b = torch.rand(8 * 2, device="cuda")
    B = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(kp.KpError) as e:
        kp.kp_create(2, 4, 2, p, B, [0b0011, 0b0110], [1, 1], b_dense=b)   # not hierarchical
    assert e.value.status == kp.KP_EINVAL
    with pytest.raises(kp.KpError) as e:
        kp.kp_create(2, 4, 2, p, B, [0b0011], [0], b_dense=b)              # C_l must be > 0
    assert e.value.status == kp.KP_EINVAL
    bneg = b.clone()
    bneg[3] = -1.0
    with pytest.raises(kp.KpError) as e:
        kp.kp_create(2, 4, 2, p, B, [0b0011], [1], b_dense=bneg)           # b >= 0 (Sec. 2)
    assert e.value.status == kp.KP_EDATA
    with pytest.raises(kp.KpError) as e:
        kp.kp_create(2, 65, 2, p, B, [], [], b_dense=b)                    # M > 64
    assert e.value.status == kp.KP_EINVAL


def test_determinism():
    inst = gen.small_dd_scd(device="cuda")
    prob = _problem(inst)
    lam = torch.full((inst.K,), 0.4, dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(2):
        R = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
        d = torch.zeros((), dtype=torch.float64, device="cuda")
        nxt = torch.zeros_like(lam)
        kp.kp_scd_step(prob, lam, nxt, R=R, dual_sum=d)
        outs.append((R.cpu().numpy().tobytes(), float(d), nxt.cpu().numpy().tobytes()))
    assert outs[0] == outs[1]


def test_graph_replay_matches_eager():
    from paper_2002_00352_gb300.solver import ScdGraph, scd_solve
    inst = gen.sparse_csr(N=20_000, device="cuda")
    prob = _problem(inst)
    lam0 = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    eager, _ = scd_solve(prob, lam0, 6)
    g = ScdGraph(prob, lam0)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(g.lam, eager)


@pytest.mark.parametrize("case", ["hier_m20", "dense_2e7", "ragged"])
def test_staging_modes_agree(case):
    """The dense passes give the same bits whether each tile is loaded by the
    block's threads (staging 0) or double-buffered by bulk asynchronous copies
    (staging 1), at several tile sizes: four SCD steps from lambda = 0 (breakpoint
    and re-run passes), then the consumption pass.  The ragged case has a last
    tile whose b and p rows end off a 16-byte boundary (60 bytes of b and 20 of p
    per user), loaded past the bulk copy's end."""
    if case == "hier_m20":
        inst = gen.hier_m20(N=30_000, device="cuda")
    elif case == "dense_2e7":
        inst = gen.dense_2e7(N=20_000, device="cuda")
    else:
        inst = gen.random_small(2001, 5, 3, seed=9, device="cuda", layout="dense", frac=0.2)
    runs = []
    for staging, tile in ((0, 0), (1, 0), (1, 12), (1, 8)):
        prob = _problem(inst)
        kp.kp_set_tile(prob, tile, staging)
        lam = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
        nxt, R = torch.zeros_like(lam), torch.zeros_like(lam)
        d, pr = torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda")
        out = []
        for _ in range(4):
            kp.kp_scd_step(prob, lam, nxt, R=R, dual_sum=d, primal_sum=pr)
            out += [nxt.clone(), R.clone(), d.clone(), pr.clone()]
            lam, nxt = nxt, lam
        kp.kp_reduce_consumption(prob, lam, R=R, dual_sum=d, primal_sum=pr)
        out += [R.clone(), d.clone(), pr.clone()]
        kp.kp_device_status(prob)
        runs.append(out)
    for r in runs[1:]:
        for a_, b_ in zip(runs[0], r):
            assert torch.equal(a_, b_)
    with pytest.raises(kp.KpError):
        kp.kp_set_tile(prob, 0, 2)


def test_bounded_wait_reports_timeout():
    """Failure detection without a fault: a wait on an mbarrier that nothing arrives
    on (the wait of staging mode 1) gives up after its limit and reports KP_ETIMEOUT
    through the status word; the context stays usable (a step runs after it)."""
    import time
    t0 = time.perf_counter()
    with pytest.raises(kp.KpError) as ei:
        kp.kp_wait_selftest(2_000_000)
    assert ei.value.status == kp.KP_ETIMEOUT
    assert time.perf_counter() - t0 >= 2e-3
    with pytest.raises(kp.KpError) as ei:
        kp.kp_wait_selftest(10)
    assert ei.value.status == kp.KP_EINVAL
    inst = gen.small_dd_scd(N=500, seed=3, device="cuda")
    prob = _problem(inst)
    lam = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    nxt = torch.zeros_like(lam)
    kp.kp_scd_step(prob, lam, nxt)
    kp.kp_device_status(prob)


def test_autotune_keeps_results():
    inst = gen.hier_m20(N=30_000, device="cuda")
    prob = _problem(inst)
    lam = torch.full((inst.K,), 0.05, dtype=torch.float64, device="cuda")
    ref = torch.zeros_like(lam)
    kp.kp_scd_step(prob, lam, ref)
    tile = kp.kp_autotune(prob)
    assert tile >= 1
    got = torch.zeros_like(lam)
    kp.kp_scd_step(prob, lam, got)
    kp.kp_device_status(prob)
    assert torch.equal(got, ref)
