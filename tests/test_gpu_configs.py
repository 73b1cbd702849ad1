"""Oracle parity on the dense hierarchical workloads of Sec. 6's recipe:

  * N=1e6, M=20, K=20: p ~ lognormal(0,1), b ~ U[0,1] * Bernoulli(0.5) dense,
    B = 0.1 sum b, four groups of five items capped at 2 under a total cap of 5,
    SCD for 100 iterations;
  * N=2e7, M=10, K=10: p, b ~ U[0,1] dense, B = 0.05 sum b, {1..5}:2, {6..10}:2
    under a total cap of 3, SCD plus the dual gradient checked by central
    differences at h = 1e-4 on 64 random lambda.

The oracle runs Algorithms 3-4 literally (O(K M^3 log M) per user), so every SCD
step is compared element by element on a down-scaled N from the same generator
(each GPU step against the oracle's step at the GPU's lambda^t: decisions,
consumption and objectives at lambda^t, lambda^{t+1} within 1e-5 relative plus the
local FP32 floor of the breakpoints next to each threshold).  At the full N the
checks are the ones that hold at any size: sampled users' decisions against the
oracle's greedy, the consumption recounted in FP64 from the GPU's decisions, the
Reduce rule of Algorithm 4 as a property, and (N=2e7) the dual gradient between
the one-sided slopes that bound its central difference.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp
from tests.gpu_util import (REL, TAU, check_scd_step, compare_state, cuda_state, excused_users, floor_ulps)

pytestmark = pytest.mark.gpu


def _scd(prob, lam, R=None, d=None, pr=None):
    lt = torch.as_tensor(lam, dtype=torch.float64, device="cuda")
    ln = torch.zeros_like(lt)
    kp.kp_scd_step(prob, lt, ln, R=R, dual_sum=d, primal_sum=pr)
    kp.kp_device_status(prob)
    return ln.cpu().numpy()


@pytest.mark.parametrize("make,N,steps", [
    (gen.hier_m20, 10_000, 6),      # the N=1e6, M=20, K=20 recipe
    (gen.dense_2e7, 20_000, 10),    # the N=2e7, M=10, K=10 recipe
])
def test_scd_trajectory_downscaled(make, N, steps):
    inst = make(N=N, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    p, b = inst.to_dense_numpy()
    B = inst.B.cpu().numpy()
    K = inst.K
    ulps = floor_ulps(inst.layout, K)
    lam = np.zeros(K)
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    d = torch.zeros((), dtype=torch.float64, device="cuda")
    pr = torch.zeros((), dtype=torch.float64, device="cuda")
    for t in range(steps):
        # state at lambda^t (Algorithms 1-2), from the state pass and from the breakpoint pass
        x, Rs, ds, ps, _, _ = cuda_state(prob, torch.tensor(lam, device="cuda"))
        xo, Ro, do, po = oracle.user_pass(p, b, inst.S, inst.C, lam)
        compare_state(p, b, lam, x, Rs, ds, ps, xo, Ro, do, po)
        got = _scd(prob, lam, R, d, pr)
        compare_state(p, b, lam, x, R.cpu().numpy(), float(d), float(pr), xo, Ro, do, po)
        # lambda^{t+1} (Algorithms 3-4)
        want, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
        emis = oracle.scd_map_users(p, b, inst.S, inst.C, lam)
        check_scd_step(got, want, p, b, lam, emis, ulps, label=f"{inst.name} N={N} t={t}",
                       max_loose_share=1.0)
        lam = got


def _sampled_decisions(inst, prob, lam_t, n=2000, seed=17):
    """Algorithm 1 at lam_t for n sampled users against the oracle's greedy; a user may
    differ only if its reduced costs are near zero or near-tied (margin 1e-6)."""
    N, M = inst.N, inst.M
    x = kp.kp_solve_users(prob, lam_t)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(N, size=min(n, N), replace=False))
    p, b = inst.users_dense(idx)
    xs = kp.unpack_x(x.view(N, prob.W)[torch.as_tensor(idx, device="cuda")].reshape(-1), len(idx), M).cpu().numpy()
    lam = lam_t.cpu().numpy()
    xo, _, _, _ = oracle.user_pass(p, b, inst.S, inst.C, lam)
    exc = excused_users(p, b, lam)
    assert np.array_equal(xs[~exc], xo[~exc]), int((xs[~exc] != xo[~exc]).any(axis=1).sum())
    return x


def _dense_recount(inst, x, K):
    """sum_ij b_ijk x_ij in float64 from the GPU's decisions (torch ops, chunked)."""
    N, M = inst.N, inst.M
    W = (M + 31) // 32
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    bv = inst.b.view(N, M, K)
    xw = x.view(N, W)
    step = 1 << 20
    for s in range(0, N, step):
        n = min(step, N - s)
        xs = kp.unpack_x(xw[s:s + n].reshape(-1), n, M).double()
        R += torch.einsum("nm,nmk->k", xs, bv[s:s + n].double())
    return R


def _threshold_rule(inst, prob, lam, nxt, ks):
    """Reduce rule (R6): with the other multipliers at lambda^t, the k-consumption
    just above the selected lambda_k fits B_k and just below it does not."""
    B = inst.B.cpu().numpy()
    lam_h, nxt_h = lam.cpu().numpy(), nxt.cpu().numpy()
    R = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    eps = 1e-5
    for k in ks:
        for f, fits in ((1 + eps, True), (1 - eps, False)):
            l2 = lam_h.copy()
            l2[k] = nxt_h[k] * f
            kp.kp_reduce_consumption(prob, torch.tensor(l2, device="cuda"), R=R)
            assert (float(R[k]) <= B[k]) == fits, (k, f, float(R[k]), B[k])


@pytest.mark.parametrize("which", ["hier_m20_N1e6", "dense_N2e7"])
def test_fullsize_dense(which):
    """The full-size dense workloads: the SCD trajectory (100 iterations for the M=20
    workload, 50 for N=2e7), then at the last lambda^t sampled decisions, the
    consumption recount and the Reduce rule."""
    if which == "hier_m20_N1e6":
        inst, steps = gen.hier_m20(device="cuda"), 100
    else:
        if torch.cuda.get_device_properties(0).total_memory < 40e9:
            pytest.skip("needs a GPU with > 40 GB")
        inst, steps = gen.dense_2e7(device="cuda"), 50
    prob = kp.kp_create_from_instance(inst)
    K = inst.K
    lam = torch.zeros(K, dtype=torch.float64, device="cuda")
    nxt = torch.zeros_like(lam)
    for _ in range(steps - 1):
        kp.kp_scd_step(prob, lam, nxt)
        lam, nxt = nxt, lam
    kp.kp_device_status(prob)
    x = _sampled_decisions(inst, prob, lam)
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    kp.kp_reduce_consumption(prob, lam, R=R)
    Rr = _dense_recount(inst, x, K)
    assert torch.all(torch.abs(R - Rr) <= 1e-9 * Rr + 1e-6), (R, Rr)
    kp.kp_scd_step(prob, lam, nxt)
    kp.kp_device_status(prob)
    pos = np.nonzero(nxt.cpu().numpy() > 0)[0]
    rng = np.random.default_rng(3)
    _threshold_rule(inst, prob, lam, nxt, rng.choice(pos, size=min(4, len(pos)), replace=False))
    prob.close()
    del inst, x
    torch.cuda.empty_cache()


def test_dual_gradient_fd_N2e7():
    """The dual autograd function on the N=2e7, M=10, K=10 workload at full size: at 64
    random lambda ~ U[0.05, 0.2]^K, the Danskin gradient dg/dlambda_k = B_k - R_k and
    the central difference of g at h = 1e-4 (both from the GPU) each lie between the
    slopes B_k - R_k(lambda -/+ h e_k), which bound them because g is convex and
    piecewise linear in lambda_k (Eq. (5)).  Allowances: R within 1e-6 relative, and
    for the difference quotient the FP32 rounding of the two dual values (six standard
    deviations of a sum of independent per-user roundings, each at most
    (K/4 + 6) u sum_{selected j} s_ij, over 2h); dg/dp = x* and dg/dB = lambda."""
    if torch.cuda.get_device_properties(0).total_memory < 40e9:
        pytest.skip("needs a GPU with > 40 GB")
    from paper_2002_00352_gb300.autograd import dual
    inst = gen.dense_2e7(device="cuda")
    prob = kp.kp_create_from_instance(inst)
    N, M, K = inst.N, inst.M, inst.K
    B = inst.B.cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e-4
    u = 2.0 ** -24
    gv = torch.zeros((), dtype=torch.float64, device="cuda")
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    bv = inst.b.view(N, M, K)
    pv = inst.p.view(N, M)

    def value_and_slope(lv):
        kp.kp_reduce_consumption(prob, torch.tensor(lv, device="cuda"), R=R, g=gv)
        return float(gv), B - R.cpu().numpy()

    def rounding_sd(lv, x):
        """sqrt(sum_i e_i^2) with e_i = (K/4 + 6) u sum_{j selected} s_ij."""
        lt = torch.tensor(lv, device="cuda")
        tot = 0.0
        step = 1 << 21
        for s in range(0, N, step):
            sl = pv[s:s + step].detach().double() + torch.einsum("nmk,k->nm", bv[s:s + step].double(), lt)
            xs = kp.unpack_x(x.view(N, -1)[s:s + step].reshape(-1), sl.shape[0], M).double()
            e = (K / 4 + 6) * u * (sl * xs).sum(1)
            tot += float((e * e).sum())
        return tot ** 0.5

    lam_req = torch.zeros(K, dtype=torch.float64, device="cuda", requires_grad=True)
    noise = 0.0
    pg = inst.p.requires_grad_(True)
    Bg = inst.B.requires_grad_(True)
    for trial in range(64):
        lam0 = rng.uniform(0.05, 0.2, size=K)
        with torch.no_grad():
            lam_req.copy_(torch.tensor(lam0))
        g = dual(lam_req, prob)
        gl, gp, gB = torch.autograd.grad(g, [lam_req, pg, Bg])
        gl = gl.cpu().numpy()
        k = trial % K
        e = np.zeros(K)
        e[k] = h
        gp_, lo_hi = value_and_slope(lam0 + e)
        gm_, lo_lo = value_and_slope(lam0 - e)
        fd = (gp_ - gm_) / (2 * h)
        tol_lo = REL * np.abs(B - lo_lo)[k] + 1e-9
        tol_hi = REL * np.abs(B - lo_hi)[k] + 1e-9
        if trial < 4:
            x = kp.kp_solve_users(prob, torch.tensor(lam0, device="cuda"))
            noise = max(noise, 6 * 2 ** 0.5 * rounding_sd(lam0, x) / (2 * h))
            assert np.array_equal(gB.cpu().numpy(), lam0)
            xp = kp.unpack_x(x, N, M).view(-1).float()
            assert torch.equal(gp.view(-1), xp)
        assert lo_lo[k] - tol_lo - noise <= fd <= lo_hi[k] + tol_hi + noise, (trial, lo_lo[k], fd, lo_hi[k], noise)
        assert lo_lo[k] - tol_lo <= gl[k] <= lo_hi[k] + tol_hi, (trial, lo_lo[k], gl[k], lo_hi[k])
    prob.close()
