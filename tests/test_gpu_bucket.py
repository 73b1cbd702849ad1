"""The bucketed Reduce of Sec. 5.2 (kp_scd_step_bucketed) against the oracle.

The bucket of a breakpoint is an integer decided by FP32 arithmetic on the
breakpoint.  The GPU's FP32 breakpoint differs from the oracle's FP64 one by
its local rounding error (a few u times the candidate's scale, as in the
local floors of the SCD parity tests) plus its own FP32 rounding, so a
breakpoint that close to a bucket boundary may fall on either side.  The
oracle brackets the GPU's result by running its Reduce twice, once with every
such breakpoint in its lower possible bucket and once in its upper one (the
buckets are monotone in v, and moving mass upward never lowers the
interpolated threshold).  The GPU's value must lie between the two, within
1e-6 relative (fixed-point masses, FP32 pair masses, FP64 interpolation).
The instances and multipliers are chosen with no user whose decision is
excused (near-zero or near-tied reduced costs), so both sides emit the same
breakpoints.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp
from tests.gpu_util import EPS32, emission_scale, excused_users, floor_ulps
from tests.helpers import random_laminar

pytestmark = pytest.mark.gpu


def _case(layout):
    """(instance, the multipliers lambda^t tested).  CSR: the sparse workload's shape
    at N = 6000; dense: a random laminar family over 8 items.  Candidates: the
    oracle's SCD iterates from 0 and scaled copies of them; the first two with no
    excused user and a positive next threshold are tested (the instance depends on
    the device's random stream, so the choice is made here)."""
    if layout == "csr":
        inst = gen.sparse_csr(N=6000, K=8, seed=5, device="cuda")
    else:
        rng = np.random.default_rng(71)
        inst = gen.random_small(3000, 8, 5, seed=71, device="cuda", layout="dense", frac=0.15)
        inst.S, inst.C = random_laminar(8, rng, max_nodes=4)
    p, b = inst.to_dense_numpy()
    B = inst.B.cpu().numpy()
    traj = [np.zeros(inst.K)]
    for _ in range(4):
        traj.append(oracle.scd_step(p, b, inst.S, inst.C, traj[-1], B)[0])
    cands = traj + [c * l for c in (0.3, 0.97, 1.03) for l in traj[1:3]]
    lams = []
    for lam in cands:
        if len(lams) == 2:
            break
        if any(np.array_equal(lam, l) for l in lams) or excused_users(p, b, lam).any():
            continue
        if not np.any(oracle.scd_step(p, b, inst.S, inst.C, lam, B)[0] > 0):
            continue
        lams.append(lam)
    assert lams, "no candidate multipliers without excused users"
    return inst, p, b, B, lams


def bracket(p, b, S, C, lam, B, delta, ulps):
    """(lower, upper) oracle thresholds with the ambiguous breakpoints moved to their
    lower / upper possible bucket, and the number of ambiguous breakpoints."""
    u, ek, v1, v2 = oracle.scd_map_users(p, b, S, C, lam)
    K = len(lam)
    low, high = np.zeros(K), np.zeros(K)
    namb = 0
    for k in range(K):
        sel = np.nonzero(ek == k)[0]
        dk = oracle.bucket_delta(lam[k], delta)
        x = v1[sel]
        ids = oracle.bucket_ids(x, lam[k], dk)
        # coarse screen, then each candidate's own error bound
        r = 1e-3
        near = np.nonzero((oracle.bucket_ids(x * (1 - r), lam[k], dk) != ids)
                          | (oracle.bucket_ids(x * (1 + r), lam[k], dk) != ids))[0]
        ilo, ihi = ids.copy(), ids.copy()
        for q in near:
            e = sel[q]
            err = ulps * EPS32 * emission_scale(p[u[e]], b[u[e]], lam, k, v1[e]) + 2.0 ** -23 * abs(v1[e])
            a = oracle.bucket_ids(np.array([v1[e] - err, v1[e] + err]), lam[k], dk)
            ilo[q], ihi[q] = a[0], a[1]
            namb += int(a[0] != a[1])
        low[k] = oracle.bucket_reduce(x, v2[sel], B[k], lam[k], dk, ids=ilo)
        high[k] = oracle.bucket_reduce(x, v2[sel], B[k], lam[k], dk, ids=ihi)
    return low, high, namb


@pytest.mark.parametrize("layout", ["csr", "dense"])
def test_bucketed_step_matches_oracle(layout):
    inst, p, b, B, lams = _case(layout)
    prob = kp.kp_create_from_instance(inst)
    for lam in lams:
        lt = torch.tensor(lam, device="cuda")
        for delta in (1e-3, 0.05, 0.5):
            out = torch.zeros_like(lt)
            kp.kp_scd_step_bucketed(prob, lt, delta, out)
            kp.kp_device_status(prob)
            got = out.cpu().numpy()
            low, high, namb = bracket(p, b, inst.S, inst.C, lam, B, delta, floor_ulps(inst.layout, inst.K))
            assert np.any(high > 0)
            tol = 1e-6 * np.maximum(np.abs(low), np.abs(high)) + 1e-12
            print(f"{layout} delta={delta}: ambiguous breakpoints {namb}, "
                  f"largest bracket {np.max(high - low):.3g}")
            assert np.all(got >= low - tol) and np.all(got <= high + tol), (delta, got, low, high)


def test_bucketed_step_leaves_the_exact_step_alone():
    """A bucketed step between two exact steps changes neither their results nor
    the threshold prediction: the exact trajectory with bucketed steps interleaved
    equals the plain one bit for bit; delta outside (0, 1e30] is rejected."""
    inst = gen.sparse_csr(N=6000, K=8, seed=5, device="cuda")
    lam0 = torch.zeros(inst.K, dtype=torch.float64, device="cuda")

    def run(interleave):
        prob = kp.kp_create_from_instance(inst)
        lam, out = lam0.clone(), torch.zeros_like(lam0)
        traj = []
        for _ in range(4):
            if interleave:
                kp.kp_scd_step_bucketed(prob, lam, 0.01, torch.zeros_like(lam))
            kp.kp_scd_step(prob, lam, out)
            lam, out = out.clone(), lam
            traj.append(lam.cpu().numpy())
        kp.kp_device_status(prob)
        return np.array(traj), prob

    a, _ = run(False)
    c, prob = run(True)
    assert np.array_equal(a, c)
    for bad in (0.0, -1.0, float("inf"), float("nan"), 1e31):
        with pytest.raises(kp.KpError):
            kp.kp_scd_step_bucketed(prob, lam0, bad, torch.zeros_like(lam0))
