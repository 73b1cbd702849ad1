"""Helpers for the GPU parity tests: tolerances derived from the arithmetic.

The CUDA path computes reduced costs in FP32 (lambda rounded to FP32, a few
partial sums), the oracle in FP64.  The FP32 reduced cost of item j has an
error well below 1e-6 * s_j with s_j = p_j + sum_k lambda_k b_jk (at most
~10 roundings of quantities bounded by s_j), so every decision whose margin
exceeds TAU * (s_j + s_j') must agree exactly.  Users with a smaller margin
(near-zero p~ or two nearly tied p~) are "excused": their decisions may
differ, and the consumption / objective comparisons allow for exactly their
contribution on top of 1e-6 relative.
"""
import numpy as np
import torch

TAU = 1e-6
REL = 1e-6       # consumption, dual and primal
REL_LAMBDA = 1e-5


def excused_users(p, b, lam, tau=TAU):
    """Boolean [N]: users with a near-zero or near-tied reduced cost."""
    pt = p - np.einsum("ijk,k->ij", b, lam)
    s = p + np.einsum("ijk,k->ij", b, lam)
    near0 = np.abs(pt) <= tau * s
    d = np.abs(pt[:, :, None] - pt[:, None, :])
    ss = s[:, :, None] + s[:, None, :]
    M = pt.shape[1]
    off = ~np.eye(M, dtype=bool)[None]
    neartie = ((d <= tau * ss) & off).any(axis=2)
    return (near0 | neartie).any(axis=1)


def compare_state(p, b, lam, x_gpu, R_gpu, dual_gpu, primal_gpu, x_o, R_o, dual_o, primal_o):
    """Asserts decision / consumption / objective parity; returns #excused users."""
    exc = excused_users(p, b, lam)
    ok = ~exc
    assert np.array_equal(x_gpu[ok], x_o[ok]), \
        f"{int((x_gpu[ok] != x_o[ok]).any(axis=1).sum())} non-excused users differ"
    slackR = b[exc].sum(axis=(0, 1)) if exc.any() else np.zeros(b.shape[2])
    assert np.all(np.abs(R_gpu - R_o) <= REL * np.abs(R_o) + slackR + 1e-9), (R_gpu, R_o)
    s = p + np.einsum("ijk,k->ij", b, lam)
    slackD = 2 * TAU * s[exc].sum() if exc.any() else 0.0
    slackP = p[exc].sum() if exc.any() else 0.0
    assert abs(dual_gpu - dual_o) <= REL * abs(dual_o) + slackD + 1e-9
    assert abs(primal_gpu - primal_o) <= REL * abs(primal_o) + slackP + 1e-9
    return int(exc.sum())


def lam_close(a, b, rel=REL_LAMBDA, abs_floor=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) <= rel * np.maximum(np.abs(b), np.abs(a)) + abs_floor


def lam_close_fp32(got, want, p, b, lam_t, rel=REL_LAMBDA):
    """lam_close with the floor of a FP32 breakpoint lambda_k^t + m / b_jk: its
    absolute error is a few ulps of s_j / b_jk (s_j = p_j + sum_k lambda_k b_jk,
    the scale of the reduced cost), which shows when a threshold lands far
    below lambda_k^t or the other quantities of its users."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    s = p + np.einsum("ijk,k->ij", b, lam_t)
    s_over_b = np.where(b > 0, s[:, :, None] / np.where(b > 0, b, 1.0), 0.0)
    floor = 4 * 2.0 ** -24 * s_over_b.max(axis=(0, 1))
    return np.abs(got - want) <= rel * np.maximum(np.abs(got), np.abs(want)) + floor + 1e-12


def cuda_state(prob, lam_t):
    from paper_2002_00352_gb300 import kp
    K = prob.K
    R = torch.zeros(K, dtype=torch.float64, device="cuda")
    d = torch.zeros((), dtype=torch.float64, device="cuda")
    pr = torch.zeros((), dtype=torch.float64, device="cuda")
    g = torch.zeros((), dtype=torch.float64, device="cuda")
    x = torch.zeros(prob.N * prob.W, dtype=torch.int32, device="cuda")
    kp.kp_reduce_consumption(prob, lam_t, R=R, dual_sum=d, primal_sum=pr, g=g, x_bits=x)
    torch.cuda.synchronize()
    xs = kp.unpack_x(x, prob.N, prob.M).cpu().numpy().astype(np.int32)
    return xs, R.cpu().numpy(), float(d), float(pr), float(g), x
