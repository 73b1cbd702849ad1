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


# Local FP32 floor of a breakpoint.  The GPU computes every breakpoint in FP32
# from reduced costs p~_j (FP32, error <= (2 + n_terms) u s_j with u = 2^-24 and
# s_j = p_j + sum_k lambda_k b_jk, n_terms = the partial sums of the item's
# entries), as (a_j - a_j') / (b_jk - b_j'k) in the notation of Algorithm 3
# (a_j' = theta_j, b_j'k = 0 for a crossing with a fixed line; a_j' = 0 for a
# zero crossing).  Its absolute error is then a few u times the candidate's
# scale (s_j + s_j') / |b_jk - b_j'k|, on top of a few u of its own value.  Only
# breakpoints next to the selected threshold can move it, so the floor of
# knapsack k is that error for the emissions near lambda_k^{t+1}, not the worst
# entry of the instance.
EPS32 = 2.0 ** -24
BAND = 1e-3      # "near": within 1e-3 relative of the oracle's or the GPU's threshold


def floor_ulps(layout, K):
    """Units of u in the local floor: 8 for CSR rows (at most 2 terms per item),
    2 (K/4 + 4) + 3 for dense rows (four partial sums of K/4 terms each)."""
    return 8.0 if layout == "csr" else 2.0 * (np.ceil(K / 4.0) + 4.0) + 3.0


def emission_scale(p_i, b_i, lam_t, k, v1):
    """Scale (s_j + s_j') / |b_jk - b_j'k| of the Algorithm 3 candidate(s) equal to the
    emitted breakpoint v1 of one user in knapsack k (largest if several coincide;
    the largest of the user's candidates if none matches, which does not happen for
    the oracle's own emissions)."""
    s_tot = p_i + b_i @ lam_t
    sl = b_i[:, k]
    a = p_i - b_i @ lam_t + lam_t[k] * sl
    M = len(p_i)
    jj, kk = np.triu_indices(M, 1)
    cand = [np.where(sl > 0, a / np.where(sl > 0, sl, 1.0), np.nan)]
    scale = [np.where(sl > 0, s_tot / np.where(sl > 0, sl, 1.0), 0.0)]
    ds = sl[jj] - sl[kk]
    ok = ds != 0
    cand.append(np.where(ok, (a[jj] - a[kk]) / np.where(ok, ds, 1.0), np.nan))
    scale.append(np.where(ok, (s_tot[jj] + s_tot[kk]) / np.where(ok, np.abs(ds), 1.0), 0.0))
    cand = np.concatenate(cand)
    scale = np.concatenate(scale)
    match = np.abs(cand - v1) <= 1e-9 * abs(v1)
    return float(scale[match].max()) if match.any() else float(scale.max())


def local_floor(got, want, p, b, lam_t, emis, ulps):
    """Per-knapsack absolute floor: ulps * u * the largest emission_scale over the
    emissions (user, k, v1, v2 from the oracle's Map at lam_t) whose v1 lies within
    BAND of want_k or got_k."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    u, ks, v1, _ = emis
    K = len(want)
    out = np.zeros(K)
    near = (np.abs(v1 - want[ks]) <= BAND * want[ks]) | (np.abs(v1 - got[ks]) <= BAND * got[ks])
    for e in np.nonzero(near)[0]:
        k = int(ks[e])
        out[k] = max(out[k], emission_scale(p[u[e]], b[u[e]], lam_t, k, v1[e]))
    return ulps * EPS32 * out


def lam_close_local(got, want, floor, rel=REL_LAMBDA):
    """|got - want| <= rel * max(|got|, |want|) + the local floor (+1e-12)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return np.abs(got - want) <= rel * np.maximum(np.abs(got), np.abs(want)) + floor + 1e-12


def floor_report(floor, want, lam_t):
    """(largest floor, largest floor / lambda_k over the knapsacks with lambda_k > 0,
    share of those where the floor exceeds 1e-5 lambda_k among the ones whose
    threshold is not far below lambda_k^t (lambda_k >= 1e-2 lambda_k^t))."""
    want = np.asarray(want, dtype=np.float64)
    pos = want > 0
    if not pos.any():
        return 0.0, 0.0, 0.0
    ratio = floor[pos] / want[pos]
    regular = pos & (want >= 1e-2 * np.asarray(lam_t, dtype=np.float64))
    share = float((floor[regular] > REL_LAMBDA * want[regular]).mean()) if regular.any() else 0.0
    return float(floor.max()), float(ratio.max()), share


def check_scd_step(got, want, p, b, lam_t, emis, ulps, label="", max_loose_share=0.05,
                   excused_k=None):
    """Asserts lam_close_local per knapsack (knapsacks in excused_k, touched by a user
    whose decisions are excused, may take a neighbouring breakpoint instead) and that
    the floor is below 1e-5 lambda_k on all but max_loose_share of the regular
    knapsacks; prints the effective floor."""
    floor = local_floor(got, want, p, b, lam_t, emis, ulps)
    ok = lam_close_local(got, want, floor)
    if excused_k is not None:
        ok |= excused_k
    fmax, rmax, share = floor_report(floor, want, lam_t)
    print(f"[{label}] local floor max {fmax:.3e}, max floor/lambda {rmax:.3e}, "
          f"share above 1e-5 lambda {share:.3f}")
    assert ok.all(), (label, np.nonzero(~ok)[0], got[~ok], want[~ok], floor[~ok])
    assert share <= max_loose_share, (label, share)
    return floor


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
