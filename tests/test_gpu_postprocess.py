"""GPU parity of the post-processing for feasibility (Sec. 5.4): kp_postprocess
through the C ABI against the oracle's postprocess on the same x.

The decisions given to both sides come from the seeded generator or from the
oracle's own greedy; the number of users reset and the returned x must match
exactly, R_after within the fixed-point rounding of the consumption sums.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_00352_gb300 import gen, kp

pytestmark = pytest.mark.gpu


def _pack(x):
    """[N, M] 0/1 -> int32 words, W = ceil(M/32) per user (bit j%32 of word j/32)."""
    N, M = x.shape
    W = (M + 31) // 32
    words = np.zeros((N, W), dtype=np.uint64)
    for j in range(M):
        words[:, j // 32] |= x[:, j].astype(np.uint64) << np.uint64(j % 32)
    return torch.tensor(words.astype(np.uint32).view(np.int32).reshape(-1), device="cuda")


def _gpu(prob, lam, x):
    xb = _pack(x)
    reset, R_after = kp.kp_postprocess(prob, torch.tensor(lam, dtype=torch.float64, device="cuda"), xb)
    kp.kp_device_status(prob)
    return kp.unpack_x(xb, x.shape[0], x.shape[1]).cpu().numpy(), int(reset), R_after.cpu().numpy()


def _check(p, b, lam, B, x, got, expect_reset=None):
    xg, rg, Rg = got
    xo, ro = oracle.postprocess(p, b, lam, B, x)
    assert rg == ro, (rg, ro)
    assert np.array_equal(xg, xo.astype(np.uint8))
    if expect_reset is not None:
        assert ro == expect_reset
    R_o = np.einsum("nmk,nm->k", b.astype(np.float64), xo.astype(np.float64))
    # per entry the fixed point rounds by at most 2^-30 of the largest b's power of two
    atol = max(1, int(xo.sum())) * b.shape[2] * float(b.max()) * 2.0 ** -29
    assert np.allclose(Rg, R_o, rtol=1e-12, atol=atol)
    assert np.all(Rg <= B * (1 + 1e-12))
    return ro


def _budgets(R, rng, lo=0.3, hi=1.2):
    return np.maximum(R * rng.uniform(lo, hi, size=R.shape[0]), 1e-3)


@pytest.mark.parametrize("layout", ["dense", "csr"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_postprocess_random_x(layout, seed):
    """Arbitrary decisions (not the greedy's) and multipliers; some knapsacks over
    budget, some not; N = 3001 spans many blocks and a ragged tail (CSR: 0 to 3
    entries per item)."""
    rng = np.random.default_rng(seed)
    M, K, N = int(rng.integers(2, 12)), int(rng.integers(1, 9)), 3001
    inst = gen.random_small(N, M, K, seed=seed, device="cuda", layout=layout)
    p, b = inst.to_dense_numpy()
    x = (rng.random((N, M)) < 0.5).astype(np.int32)
    R = np.einsum("nmk,nm->k", b, x.astype(np.float64))
    B = _budgets(R, rng)
    inst.B = torch.tensor(B, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    lam = rng.uniform(0, 0.6, size=K) * (rng.random(K) < 0.8)
    r = _check(p, b, lam, B, x, _gpu(prob, lam, x))
    assert r > 0


def test_postprocess_csr_wide_rows():
    """CSR with M = 16 and up to 48 entries per user: some tiles of 256 users hold
    more entries than the shared-memory stage and are read from global memory."""
    rng = np.random.default_rng(4)
    N, M, K = 3001, 16, 6
    inst = gen.random_small(N, M, K, seed=4, device="cuda", layout="csr")
    p, b = inst.to_dense_numpy()
    x = (rng.random((N, M)) < 0.5).astype(np.int32)
    R = np.einsum("nmk,nm->k", b, x.astype(np.float64))
    B = _budgets(R, rng)
    inst.B = torch.tensor(B, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    lam = rng.uniform(0, 0.3, size=K)
    assert _check(p, b, lam, B, x, _gpu(prob, lam, x)) > 0


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_postprocess_greedy_x(layout):
    """x = the oracle's Algorithm 1 decisions at lambda = 0 and at a small lambda
    (the situation of Sec. 5.4: a dual solution that overfills)."""
    if layout == "dense":
        inst = gen.small_dd_scd(device="cuda")
    else:
        inst = gen.sparse_csr(N=20_000, device="cuda", K=24)
    prob = kp.kp_create_from_instance(inst)
    p, b = inst.to_dense_numpy()
    B = inst.B.cpu().numpy()
    for scale in (0.0, 0.05):
        lam = np.full(inst.K, scale)
        xo, _, _, _ = oracle.user_pass(p, b, inst.S, inst.C, lam)
        xo = np.asarray(xo, dtype=np.int32)
        r = _check(p, b, lam, B, xo, _gpu(prob, lam, xo))
        assert r > 0


def test_postprocess_feasible_and_all_reset():
    """Budgets above the consumption: nothing reset, x unchanged.  Budgets below
    every user's consumption: every consuming user is reset."""
    rng = np.random.default_rng(7)
    N, M, K = 777, 5, 3
    inst = gen.random_small(N, M, K, seed=7, device="cuda", layout="dense")
    p, b = inst.to_dense_numpy()
    x = (rng.random((N, M)) < 0.5).astype(np.int32)
    R = np.einsum("nmk,nm->k", b, x.astype(np.float64))
    lam = np.array([0.1, 0.0, 0.3])
    for B, want in ((R * 2 + 1.0, 0), (np.full(K, 1e-9), None)):
        inst.B = torch.tensor(B, device="cuda")
        prob = kp.kp_create_from_instance(inst)
        got = _gpu(prob, lam, x)
        r = _check(p, b, lam, B, x, got, expect_reset=want)
        if want == 0:
            assert np.array_equal(got[0], x.astype(np.uint8))
        else:
            assert r > 0 and np.all(np.einsum("nmk,nm->k", b, got[0].astype(np.float64)) == 0)


def test_postprocess_equal_keys_lower_index_first():
    """Users with identical rows have equal group profits: the lower index is
    reset first (R7); one budget crossing inside the tied run decides the count."""
    rng = np.random.default_rng(8)
    N, M, K = 600, 4, 2
    p1 = rng.random((3, M)).astype(np.float32)
    b1 = rng.random((3, M, K)).astype(np.float32)
    pick = rng.integers(0, 3, size=N)
    p = p1[pick]
    b = b1[pick]
    x = np.tile((rng.random((1, M)) < 0.7).astype(np.int32), (N, 1))
    x[:, 0] = 1
    R = np.einsum("nmk,nm->k", b.astype(np.float64), x.astype(np.float64))
    B = R * np.array([0.55, 0.8])
    tp, tb = torch.tensor(p, device="cuda"), torch.tensor(b, device="cuda")
    tB = torch.tensor(B, device="cuda")
    prob = kp.kp_create(N, M, K, tp.reshape(-1), tB, [], [], b_dense=tb.reshape(-1))
    lam = np.array([0.25, 0.5])
    _check(p, b, lam, B, x, _gpu(prob, lam, x))


def test_postprocess_all_users_identical():
    """Every key equal (no key bit separates the users): the order is the user
    index alone."""
    rng = np.random.default_rng(10)
    N, M, K = 257, 3, 2
    p = np.tile(rng.random((1, M)).astype(np.float32), (N, 1))
    b = np.tile(rng.random((1, M, K)).astype(np.float32), (N, 1, 1))
    x = np.tile(np.array([[1, 0, 1]], dtype=np.int32), (N, 1))
    R = np.einsum("nmk,nm->k", b.astype(np.float64), x.astype(np.float64))
    B = R * np.array([0.61, 0.93])
    tp, tb = torch.tensor(p, device="cuda"), torch.tensor(b, device="cuda")
    prob = kp.kp_create(N, M, K, tp.reshape(-1), torch.tensor(B, device="cuda"), [], [],
                        b_dense=tb.reshape(-1))
    lam = np.array([0.125, 0.5])
    r = _check(p, b, lam, B, x, _gpu(prob, lam, x))
    assert 0 < r < N


@pytest.mark.parametrize("K,hi", [(900, 1.1), (2048, 0.9)])
def test_postprocess_many_knapsacks_narrow_digits(K, hi):
    """Many knapsacks over budget: the per-digit sums leave room for 4-bit
    (K = 900, about 750 over budget) or 3-bit digits (K = 2048, all over)."""
    rng = np.random.default_rng(9)
    N, M = 300, 2
    inst = gen.random_small(N, M, K, seed=9, device="cuda", layout="dense")
    p, b = inst.to_dense_numpy()
    x = (rng.random((N, M)) < 0.6).astype(np.int32)
    R = np.einsum("nmk,nm->k", b, x.astype(np.float64))
    B = _budgets(R, rng, 0.5, hi)
    inst.B = torch.tensor(B, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    lam = rng.uniform(0, 0.01, size=K)
    assert _check(p, b, lam, B, x, _gpu(prob, lam, x)) > 0


@pytest.mark.parametrize("N", [1, 2, 33])
def test_postprocess_tiny(N):
    rng = np.random.default_rng(N)
    M, K = 3, 2
    inst = gen.random_small(N, M, K, seed=N, device="cuda", layout="dense")
    p, b = inst.to_dense_numpy()
    x = np.ones((N, M), dtype=np.int32)
    R = np.einsum("nmk,nm->k", b, x.astype(np.float64))
    B = np.maximum(R * 0.5, 1e-6)
    inst.B = torch.tensor(B, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    _check(p, b, np.array([0.0, 0.2]), B, x, _gpu(prob, np.array([0.0, 0.2]), x))


def test_postprocess_csr_large():
    """N = 2e6 CSR (M = 10, two entries per item, K = 200) at a small lambda, x
    from kp_solve_users: the bench's shape at 1/50 scale, too large for the
    oracle.  Checked instead, with keys and consumption recomputed in FP64 by
    torch: the returned x fits every budget and R_after is its consumption; the
    users reset are whole users whose keys are at most every kept consuming
    user's; putting back the last one reset overfills some knapsack (the prefix
    is the shortest); the count is the number of users ordered before it."""
    N, M, Cn = 2_000_000, 10, 2
    inst = gen.regular_csr(N, M, 200, Cn, seed=21, device="cuda")
    prob = kp.kp_create_from_instance(inst)
    lam = torch.full((inst.K,), 0.02, dtype=torch.float64, device="cuda")
    xb = kp.kp_solve_users(prob, lam)
    x0 = kp.unpack_x(xb, N, M).bool()
    reset, R_after = kp.kp_postprocess(prob, lam, xb)
    kp.kp_device_status(prob)
    x1 = kp.unpack_x(xb, N, M).bool()
    r = int(reset)
    B = inst.B
    val = inst.val.view(N, M, Cn).double()
    kk = inst.kidx.view(N, M, Cn).long()
    q = ((inst.p.view(N, M).double() - (lam[kk] * val).sum(-1)) * x0).sum(1)
    R1 = torch.zeros(inst.K, dtype=torch.float64, device="cuda")
    R1.index_add_(0, kk[x1].reshape(-1), val[x1].reshape(-1))
    assert torch.allclose(R_after, R1, rtol=1e-7, atol=1e-6)
    assert bool((R_after <= B).all())
    R0 = torch.zeros_like(R1).index_add_(0, kk[x0].reshape(-1), val[x0].reshape(-1))
    assert r > 0 and bool((R0 > B).any())
    changed = (x0 != x1).any(1)
    assert not bool(x1[changed].any())
    consuming = x0.any(1)
    gone = changed & consuming
    kept = ~changed & consuming
    qt = q[gone].max()
    assert bool(qt <= q[kept].min() + 1e-9)
    t = int(torch.nonzero(gone & (q == qt))[-1])
    cons_t = torch.zeros_like(R1).index_add_(0, kk[t][x0[t]].reshape(-1), val[t][x0[t]].reshape(-1))
    assert bool(((R_after + cons_t) > B).any())
    eps = 1e-9 * float(qt.abs()) + 1e-12
    lo = int((q < qt - eps).sum())
    hi = int((q <= qt + eps).sum())
    assert lo < r <= hi, (lo, r, hi)
