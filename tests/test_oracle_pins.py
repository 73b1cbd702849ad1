"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle routine against something other than itself:
exhaustive search, a closed form, a textbook special case, an invariant or a
duality bound.  Marked "not gpu" (no marker): runs on CPU.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.helpers import feasible_local, random_laminar


# ---------------------------------------------------------------------------
# Algorithm 1 / Proposition 1
# ---------------------------------------------------------------------------

def test_hierarchical_definition():
    # Sec. 2.1, Definition 1
    assert oracle.is_hierarchical([0b0011, 0b1100, 0b1111])
    assert oracle.is_hierarchical([0b0011, 0b0011])
    assert not oracle.is_hierarchical([0b0011, 0b0110])


@pytest.mark.parametrize("seed", range(40))
def test_greedy_is_optimal_vs_brute_force(seed):
    """Proposition 1: Algorithm 1 solves Eq. (11)-(13) optimally (exchange argument);
    checked by exhaustive 2^M search on random hierarchical families."""
    rng = np.random.default_rng(seed)
    M = int(rng.integers(1, 13))
    S, C = random_laminar(M, rng)
    assert oracle.is_hierarchical(S)
    for _ in range(20):
        pt = rng.normal(size=M)
        if rng.random() < 0.3:  # ties
            pt = np.round(pt, 1)
        x = oracle.greedy(pt, S, C)
        mask = sum(1 << j for j in range(M) if x[j])
        assert feasible_local(mask, S, C)
        assert np.all(pt[x == 1] > 0)
        best, _ = oracle.brute_force(pt, S, C)
        assert float(pt @ x) == pytest.approx(best, abs=1e-12)


def _walk_greedy(pt, S, C):
    """Second, independent form of the greedy: visit items by non-increasing p~
    (ties: lower index) and accept an item if p~ > 0 and every set containing it
    still has room.  Equivalent to Algorithm 1's bottom-up pass for laminar sets."""
    M = len(pt)
    order = sorted(range(M), key=lambda j: (-pt[j], j))
    cnt = [0] * len(S)
    x = [0] * M
    for j in order:
        if pt[j] <= 0:
            continue
        if all(cnt[l] < C[l] for l in range(len(S)) if (S[l] >> j) & 1):
            x[j] = 1
            for l in range(len(S)):
                if (S[l] >> j) & 1:
                    cnt[l] += 1
    return np.array(x)


@pytest.mark.parametrize("seed", range(40))
def test_greedy_two_forms_agree(seed):
    rng = np.random.default_rng(100 + seed)
    M = int(rng.integers(1, 20))
    S, C = random_laminar(M, rng, max_nodes=8)
    for _ in range(30):
        pt = np.round(rng.normal(size=M), 1)  # many exact ties
        assert np.array_equal(oracle.greedy(pt, S, C), _walk_greedy(pt, S, C))


def test_greedy_sort_direction_and_caps():
    """Algorithm 1 keeps the LARGEST cost-adjusted profits (reading R1) and counts
    items against C_l (reading R2)."""
    pt = np.array([0.1, 0.5, 0.3, -0.2, 0.4])
    S = [0b00111, 0b11111]  # {0,1,2} cap 1, all cap 2
    C = [1, 2]
    x = oracle.greedy(pt, S, C)
    # group {0,1,2}: keep item 1 (0.5); overall cap 2: items 1 and 4 (0.4)
    assert x.tolist() == [0, 1, 0, 0, 1]


def test_reduced_costs_closed_form():
    p = np.array([1.0, 2.0])
    b = np.array([[0.5, 0.25], [1.0, 0.0]])
    lam = np.array([2.0, 4.0])
    assert oracle.reduced_costs(p, b, lam).tolist() == [1.0 - 1.0 - 1.0, 2.0 - 2.0]


# ---------------------------------------------------------------------------
# Algorithms 3-4 Map: the per-user step function of k-consumption in lambda_k
# ---------------------------------------------------------------------------

def _consumption_bf(p_i, b_i, S, C, lam, k, lk):
    lam2 = lam.copy()
    lam2[k] = lk
    pt = p_i - b_i @ lam2
    _, x = oracle.brute_force(pt, S, C)
    return float(b_i[:, k] @ x)


@pytest.mark.parametrize("seed", range(25))
def test_scd_map_is_the_consumption_step_function(seed):
    """The pairs emitted by the Map of Algorithm 4 describe the user's k-consumption as
    lambda_k varies with the other multipliers fixed: at any generic lambda_k,
    consumption = sum of v2 over emitted v1 > lambda_k (reading R4).  The consumption
    is computed here by exhaustive search, independent of Algorithm 1."""
    rng = np.random.default_rng(200 + seed)
    M = int(rng.integers(1, 8))
    K = int(rng.integers(1, 4))
    S, C = random_laminar(M, rng)
    p_i = rng.uniform(0, 1, size=M)
    b_i = rng.uniform(0, 1, size=(M, K)) * (rng.random((M, K)) < 0.7)
    lam = rng.uniform(0, 0.8, size=K)
    ek, v1, v2 = oracle.scd_map_user(p_i, b_i, S, C, lam)
    assert np.all(v2 > 0)          # consumption never decreases as lambda_k decreases
    assert np.all(v1 > 0)
    for k in range(K):
        sel = ek == k
        for lk in rng.uniform(0, 3.0, size=25):
            if sel.any() and np.min(np.abs(v1[sel] - lk)) < 1e-9:
                continue
            want = _consumption_bf(p_i, b_i, S, C, lam, k, lk)
            got = float(v2[sel & (v1 > lk)].sum())
            assert got == pytest.approx(want, abs=1e-9)
        # at lambda_k -> infinity the user consumes nothing of k
        assert _consumption_bf(p_i, b_i, S, C, lam, k, 1e9) == 0.0


@pytest.mark.parametrize("seed", range(6))
def test_scd_map_all_users_is_each_users_step_function(seed):
    """The all-users listing of the Map (users split over threads) describes every
    listed user's k-consumption step function, checked by exhaustive search as
    above, and its Reduce per k is the step of Algorithm 4."""
    rng = np.random.default_rng(900 + seed)
    N = 7
    M = int(rng.integers(1, 7))
    K = int(rng.integers(1, 4))
    S, C = random_laminar(M, rng)
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K)) * (rng.random((N, M, K)) < 0.7)
    lam = rng.uniform(0, 0.8, size=K)
    eu, ek, v1, v2 = oracle.scd_map_users(p, b, S, C, lam)
    assert np.all(np.diff(eu) >= 0)
    for i in range(N):
        for k in range(K):
            sel = (eu == i) & (ek == k)
            for lk in rng.uniform(0, 3.0, size=10):
                if sel.any() and np.min(np.abs(v1[sel] - lk)) < 1e-9:
                    continue
                want = _consumption_bf(p[i], b[i], S, C, lam, k, lk)
                assert float(v2[sel & (v1 > lk)].sum()) == pytest.approx(want, abs=1e-9)
    B = rng.uniform(0.2, 2.0, size=K)
    step, _, _ = oracle.scd_step(p, b, S, C, lam, B)
    for k in range(K):
        assert oracle.scd_reduce(v1[ek == k], v2[ek == k], B[k]) == step[k]
    sub = oracle.scd_map_users(p, b, S, C, lam, users=[5, 2])
    assert set(sub[0].tolist()) <= {2, 5}


def test_scd_map_single_item_closed_form():
    """One item, one knapsack, no local constraint: the only breakpoint is the zero
    crossing p/b, with jump b (Algorithm 3's zero-crossing candidate)."""
    ek, v1, v2 = oracle.scd_map_user([0.6], [[0.3]], [], [], [0.0])
    assert ek.tolist() == [0] and v1 == pytest.approx([2.0]) and v2 == pytest.approx([0.3])


def test_scd_map_two_items_cap_one_hand_example():
    """Two items sharing one knapsack under a cap of 1 (MCKP-like user).
    z_0 = 1 - 0.5 l, z_1 = 0.8 - 0.1 l.  Zero crossings: 2 and 8; crossing:
    (1-0.8)/(0.5-0.1) = 0.5.  For l > 8 nothing; 0.5 < l < 8: item 1 (0.1);
    l < 0.5: item 0 (0.5).  Emissions: (8, 0.1), (0.5, 0.4)."""
    ek, v1, v2 = oracle.scd_map_user([1.0, 0.8], [[0.5], [0.1]], [0b11], [1], [0.0])
    assert v1.tolist() == pytest.approx([8.0, 0.5])
    assert v2.tolist() == pytest.approx([0.1, 0.4])


# ---------------------------------------------------------------------------
# Algorithm 4 Reduce (reading R6)
# ---------------------------------------------------------------------------

def _reduce_bf(v1, v2, B):
    cands = sorted(set([0.0] + list(v1)))
    for v in cands:  # smallest first
        if sum(m for a, m in zip(v1, v2) if a > v) <= B:
            return v
    raise AssertionError


@pytest.mark.parametrize("seed", range(30))
def test_scd_reduce_matches_definition(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(0, 40))
    v1 = np.round(rng.uniform(0.01, 2, size=n), 2)   # repeated values
    v2 = rng.uniform(0.01, 1, size=n)
    B = float(rng.uniform(0, max(v2.sum(), 0.1) * 1.2))
    assert oracle.scd_reduce(v1, v2, B) == _reduce_bf(list(v1), list(v2), B)


def test_dantzig_critical_ratio_K1_M1():
    """Sec. 4.4: for K=1 SCD is the rounded fractional knapsack.  With M=1, L=0 the
    threshold equals Dantzig's critical ratio: sort users by p/b decreasingly and
    stop at the first whose b no longer fits in B."""
    rng = np.random.default_rng(7)
    N = 500
    p = rng.uniform(0, 1, size=(N, 1))
    b = rng.uniform(0.05, 1, size=(N, 1, 1))
    B = np.array([0.3 * b.sum()])
    lam1, _, _ = oracle.scd_step(p, b, [], [], np.zeros(1), B)
    ratio = p[:, 0] / b[:, 0, 0]
    order = np.argsort(-ratio, kind="stable")
    cum = np.cumsum(b[order, 0, 0])
    crit = order[np.argmax(cum > B[0])]
    assert lam1[0] == pytest.approx(ratio[crit], rel=1e-14)
    # the critical user is tied at the threshold itself; just above it the
    # consumption fits (Eq. (9)) and just below it does not
    _, R_hi, _, _ = oracle.user_pass(p, b, [], [], lam1 * (1 + 1e-9))
    _, R_lo, _, _ = oracle.user_pass(p, b, [], [], lam1 * (1 - 1e-9))
    assert R_hi[0] <= B[0] < R_lo[0]


def test_scd_K1_fixed_point_after_one_step():
    """Sec. 4.4: for K=1 the Map does not depend on lambda^t, so one SCD step from any
    start reaches the same lambda, which is then a fixed point (cf. Table 1, M=1)."""
    rng = np.random.default_rng(8)
    N, M = 300, 4
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, 1))
    S, C = [0b0011, 0b1111], [1, 2]
    B = np.array([0.2 * b.sum()])
    l1a, _, _ = oracle.scd_step(p, b, S, C, np.zeros(1), B)
    l1b, _, _ = oracle.scd_step(p, b, S, C, np.array([0.77]), B)
    l2, _, _ = oracle.scd_step(p, b, S, C, l1a, B)
    assert l1a[0] == l1b[0] == l2[0]


# ---------------------------------------------------------------------------
# Eq. (14), duality, Everett's property, LP bound, Danskin gradient, Sec. 5.4
# ---------------------------------------------------------------------------

def test_dd_update_closed_form():
    lam = np.array([0.5, 0.1, 0.0])
    R = np.array([10.0, 2.0, 1.0])
    B = np.array([8.0, 4.0, 3.0])
    out = oracle.dd_update(lam, R, B, 0.1)
    assert out.tolist() == pytest.approx([0.7, 0.0, 0.0])


def _tiny_instance(seed, N=3, M=3, K=2):
    rng = np.random.default_rng(seed)
    S, C = random_laminar(M, rng, max_nodes=3)
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.3 * b.sum(axis=(0, 1))
    return p, b, S, C, B


def _all_feasible_primal(p, b, S, C, B, Bcap=None):
    """Exhaustive maximum of Eq. (1) subject to (2)-(4); Bcap overrides B per k
    (np.inf = unconstrained)."""
    N, M, K = b.shape
    Bc = B if Bcap is None else Bcap
    local = [m for m in range(1 << M) if feasible_local(m, S, C)]
    best = -1.0
    for combo in itertools.product(local, repeat=N):
        x = np.array([[(m >> j) & 1 for j in range(M)] for m in combo], dtype=float)
        R = np.einsum("ij,ijk->k", x, b)
        if np.all(R <= Bc + 1e-12):
            best = max(best, float((p * x).sum()))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_weak_duality(seed):
    """Eq. (5)-(10): g(lambda) >= every feasible primal value, for every lambda >= 0."""
    p, b, S, C, B = _tiny_instance(400 + seed)
    best = _all_feasible_primal(p, b, S, C, B)
    rng = np.random.default_rng(seed)
    for _ in range(30):
        lam = rng.uniform(0, 2, size=B.shape)
        assert oracle.dual_value(p, b, S, C, lam, B) >= best - 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_everett_property(seed):
    """Sec. 4.4 (Everett / Shapiro): x(lambda) is optimal for the KP whose budgets are
    replaced by its own consumption R_k(lambda) where lambda_k > 0 (and left free where
    lambda_k = 0)."""
    p, b, S, C, B = _tiny_instance(500 + seed)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        lam = rng.uniform(0, 1.5, size=B.shape) * (rng.random(B.shape) < 0.8)
        x, R, _, primal = oracle.user_pass(p, b, S, C, lam)
        cap = np.where(lam > 0, R, np.inf)
        assert primal == pytest.approx(_all_feasible_primal(p, b, S, C, B, cap), abs=1e-12)


def test_lagrangian_dual_equals_lp_relaxation():
    """The Lagrangian dual min_lambda g(lambda) of a KP whose local constraints form a
    laminar (matroid) family equals its LP relaxation (the local polytope is integral).
    g evaluated at the LP's optimal multipliers of the global rows must equal the LP
    optimum; any other lambda gives more (weak duality)."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(11)
    N, M, K = 30, 4, 2
    S, C = [0b0011, 0b1111], [1, 2]
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.15 * b.sum(axis=(0, 1))
    nv = N * M
    A_glob = b.reshape(nv, K).T
    rows = [A_glob]
    rhs = [B]
    for i in range(N):
        for s, c in zip(S, C):
            r = np.zeros(nv)
            for j in range(M):
                if (s >> j) & 1:
                    r[i * M + j] = 1
            rows.append(r[None, :])
            rhs.append(np.array([c]))
    res = linprog(-p.reshape(-1), A_ub=np.vstack(rows), b_ub=np.concatenate(rhs),
                  bounds=[(0, 1)] * nv, method="highs")
    assert res.status == 0
    lp = -res.fun
    lam_star = -res.ineqlin.marginals[:K]
    g = oracle.dual_value(p, b, S, C, lam_star, B)
    assert g == pytest.approx(lp, rel=1e-9)
    for _ in range(20):
        lam = np.maximum(lam_star + rng.normal(scale=0.05, size=K), 0)
        assert oracle.dual_value(p, b, S, C, lam, B) >= lp - 1e-9


def test_danskin_gradient_by_central_differences():
    """At a generic lambda the maximiser x* is unique and locally constant, so
    dg/dlambda_k = B_k - R_k, dg/dp_ij = x*_ij and dg/dB_k = lambda_k."""
    rng = np.random.default_rng(12)
    N, M, K = 50, 5, 3
    S, C = [0b00111, 0b11111], [1, 2]
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.2 * b.sum(axis=(0, 1))
    lam = rng.uniform(0.05, 0.4, size=K)
    x, R, _, _ = oracle.user_pass(p, b, S, C, lam)
    h = 1e-7
    for k in range(K):
        e = np.zeros(K)
        e[k] = h
        fd = (oracle.dual_value(p, b, S, C, lam + e, B) -
              oracle.dual_value(p, b, S, C, lam - e, B)) / (2 * h)
        assert fd == pytest.approx(B[k] - R[k], rel=1e-6, abs=1e-6)
        e2 = np.zeros(K)
        e2[k] = h
        fdB = (oracle.dual_value(p, b, S, C, lam, B + e2) -
               oracle.dual_value(p, b, S, C, lam, B - e2)) / (2 * h)
        assert fdB == pytest.approx(lam[k], rel=1e-6)
    for (i, j) in [(0, 0), (3, 2), (7, 4), (11, 1)]:
        pp = p.copy()
        pp[i, j] += h
        pm = p.copy()
        pm[i, j] -= h
        fd = (oracle.dual_value(pp, b, S, C, lam, B) - oracle.dual_value(pm, b, S, C, lam, B)) / (2 * h)
        assert fd == pytest.approx(float(x[i, j]), abs=1e-6)


def test_mckp_special_case():
    """Sec. 2.2: K=1, one set with C=1 is the multiple-choice KP; the per-user
    subproblem then picks the single item of largest positive p~."""
    rng = np.random.default_rng(13)
    N, M = 40, 6
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, 1))
    lam = np.array([0.7])
    x, _, _, _ = oracle.user_pass(p, b, [(1 << M) - 1], [1], lam)
    pt = p - 0.7 * b[:, :, 0]
    for i in range(N):
        j = int(np.argmax(pt[i]))
        want = np.zeros(M, dtype=int)
        if pt[i, j] > 0:
            want[j] = 1
        assert x[i].tolist() == want.tolist()


def test_postprocess_feasible_and_ordered():
    """Sec. 5.4: users are reset in non-decreasing order of the cost-adjusted group
    profit until every global constraint holds."""
    rng = np.random.default_rng(14)
    N, M, K = 200, 4, 3
    S, C = [0b1111], [2]
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.05 * b.sum(axis=(0, 1))
    lam = np.zeros(K)
    x, R, _, _ = oracle.user_pass(p, b, S, C, lam)
    assert np.any(R > B)
    x2, nreset = oracle.postprocess(p, b, lam, B, x)
    R2 = np.einsum("ij,ijk->k", x2, b)
    assert np.all(R2 <= B + 1e-12)
    gp = (p * x).sum(1) - np.einsum("ij,ijk,k->i", x, b, lam)
    order = np.lexsort((np.arange(N), gp))
    reset_users = order[:nreset]
    assert np.all(x2[reset_users] == 0)
    keep = order[nreset:]
    assert np.array_equal(x2[keep], x[keep])
    # minimal: un-resetting the last reset user breaks feasibility
    last = order[nreset - 1]
    R3 = R2 + np.einsum("j,jk->k", x[last], b[last])
    assert np.any(R3 > B)


def test_scd_emitted_mass_is_consumption_at_zero():
    """Summing a user's emitted v2 for k over all v1 > 0 gives the user's
    k-consumption just above lambda_k = 0 (others fixed)."""
    rng = np.random.default_rng(15)
    N, M, K = 40, 5, 3
    S, C = [0b00011, 0b11100, 0b11111], [1, 2, 2]
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.2 * b.sum(axis=(0, 1))
    lam = rng.uniform(0, 0.5, size=K)
    _, _, mass = oracle.scd_step(p, b, S, C, lam, B)
    for k in range(K):
        lam0 = lam.copy()
        lam0[k] = 1e-12
        _, R0, _, _ = oracle.user_pass(p, b, S, C, lam0)
        assert mass[k] == pytest.approx(R0[k], rel=1e-12)


def test_presolve_scaling_on_a_doubled_instance():
    """Sec. 5.3: sampling the first copy of an instance whose users all appear twice
    (budgets = those of the doubled instance) scales the budgets back to the
    original's, so pre-solving equals plain SCD on the original instance."""
    rng = np.random.default_rng(3)
    N, M, K = 40, 4, 2
    p = rng.uniform(0, 1, (N, M))
    b = rng.uniform(0, 1, (N, M, K))
    S, C = [0b1111], [2]
    B = 0.3 * b.sum(axis=(0, 1))
    p2, b2 = np.concatenate([p, p]), np.concatenate([b, b])
    B2 = 2 * B
    lam = np.zeros(K)
    for _ in range(3):
        lam, _, _ = oracle.scd_step(p, b, S, C, lam, B)
    got = oracle.presolve(p2, b2, S, C, B2, np.arange(N), 3)
    assert np.allclose(got, lam, rtol=0, atol=0)
    # the whole instance as the sample: plain SCD on it
    full = oracle.presolve(p, b, S, C, B, np.arange(N), 3)
    assert np.allclose(full, lam, rtol=0, atol=0)


# ---------------------------------------------------------------------------
# Algorithm 5 (Sec. 5.1): one item per knapsack, one cap Q
# ---------------------------------------------------------------------------

def _one_to_one(rng, K):
    p = rng.uniform(0, 1, size=K)
    bd = rng.uniform(0.05, 1, size=K)
    b = np.zeros((K, K))
    np.fill_diagonal(b, bd)
    return p, bd, b


@pytest.mark.parametrize("seed", range(30))
def test_alg5_map_equals_general_map(seed):
    """Algorithm 5 emits what Algorithms 3-4 emit when item k alone consumes
    knapsack k and one set caps the count at Q (including Q >= K, where the cap
    never binds, and multipliers that push items to zero profit)."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 13))
    Q = int(rng.integers(1, K + 2))
    p, bd, b = _one_to_one(rng, K)
    S, C = [(1 << K) - 1], [Q]
    for _ in range(10):
        lam = rng.uniform(0, 1.5, size=K) * (rng.random(K) < 0.7)
        k5, v15, v25 = oracle.alg5_map_user(p, bd, Q, lam)
        kg, v1g, v2g = oracle.scd_map_user(p, b, S, C, lam)
        og = np.lexsort((v1g, kg))
        o5 = np.lexsort((v15, k5))
        assert np.array_equal(k5[o5], kg[og])
        assert np.allclose(v15[o5], v1g[og], rtol=1e-12, atol=0)
        assert np.array_equal(v25[o5], v2g[og])


def test_alg5_without_binding_cap_is_the_zero_crossing():
    """Q >= K: every item with p_k > 0 is taken while its adjusted profit is
    positive, so its only breakpoint is p_k / b_kk (Eq. (11)-(13) without (3))."""
    rng = np.random.default_rng(5)
    K = 7
    p, bd, _ = _one_to_one(rng, K)
    for Q in (K, K + 3):
        k5, v1, v2 = oracle.alg5_map_user(p, bd, Q, rng.uniform(0, 1, size=K))
        assert np.array_equal(k5, np.arange(K))
        assert np.allclose(v1, p / bd, rtol=1e-15)
        assert np.array_equal(v2, bd)


def test_alg5_single_item_cap_threshold():
    """Q = 1: item k takes the user's single slot while p_k - lambda_k b_kk beats
    the best other adjusted profit a*, so its breakpoint is (p_k - a*) / b_kk."""
    p = np.array([0.9, 0.5, 0.2])
    bd = np.array([0.5, 0.25, 1.0])
    lam = np.array([1.0, 0.4, 0.0])
    # adjusted profits: 0.4, 0.4, 0.2 (item 0 ranks first on ties: lower index)
    k5, v1, v2 = oracle.alg5_map_user(p, bd, 1, lam)
    want = {0: (0.9 - 0.4) / 0.5, 1: (0.5 - 0.4) / 0.25}
    assert sorted(k5.tolist()) == [0, 1]
    for k, v in zip(k5, v1):
        assert v == pytest.approx(want[int(k)], rel=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_alg5_step_equals_general_step(seed):
    """One Algorithm 4 iteration with Algorithm 5 as Map reaches the same
    multipliers as with the general Map (same Reduce)."""
    rng = np.random.default_rng(100 + seed)
    N, K, Q = 300, int(rng.integers(2, 9)), int(rng.integers(1, 4))
    p = rng.uniform(0, 1, size=(N, K))
    bd = rng.uniform(0.05, 1, size=(N, K))
    b = np.zeros((N, K, K))
    for k in range(K):
        b[:, k, k] = bd[:, k]
    B = 0.2 * bd.sum(axis=0)
    lam = np.zeros(K)
    for _ in range(4):
        got = oracle.alg5_step(p, bd, Q, lam, B)
        want, _, _ = oracle.scd_step(p, b, [(1 << K) - 1], [Q], lam, B)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
        lam = got


def test_one_to_one_instance_layout():
    """The seeded generator of Sec. 5.1's special case stores item k's only entry
    in knapsack k, with one cap of Q over all items (layout check, CPU)."""
    from paper_2002_00352_gb300 import gen
    inst = gen.one_to_one(50, 6, 2, seed=3)
    p, b = inst.to_dense_numpy()
    bd = inst.val.view(50, 6).double().numpy()
    for k in range(6):
        assert np.array_equal(b[:, k, k], bd[:, k])
    off = b.copy()
    for k in range(6):
        off[:, k, k] = 0
    assert not off.any()
    assert inst.S == [(1 << 6) - 1] and inst.C == [2]
    want = oracle.alg5_step(p, bd, 2, np.zeros(6), inst.B.numpy())
    got, _, _ = oracle.scd_step(p, b, inst.S, inst.C, np.zeros(6), inst.B.numpy())
    assert np.allclose(got, want, rtol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_postprocess_shortest_prefix_by_enumeration(seed):
    """Sec. 5.4 on values from a coarse dyadic grid (all sums exact in FP64, many
    equal group profits): the oracle resets exactly the shortest prefix of the
    order (group profit, user index) after which every budget holds, found here
    by enumerating every prefix length."""
    rng = np.random.default_rng(200 + seed)
    N, M, K = 40, 3, 2
    p = rng.integers(0, 8, size=(N, M)) / 8.0
    b = rng.integers(0, 8, size=(N, M, K)) / 8.0
    lam = rng.integers(0, 4, size=K) / 4.0
    x = (rng.random((N, M)) < 0.6).astype(np.int32)
    R = np.einsum("nmk,nm->k", b, x)
    B = np.maximum(np.floor(R * rng.uniform(0.3, 0.9, size=K)), 1.0)
    q = np.einsum("nm,nm->n", p, x) - np.einsum("nmk,nm,k->n", b, x, lam)
    order = np.lexsort((np.arange(N), q))
    want = None
    for r in range(N + 1):
        keep = np.ones(N, dtype=bool)
        keep[order[:r]] = False
        if np.all(np.einsum("nmk,nm->k", b[keep], x[keep]) <= B):
            want = r
            break
    x2, nreset = oracle.postprocess(p, b, lam, B, x)
    assert nreset == want
    reset = np.zeros(N, dtype=bool)
    reset[order[:want]] = True
    assert np.array_equal(x2[reset], np.zeros_like(x2[reset]))
    assert np.array_equal(x2[~reset], x[~reset])


@pytest.mark.parametrize("seed", range(8))
def test_coordinate_step_minimises_the_dual_along_k(seed):
    """Cyclic CD (Sec. 4.3.2) updates one multiplier by the Reduce of Algorithm 4 at
    lambda^t.  The dual g (Eq. (5)) is convex and piecewise linear in lambda_k with
    slope B_k - R_k, so that update must be the smallest minimiser of g along
    coordinate k: checked against g itself on a grid and at every candidate, and
    by the strict decrease just below it."""
    rng = np.random.default_rng(700 + seed)
    N, M, K = 6, int(rng.integers(2, 6)), int(rng.integers(1, 4))
    S, C = random_laminar(M, rng)
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K)) * (rng.random((N, M, K)) < 0.8)
    lam = rng.uniform(0, 0.6, size=K)
    B = rng.uniform(0.2, 1.5, size=K) * b.sum(axis=(0, 1)) / 3 + 1e-3
    for k in range(K):
        block = np.zeros(K, dtype=bool)
        block[k] = True
        nxt = oracle.bcd_step(p, b, S, C, lam, B, block)
        assert np.array_equal(nxt[~block], lam[~block])
        v = nxt[k]

        def g(x):
            l2 = lam.copy()
            l2[k] = x
            return oracle.dual_value(p, b, S, C, l2, B)

        gv = g(v)
        _, _, v1, _ = oracle.scd_map_users(p, b, S, C, lam)
        grid = np.concatenate([np.linspace(0, 4, 81), v1, v1 * (1 + 1e-7), v1 * (1 - 1e-7)])
        for x in grid[grid >= 0]:
            assert gv <= g(x) + 1e-9 * (1 + abs(gv)), (k, v, x)
        if v > 0:
            assert g(v * (1 - 1e-6)) > gv


def test_block_step_extremes():
    """A block of every knapsack is the SCD step; an empty block changes nothing."""
    rng = np.random.default_rng(5)
    N, M, K = 20, 5, 3
    S, C = random_laminar(M, rng)
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    lam = rng.uniform(0, 0.6, size=K)
    B = 0.2 * b.sum(axis=(0, 1))
    full, _, _ = oracle.scd_step(p, b, S, C, lam, B)
    assert np.array_equal(oracle.bcd_step(p, b, S, C, lam, B, np.ones(K, dtype=bool)), full)
    assert np.array_equal(oracle.bcd_step(p, b, S, C, lam, B, np.zeros(K, dtype=bool)), lam)


@pytest.mark.parametrize("seed", range(6))
def test_categorical_expansion_is_the_integer_optimum(seed):
    """Categorical x (Sec. 2): x_j in {0..u_j} is solved as u_j binary copies of item j.
    Algorithm 1 on the expanded user gives the optimum of the integer program
    max sum_j p~_j x_j s.t. the local count constraints, found here by exhaustive
    search over the integer vectors."""
    import itertools

    import torch
    from paper_2002_00352_gb300.categorical import expand_categorical, fold_decisions
    from paper_2002_00352_gb300.gen import random_small
    rng = np.random.default_rng(1300 + seed)
    M = int(rng.integers(2, 5))
    u = [int(v) for v in rng.integers(1, 4, size=M)]
    S, C = random_laminar(M, rng)
    inst = random_small(3, M, 2, seed=seed, device="cpu", layout="dense" if seed % 2 else "csr")
    inst.S, inst.C = S, C
    big = expand_categorical(inst, u)
    lam = rng.uniform(0, 0.5, size=2)
    p, b = inst.to_dense_numpy()
    p2, b2 = big.to_dense_numpy()
    for i in range(3):
        pt = p[i] - b[i] @ lam
        best = max(float(pt @ np.array(x)) for x in itertools.product(*[range(v + 1) for v in u])
                   if all(sum(x[j] for j in range(M) if (s >> j) & 1) <= c for s, c in zip(S, C)))
        x2 = oracle.greedy(p2[i] - b2[i] @ lam, big.S, big.C)
        xi = fold_decisions(torch.tensor(x2)[None], u)[0].numpy()
        assert all(0 <= xi[j] <= u[j] for j in range(M))
        assert float(pt @ xi) == pytest.approx(best, abs=1e-12)


def test_bucket_ids_at_the_boundaries():
    """Sec. 5.2 buckets (id 0 for |d| < Delta, else sign(d) (1 + floor(log2(|d| / Delta)))),
    with lambda_k^t = 1 and Delta = 0.25, both exact in FP32: a boundary value belongs
    to the bucket above it in |d|, ids are clamped at 127."""
    v = np.array([1.0, 1.2499, 1.25, 1.4999, 1.5, 2.0, 2.0001, 0.7501, 0.75, 0.5, 0.4999,
                  1.0 + 2.0 ** 100, 2.0 ** 125, 2.0 ** 126])
    # 2^100 / 0.25 = 2^102: 1 + 102; 2^125 / 0.25 = 2^127: 128, clamped; 2^126 / 0.25
    # overflows FP32 to inf: clamped
    want = [0, 0, 1, 1, 2, 3, 3, 0, -1, -2, -2, 103, 127, 127]
    assert oracle.bucket_ids(v, 1.0, 0.25).tolist() == want


def test_bucket_reduce_worked_example():
    """Hand-worked example of the bucketed Reduce: lambda^t = 1, Delta = 0.1 (FP32:
    0.100000001490116), candidates 1.05 (mass 1, bucket 0 = [0.9, 1.1)), 1.15 (mass
    2, bucket 1 = [1.1, 1.2)), 1.35 (mass 4, bucket 2 = [1.2, 1.4)), 0.7 (mass 8,
    bucket -2 = [0.6, 0.8)).
      B = 4.5: bucket 2 leaves 4 <= 4.5, bucket 1 takes it to 6: 1.2 - (0.5 / 2) 0.1
      B = 5:   1.2 - (1 / 2) 0.1 = 1.15
      B = 0.5: bucket 2 crosses: 1.4 - (0.5 / 4) 0.2 = 1.375
      B = 14:  7 above bucket -2, which crosses: 0.8 - (7 / 8) 0.2 = 0.625
      B = 15:  the whole mass fits: 0."""
    v1 = np.array([1.05, 1.15, 1.35, 0.7])
    v2 = np.array([1.0, 2.0, 4.0, 8.0])
    d = float(np.float32(0.1))
    for Bk, want in [(4.5, 1.0 + 2 * d - 0.25 * d), (5.0, 1.0 + 2 * d - 0.5 * d), (0.5, 1.0 + 4 * d - 0.125 * 2 * d),
                     (14.0, 1.0 - 2 * d - 0.875 * 2 * d), (15.0, 0.0)]:
        got = oracle.bucket_reduce(v1, v2, Bk, 1.0, oracle.bucket_delta(1.0, 0.1))
        assert got == pytest.approx(want, abs=1e-12), (Bk, got, want)
    # the worked numbers themselves
    assert oracle.bucket_reduce(v1, v2, 4.5, 1.0, oracle.bucket_delta(1.0, 0.1)) == pytest.approx(1.175, abs=1e-8)
    assert oracle.bucket_reduce(v1, v2, 14.0, 1.0, oracle.bucket_delta(1.0, 0.1)) == pytest.approx(0.625, abs=1e-8)


def test_bucket_reduce_one_bucket_closed_form():
    """With every candidate inside bucket 0 the mass is spread uniformly over
    [lambda^t - Delta, lambda^t + Delta): the threshold is lambda^t + Delta - 2 Delta B / M
    (M the total mass), or 0 when B >= M."""
    rng = np.random.default_rng(11)
    lt, dl = 2.0, np.float32(0.5)
    v1 = rng.uniform(1.6, 2.4, size=50)
    v2 = rng.uniform(0.1, 1.0, size=50)
    Mt = v2.sum()
    for frac in (0.1, 0.5, 0.9):
        got = oracle.bucket_reduce(v1, v2, frac * Mt, lt, dl)
        assert got == pytest.approx(lt + float(dl) - 2 * float(dl) * frac, rel=1e-12)
    assert oracle.bucket_reduce(v1, v2, Mt * 1.0001, lt, dl) == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_bucketed_reduce_brackets_the_exact_reduce(seed):
    """The exact threshold of Algorithm 4 (pinned above by its definition) lies in
    the bucket the bucketed Reduce interpolates in, so the two differ by at most that
    bucket's width; the buckets are monotone in v, so the crossing bucket is the
    exact threshold's."""
    rng = np.random.default_rng(1400 + seed)
    N, M, K = 60, 6, 3
    S, C = random_laminar(M, rng)
    p = rng.uniform(0, 1, size=(N, M))
    b = rng.uniform(0, 1, size=(N, M, K))
    B = 0.15 * b.sum(axis=(0, 1))
    lam = rng.uniform(0.2, 0.8, size=K)
    exact, _, _ = oracle.scd_step(p, b, S, C, lam, B)
    _, ek, v1, v2 = oracle.scd_map_users(p, b, S, C, lam)
    for delta in (1e-4, 1e-2, 0.5):
        for k in range(K):
            sel = ek == k
            dk = oracle.bucket_delta(lam[k], delta)
            got = oracle.bucket_reduce(v1[sel], v2[sel], B[k], lam[k], dk)
            if exact[k] == 0.0:
                assert got == 0.0 or v2[sel][v1[sel] > 0].sum() > B[k]
                continue
            idb = int(oracle.bucket_ids(np.array([exact[k]]), lam[k], dk)[0])
            lo, hi = oracle.bucket_range(idb, lam[k], dk)
            assert abs(got - exact[k]) <= (hi - lo) * (1 + 1e-9), (seed, delta, k, got, exact[k], lo, hi)


def test_bucket_reduce_degenerate_cases():
    """No candidate, or all mass within the budget: 0 (Algorithm 4).  At
    lambda^t = 0 the width is delta itself and every candidate lies above: with
    delta = 0.25, candidates 0.1 (|d| / Delta = 0.4: bucket 0 = [-0.25, 0.25)),
    0.3 (1.2: bucket 1 = [0.25, 0.5)) and 0.9 (3.6: bucket 2 = [0.5, 1)) of mass 1
    each; B = 1.5: bucket 2 holds 1 <= 1.5, bucket 1 crosses:
    0.5 - 0.5 * 0.25 = 0.375; B = 2.5: bucket 0 crosses at
    0.25 - 0.5 * 0.5 = 0, inside its range and not below 0."""
    assert oracle.bucket_reduce(np.array([]), np.array([]), 1.0, 0.7, 0.1) == 0.0
    assert oracle.bucket_reduce(np.array([0.5, 0.9]), np.array([1.0, 1.0]), 2.0, 0.7, 0.1) == 0.0
    v1 = np.array([0.1, 0.3, 0.9])
    v2 = np.ones(3)
    dl = oracle.bucket_delta(0.0, 0.25)
    assert float(dl) == 0.25
    assert oracle.bucket_ids(v1, 0.0, dl).tolist() == [0, 1, 2]
    assert oracle.bucket_reduce(v1, v2, 1.5, 0.0, dl) == pytest.approx(0.375, abs=1e-12)
    assert oracle.bucket_reduce(v1, v2, 2.5, 0.0, dl) == 0.0
