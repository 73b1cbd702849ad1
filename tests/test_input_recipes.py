"""The seeded synthetic workloads follow their stated recipes (shapes, value
ranges, sparsity, budgets, local constraints): checked on the CPU at small N."""
import numpy as np
import pytest

from paper_2002_00352_gb300 import gen


def _sets(inst):
    return list(zip(inst.S, inst.C))


def test_small_dd_scd_recipe():
    x = gen.small_dd_scd(N=2000, device="cpu")
    p, b = x.to_dense_numpy()
    assert (x.N, x.M, x.K, x.layout) == (2000, 10, 5, "dense")
    assert p.min() >= 0 and p.max() <= 1 and b.min() >= 0 and b.max() <= 1
    assert np.allclose(x.B.numpy(), 0.2 * b.sum(axis=(0, 1)), rtol=1e-6)
    assert _sets(x) == [((1 << 10) - 1, 3)]


def test_hier_m20_recipe():
    x = gen.hier_m20(N=3000, device="cpu")
    p, b = x.to_dense_numpy()
    assert (x.M, x.K) == (20, 20)
    assert p.min() > 0 and 0.3 < (b == 0).mean() < 0.7  # Bernoulli(0.5) mask
    assert np.allclose(x.B.numpy(), 0.1 * b.sum(axis=(0, 1)), rtol=1e-6)
    groups = [(((1 << 5) - 1) << (5 * g), 2) for g in range(4)]
    assert sorted(_sets(x)) == sorted(groups + [((1 << 20) - 1, 5)])


def test_dense_2e7_recipe():
    x = gen.dense_2e7(N=3000, device="cpu")
    p, b = x.to_dense_numpy()
    assert (x.M, x.K) == (10, 10)
    assert p.max() <= 1 and b.max() <= 1 and p.min() >= 0 and b.min() >= 0
    assert np.allclose(x.B.numpy(), 0.05 * b.sum(axis=(0, 1)), rtol=1e-6)
    assert sorted(_sets(x)) == sorted([(0b11111, 2), (0b1111100000, 2), ((1 << 10) - 1, 3)])


def test_sparse_csr_recipe():
    x = gen.sparse_csr(N=4000, device="cpu")
    assert (x.M, x.K, x.layout) == (10, 200, "csr")
    nnz = x.item_nnz.numpy()
    assert np.all(nnz == 2)
    k = x.kidx.numpy().astype(np.int64).reshape(-1, 2)
    assert np.all(k[:, 0] < k[:, 1])  # two distinct knapsacks per item, ascending
    assert k.min() >= 0 and k.max() < 200
    v = x.val.numpy()
    assert v.min() >= 0 and v.max() <= 1
    assert np.array_equal(x.user_off.numpy(), np.arange(x.N + 1) * 20)
    B = np.zeros(200)
    np.add.at(B, k.reshape(-1), v.astype(np.float64))
    assert np.allclose(x.B.numpy(), 0.05 * B, rtol=1e-9)
    assert sorted(_sets(x)) == sorted([(0b11111, 2), (0b1111100000, 2), ((1 << 10) - 1, 3)])


@pytest.mark.parametrize("seed", [4, 5])
def test_batched_specs_ranges(seed):
    specs = gen.batched_specs(count=64, seed=seed)
    N = np.array([s["N"] for s in specs])
    M = np.array([s["M"] for s in specs])
    K = np.array([s["K"] for s in specs])
    cap = np.array([s["cap"] for s in specs])
    assert N.min() >= 1_000 and N.max() <= 1_000_000
    assert M.min() >= 5 and M.max() <= 50 and K.min() >= 1 and K.max() <= 64
    assert np.all(cap >= 1) and np.all(cap <= M // 2)
    x = gen.batched_instance(dict(specs[0], N=500), device="cpu")
    p, b = x.to_dense_numpy()
    assert np.allclose(x.B.numpy(), 0.1 * b.sum(axis=(0, 1)), rtol=1e-6)
    assert _sets(x) == [((1 << x.M) - 1, specs[0]["cap"])]
