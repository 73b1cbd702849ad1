"""The allocation-free consumption entry point, against the handle-based one.

Callers whose device memory belongs to their own pool, or that must not take
the driver's allocation locks on a latency-critical path, cannot call
cudaMalloc; kp_reduce_consumption_noalloc serves them from a fixed
__device__ scratch array.  This file is collected last so that a run stopping
at the first failure has run every other test already; it also passes when
run alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2002_00352_gb300 import gen, kp

pytestmark = pytest.mark.gpu

REL = 1e-6


def _outputs(K, N, W):
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    return z(K), z(()), z(()), z(()), torch.zeros(N * W, dtype=torch.int32, device="cuda")


def _kw(inst):
    if inst.layout == "dense":
        return dict(b_dense=inst.b)
    return dict(csr_user_off=inst.user_off, csr_item_nnz=inst.item_nnz, csr_val=inst.val,
                csr_k=inst.kidx)


@pytest.mark.parametrize("make", [
    lambda: gen.small_dd_scd(N=5000, device="cuda"),
    lambda: gen.sparse_csr(N=20000, device="cuda"),
    lambda: gen.random_small(3001, 7, 4, seed=3, device="cuda", layout="csr", L_groups=[((0, 3), 1)], total_cap=2),
])
def test_noalloc_matches_handle_path_twice(make):
    inst = make()
    prob = kp.kp_create_from_instance(inst)
    rng = np.random.default_rng(0)
    lam = torch.tensor(rng.uniform(0, 0.5, inst.K), dtype=torch.float64, device="cuda")
    R0, d0, p0, g0, x0 = _outputs(inst.K, inst.N, prob.W)
    kp.kp_reduce_consumption(prob, lam, R=R0, dual_sum=d0, primal_sum=p0, g=g0, x_bits=x0)
    torch.cuda.synchronize()
    for call in range(2):
        R1, d1, p1, g1, x1 = _outputs(inst.K, inst.N, prob.W)
        kp.kp_reduce_consumption_noalloc(inst.N, inst.M, inst.K, inst.p, inst.B, inst.S, inst.C, lam,
                                         R=R1, dual_sum=d1, primal_sum=p1, g=g1, x_bits=x1, **_kw(inst))
        torch.cuda.synchronize()
        assert torch.equal(x1, x0), call
        assert torch.all(torch.abs(R1 - R0) <= REL * torch.abs(R0) + 1e-12), call
        for a, b in ((d1, d0), (p1, p0), (g1, g0)):
            assert abs(float(a) - float(b)) <= REL * abs(float(b)) + 1e-12, call
    prob.close()


def test_noalloc_rejects_too_many_knapsacks():
    p = torch.rand(4, device="cuda")
    b = torch.rand(4 * 4, device="cuda")
    B = torch.ones(kp_max_k() + 1, dtype=torch.float64, device="cuda")
    lam = torch.zeros(kp_max_k() + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(kp.KpError) as e:
        kp.kp_reduce_consumption_noalloc(1, 4, kp_max_k() + 1, p, B, [], [], lam, b_dense=b)
    assert e.value.status == kp.KP_EINVAL
    assert "KP_MAX_K" in str(e.value)


def kp_max_k():
    return kp.kp_limits()["max_k"]
