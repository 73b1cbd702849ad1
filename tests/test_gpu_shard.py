"""User-sharded instances: the users of one instance split over two handles (as
over two GPUs), solved through a shard group, against one handle over all the
users.  Users are independent given lambda (Sec. 4.1), and the shards' partials
are exact integers, so every SCD step (Algorithm 4) must give the same
lambda^{t+1}, R, dual and primal sums bit for bit."""
import pytest
import torch

from paper_2002_00352_gb300 import gen, kp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,cut", [
    (lambda: gen.sparse_csr(N=20_000, device="cuda"), 0.5),
    (lambda: gen.sparse_csr(N=20_000, device="cuda"), 0.13),
    (lambda: gen.small_dd_scd(device="cuda"), 0.5),
    (lambda: gen.hier_m20(N=8000, device="cuda"), 0.37),
])
def test_two_shards_equal_one_handle(make, cut):
    inst = make()
    N, K = inst.N, inst.K
    one = kp.kp_create_from_instance(inst)
    m = int(N * cut)
    group = kp.kp_shard_group_create([kp.kp_create_user_range(inst, 0, m), kp.kp_create_user_range(inst, m, N)])
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    lam1, lam2 = z(K), z(K)
    for t in range(8):
        n1, R1, d1, p1 = z(K), z(K), z(()), z(())
        n2, R2, d2, p2 = z(K), z(K), z(()), z(())
        kp.kp_scd_step(one, lam1, n1, R=R1, dual_sum=d1, primal_sum=p1)
        kp.kp_shard_group_scd_step(group, lam2, n2, R=R2, dual_sum=d2, primal_sum=p2)
        kp.kp_device_status(one)
        kp.kp_device_status(group.shards[0])
        assert torch.equal(n1, n2), (t, (n1 - n2).abs().max())
        assert torch.equal(R1, R2), t
        assert torch.equal(d1, d2) and torch.equal(p1, p2), t
        lam1, lam2 = n1, n2
    group.close()
