"""Multi-process replicas of bench.py on the CPU (gloo, world size 2): every rank
solves its own instance and the job's time is the slowest rank's.  The GPU path
has no cross-rank data exchange, so the host logic is what the processes share."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    values = [3.25, 7.5]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, values, out), nprocs=2, join=True)
        assert out[0] == out[1] == pytest.approx(7.5)


def test_max_over_ranks_single():
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0


# ---------------------------------------------------------------------------
# user-sharded Reduce on the CPU: each rank holds half of an instance's users
# ---------------------------------------------------------------------------

def _partials(p, b, S, C, lam, wlo, whi, s):
    """Integer partials of one rank's users: fixed-point consumption at lam (units
    2^-s), the masses of the breakpoints (Algorithm 4 Map) above / inside / below
    the window [wlo, whi) per knapsack, and the breakpoints inside it."""
    import numpy as np
    import oracle
    K = b.shape[2]
    x, _, _, _ = oracle.user_pass(p, b, S, C, lam)
    R = np.rint(np.einsum("ij,ijk->ijk", x, b) * 2.0 ** s).astype(np.int64).sum(axis=(0, 1))
    _, ek, v1, v2 = oracle.scd_map_users(p, b, S, C, lam)
    m = np.rint(v2 * 2.0 ** s).astype(np.int64)
    reg = np.zeros((K, 3), dtype=np.int64)
    r = np.where(v1 >= whi[ek], 0, np.where(v1 >= wlo[ek], 1, 2))
    np.add.at(reg, (ek, r), m)
    inside = r == 1
    return R, reg, ek[inside], v1[inside], m[inside]


def _reduce(reg, ks, v1s, ms, Bfix):
    """The Reduce of Algorithm 4 from the combined partials: the breakpoint at which
    the mass from the top first exceeds B_k when it lies in the window (else -1:
    the crossing is outside it)."""
    import numpy as np
    out = np.full(len(Bfix), -1.0)
    for k in range(len(Bfix)):
        A, W = reg[k, 0], reg[k, 1]
        if A > Bfix[k] or A + W <= Bfix[k]:
            continue
        sel = ks == k
        order = np.lexsort((-ms[sel], -v1s[sel]))
        acc = A
        for v, mm in zip(v1s[sel][order], ms[sel][order]):
            acc += mm
            if acc > Bfix[k]:
                out[k] = v
                break
    return out


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2002_00352_gb300 import gen
    inst = gen.sparse_csr(N=3000, K=40, device="cpu")
    p, b = inst.to_dense_numpy()
    import oracle
    lam = np.full(inst.K, 0.5)
    nxt, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, inst.B.numpy())
    wlo, whi = 0.97 * nxt, 1.03 * nxt + 1e-9   # windows around the thresholds
    s = 40
    half = np.array_split(np.arange(inst.N), world)[rank]
    R, reg, ks, v1s, ms = _partials(p[half], b[half], inst.S, inst.C, lam, wlo, whi, s)
    # exact integer all-reduce of the partial sums
    Rt, regt = torch.from_numpy(R), torch.from_numpy(reg)
    dist.all_reduce(Rt)
    dist.all_reduce(regt)
    # union of the breakpoints inside the window
    n = torch.tensor([len(ks)])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    mx = int(max(int(z) for z in sizes))
    pack = torch.zeros(mx, 3, dtype=torch.float64)
    pack[:len(ks), 0] = torch.from_numpy(ks.astype(np.float64))
    pack[:len(ks), 1] = torch.from_numpy(v1s)
    pack[:len(ks), 2] = torch.from_numpy(ms.astype(np.float64))
    got = [torch.zeros(mx, 3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, pack)
    rows = torch.cat([g[:int(z)] for g, z in zip(got, sizes)]).numpy()
    Bfix = np.floor(inst.B.numpy() * 2.0 ** s).astype(np.int64)
    lam_next = _reduce(regt.numpy(), rows[:, 0].astype(np.int64), rows[:, 1], rows[:, 2].astype(np.int64), Bfix)
    # one process over all the users
    R1, reg1, ks1, v11, ms1 = _partials(p, b, inst.S, inst.C, lam, wlo, whi, s)
    want = _reduce(reg1, ks1, v11, ms1, Bfix)
    inw = want >= 0
    out[rank] = (bool(np.array_equal(Rt.numpy(), R1)), bool(np.array_equal(regt.numpy(), reg1)),
                 bool(np.array_equal(lam_next, want)), int(inw.sum()),
                 bool(np.array_equal(want[inw], nxt[inw])))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_reduce_gloo_world2():
    """Two CPU processes each hold half the users: their fixed-point consumption and
    window masses all-reduced over gloo, and the union of their in-window
    breakpoints, give exactly the single process's sums and thresholds."""
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(2, port, out), nprocs=2, join=True)
        for r in (0, 1):
            sameR, samereg, samelam, nin, oracle_agrees = out[r]
            assert sameR and samereg and samelam
            assert nin > 0 and oracle_agrees   # thresholds resolved inside the window: Algorithm 4's
