#!/usr/bin/env python
"""Benchmark of one synchronous-coordinate-descent iteration (Algorithm 4) plus the
dual-gradient kernel, on the sparse billion-variable workload:

  N = 1e8 users, M = 10 items (1e9 decision variables), K = 200 knapsacks, b in
  CSR with 2 nonzeros per item (int16 knapsack index), p ~ lognormal(0,1),
  constraints {1..5}:2, {6..10}:2 and a total cap of 3 per user (3e8 local
  constraints), B_k = 0.05 * sum b.

A step = kp_scd_breakpoints (user pass: reduced costs, greedy, consumption,
breakpoint histograms) + kp_threshold_select (Reduce of Algorithm 4, with any
re-run passes it needs) + kp_dual_backward (gradient of the dual, x* and
B - R), all through the C ABI, continuing one SCD trajectory from lambda = 0.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SCD users*iters/s at N=1e8, M=10 (K=200, CSR 2 nnz/item)"
UNIT = "users*iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="csr_N1e8_M10_K200")
    ap.add_argument("--N", type=int, default=None, help="override the number of users")
    ap.add_argument("--cpu-sample", type=int, default=20000)
    ap.add_argument("--ref-sample", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the post-processing measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched measurement")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-warmup", type=int, default=1)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-nhi", type=int, default=1_000_000)
    return ap.parse_args()


def workload(name, N, device):
    from paper_2002_00352_gb300 import gen
    if name.startswith("csr"):
        inst = gen.sparse_csr(N=N or 100_000_000, device=device)
    elif name == "dense_N2e7_M10_K10":
        inst = gen.dense_2e7(N=N or 20_000_000, device=device)
    elif name == "dense_N1e6_M20_K20":
        inst = gen.hier_m20(N=N or 1_000_000, device=device)
    elif name == "dense_N1e4_M10_K5":
        inst = gen.small_dd_scd(N=N or 10_000, device=device)
    else:
        raise SystemExit(f"unknown workload {name}")
    return inst


def algo_bytes_per_user(inst):
    """Bytes the user pass must read per user: p (4M), b (CSR: 6 per entry + 1 per
    item count; dense: 4MK)."""
    if inst.layout == "csr":
        nnz_per_user = inst.val.numel() / inst.N
        return 4 * inst.M + 6 * nnz_per_user + inst.M
    return 4 * inst.M + 4 * inst.M * inst.K


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over the ranks of the job (replicas: the job's time is
    its slowest rank's); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def kernel_source_hash():
    """Hash of the breakpoint pass's sources with comments and blank lines removed
    (a capture stays valid across comment edits, not across code changes)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ["kp_pass.cu", "kp_device.cuh", "kp_internal.h"]:
        with open(os.path.join(ROOT, "paper_2002_00352_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def measured_traffic(N, layout):
    """DRAM bytes (read + write) per launch of the breakpoint pass: the per-user
    figure of the committed ncu capture (profiles/csr_pass_kernel_hist_N2e6.md,
    taken at N = 2e6 and scaled by the users of one launch), or None when the
    kernel sources changed since that capture."""
    if layout != "csr":
        return None
    try:
        with open(os.path.join(ROOT, "profiles", "csr_pass_kernel_hist_N2e6.md")) as f:
            text = f.read()
        per_user = float(text.split("traffic_bytes_per_user:")[1].split()[0])
        src = text.split("source_hash:")[1].split()[0]
    except Exception:
        return None
    return per_user * N if src == kernel_source_hash() else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def quality(inst, prob, x_after, R_before, R_after, g, primal_before):
    """Solution quality at the last lambda (Sec. 6.1-6.2): duality gap (dual value minus
    primal objective), the number of knapsacks over budget and the max constraint
    violation ratio (excess over budget / budget), for x = Algorithm 1 at lambda and
    after Sec. 5.4's post-processing (x_after)."""
    import torch
    from paper_2002_00352_gb300 import kp
    B = inst.B
    N, M = inst.N, inst.M
    pv = inst.p.view(N, M)
    W = (M + 31) // 32
    xw = x_after.view(N, W)
    primal_after = 0.0
    step = 1 << 24
    for s in range(0, N, step):
        n = min(step, N - s)
        xs = kp.unpack_x(xw[s:s + n].reshape(-1), n, M).double()
        primal_after += float((xs * pv[s:s + n].double()).sum())

    def viol(R):
        r = torch.clamp((R - B) / B, min=0.0)
        return int((R > B).sum()), float(r.max())

    nb, mb = viol(R_before)
    na, ma = viol(R_after)
    return {"dual_value": g, "primal_before": primal_before, "duality_gap_before": g - primal_before,
            "violated_before": nb, "max_violation_ratio_before": mb,
            "primal_after": primal_after, "duality_gap_after": g - primal_after,
            "violated_after": na, "max_violation_ratio_after": ma,
            "note": "at the lambda after the timed steps; primal after post-processing summed here "
                    "(torch, float64) from the returned x"}


def cpu_baseline(inst, n, min_seconds=10.0):
    """The oracle as it stands on the first n users of the same instance (budgets
    scaled by n/N): SCD iterations, each a state pass (Algorithms 1-2) plus a
    step of Algorithms 3-4, repeated for about min_seconds."""
    import numpy as np
    import oracle
    p, b = inst.users_dense(np.arange(n))
    B = inst.B.cpu().numpy() * (n / inst.N)
    lam = np.zeros(inst.K)
    iters = 0
    t0 = time.perf_counter()
    while True:
        oracle.user_pass(p, b, inst.S, inst.C, lam, want_x=True)
        lam, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
        iters += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds and iters >= 3:
            break
    return {"value": n * iters / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {n} users of the workload (budgets scaled by n/N), {iters} SCD "
                      f"iterations from lambda = 0 with the state pass, {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np
    import torch
    import oracle
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    inst = workload(args.workload, min(args.N or 10**9, max(args.ref_sample, 1000)), dev)
    n = min(args.ref_sample, inst.N)
    p, b = inst.users_dense(np.arange(n))
    B = inst.B.cpu().numpy()
    lam = np.zeros(inst.K)
    for _ in range(args.warmup):
        oracle.user_pass(p, b, inst.S, inst.C, lam, want_x=False)
        lam, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.user_pass(p, b, inst.S, inst.C, lam, want_x=True)
        lam, _, _ = oracle.scd_step(p, b, inst.S, inst.C, lam, B)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"{args.workload} sample of {n} users (CPU oracle)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": f"{n} users of the workload per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batched_measure(count, n_hi, steps, warmup, graph=True):
    """`count` independent dense instances (N log-uniform in [1e3, n_hi], M in 5..50,
    K in 1..64, total cap C in 1..M/2): SCD steps of the whole batch by the batched
    path (one persistent launch per pass), and the same steps by looping the
    per-instance path over the instances, from lambda = 0 (warm-up steps first);
    instances*iters/s of both and whether their lambdas agree bit for bit."""
    import torch
    from paper_2002_00352_gb300 import gen, kp
    specs = gen.batched_specs(count=count, n_hi=n_hi)
    insts = [gen.batched_instance(sp, device="cuda") for sp in specs]
    batch = kp.kp_batch_create(insts)
    probs = [kp.kp_create_from_instance(x) for x in insts]
    totK = batch.totK
    koff = batch.koff

    def batched_steps(n, lam):
        nxt = torch.empty_like(lam)
        for _ in range(n):
            kp.kp_batch_scd_step(batch, lam, nxt)
            lam, nxt = nxt, lam
        return lam

    def looped_steps(n, lam):
        nxt = torch.empty_like(lam)
        for _ in range(n):
            for i, pr in enumerate(probs):
                kp.kp_scd_step(pr, lam[koff[i]:koff[i + 1]], nxt[koff[i]:koff[i + 1]])
            lam, nxt = nxt, lam
        return lam

    def graph_steps(n, lam):
        from paper_2002_00352_gb300.solver import BatchScdGraph
        g = graph_cache.get("g")
        if g is None:  # a batch of its own: its selection state starts fresh like the others'
            graph_cache["batch"] = kp.kp_batch_create(insts)
            g = graph_cache["g"] = BatchScdGraph(graph_cache["batch"], lam)
        else:
            g.a.copy_(lam)
        for _ in range(n // 2):
            g.replay()
        return g.a

    graph_cache = {}
    res = {}
    modes = [("batched", batched_steps), ("looped", looped_steps)]
    if graph and steps % 2 == 0 and warmup % 2 == 0:
        modes.append(("graph", graph_steps))
    for name, fn in modes:
        lam = torch.zeros(totK, dtype=torch.float64, device="cuda")
        lam = fn(warmup, lam)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lam = fn(steps, lam)
        e1.record()
        torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1), lam.cpu())
    kp.kp_batch_device_status(batch)
    same = bool(torch.equal(res["batched"][1], res["looped"][1]))
    ms_b, ms_l = res["batched"][0], res["looped"][0]
    n = len(insts)
    out = {"metric": f"batched SCD instances*iters/s ({n} instances)", "value": n * steps / (ms_b / 1e3),
           "unit": "instances*iters/s", "steps": steps, "warmup": warmup, "ms_per_step": ms_b / steps,
           "workload": f"{n} dense instances, N log-uniform [1e3, {n_hi:.0e}], M 5..50, K 1..64, "
                       f"total cap 1..M/2, SCD from lambda = 0 ({warmup} warm-up steps)",
           "users": sum(x.N for x in insts), "total_knapsacks": totK,
           "instance_bytes": sum(x.nbytes() for x in insts),
           "looped_value": n * steps / (ms_l / 1e3), "looped_ms_per_step": ms_l / steps,
           "speedup_vs_looped": ms_l / ms_b, "same_lambda_as_looped": same}
    if "graph" in res:
        ms_g = res["graph"][0]
        out["graph_ms_per_step"] = ms_g / steps
        out["graph_value"] = n * steps / (ms_g / 1e3)
        out["same_lambda_graph"] = bool(torch.equal(res["graph"][1], res["batched"][1]))
    del batch, probs, insts, graph_cache
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    b = batched_measure(args.batch_count, args.batch_nhi, args.steps, args.warmup)
    out = {"metric": b["metric"], "value": b["value"], "unit": b["unit"], "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {k: v for k, v in b.items() if k not in ("metric", "value", "unit", "steps", "warmup",
                                                              "ms_per_step")}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.workload == "batched_256":
        run_batched(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_2002_00352_gb300 import kp

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = "cuda"
    inst = workload(args.workload, args.N, dev)
    # replicas: every rank solves its own instance (seeded per rank)
    prob = kp.kp_create_from_instance(inst)
    N, M, K = inst.N, inst.M, inst.K
    lam = [torch.zeros(K, dtype=torch.float64, device=dev), torch.zeros(K, dtype=torch.float64, device=dev)]
    R = torch.zeros(K, dtype=torch.float64, device=dev)
    dsum = torch.zeros((), dtype=torch.float64, device=dev)
    psum = torch.zeros((), dtype=torch.float64, device=dev)
    xb = torch.zeros(N * prob.W, dtype=torch.int32, device=dev)
    gp = torch.empty(N * M, dtype=torch.float32, device=dev)
    gl = torch.zeros(K, dtype=torch.float64, device=dev)
    gB = torch.zeros(K, dtype=torch.float64, device=dev)
    up = torch.ones((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    cur = [0]

    def step(i=None, h=None):
        h = prob if h is None else h
        a, b = lam[cur[0]], lam[1 - cur[0]]
        if i is not None:
            ev[i][0].record(stream)
        kp.kp_scd_breakpoints(h, a, R=R, dual_sum=dsum, primal_sum=psum, x_bits=xb)
        if i is not None:
            ev[i][1].record(stream)
        kp.kp_threshold_select(h, a, b)
        kp.kp_dual_backward(h, a, xb, R, up, grad_lambda=gl, grad_p=gp, grad_B=gB)
        cur[0] = 1 - cur[0]

    for _ in range(args.warmup):
        step()
    kp.kp_device_status(prob)
    torch.cuda.synchronize()
    stats0 = kp.kp_select_stats(prob)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    passes = 0
    t_start.record(stream)
    for i in range(args.steps):
        step(i)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    kp.kp_device_status(prob)
    ms_total = t_start.elapsed_time(t_end)
    ms_total = max_over_ranks(ms_total, world, dev)
    pass_ms = [a.elapsed_time(b) for a, b in ev]
    value = N * args.steps * world / (ms_total / 1e3)

    # the dominant kernel: the breakpoint pass (one launch per kp_scd_breakpoints)
    peak, peak_kind = measured_peaks()
    per_user = algo_bytes_per_user(inst)
    k_ms = statistics.mean(pass_ms)
    achieved = N * per_user / (k_ms / 1e3) / 1e9
    traffic = measured_traffic(N, inst.layout)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "user pass, breakpoint mode (csr_pass_kernel MODE_HIST) + finalize",
                "kernel_ms": k_ms, "algo_bytes_per_user": per_user,
                "peak_source": f"{peak_kind} hbm_gbs"}

    # second kernel: the DD / state pass (kp_reduce_consumption: Algorithms 1-2) at the
    # last lambda, timed alone on the same stream
    lam_f = lam[cur[0]]
    st_ms = []
    for rep in range(6):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kp.kp_reduce_consumption(prob, lam_f, R=R, dual_sum=dsum, primal_sum=psum)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= 2:
            st_ms.append(e0.elapsed_time(e1))
    s_ms = statistics.mean(st_ms)
    s_ach = N * per_user / (s_ms / 1e3) / 1e9
    roofline_state = {"bound": "hbm", "achieved": s_ach, "peak": peak, "unit": "GB/s",
                      "frac": s_ach / peak, "traffic": None,
                      "kernel": "user pass, state mode (csr_pass_kernel MODE_STATE) + finalize",
                      "kernel_ms": s_ms, "algo_bytes_per_user": per_user,
                      "peak_source": f"{peak_kind} hbm_gbs"}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic",
              "config": {"workload": inst.name, "N": N, "M": M, "K": K, "layout": inst.layout,
                         "nnz_per_item": 2 if inst.layout == "csr" else None,
                         "instance_bytes": inst.nbytes(),
                         "l2": "inputs (%.1f GB) exceed L2 (129 MB); no flush" % (inst.nbytes() / 1e9),
                         "parallelism": "replicas" if world > 1 else "single GPU",
                         "lambda0": 0.0},
              "roofline": roofline, "roofline_state_pass": roofline_state, "clocks": clocks,
              # per step: pass + finalize + select, 4 x (select + re-run pass), backward;
              # and the rare-knapsack kernel after each of the 5 passes when the instance has some
              "gpu_launches": args.steps * (3 + 2 * 4 + 1 + (5 if kp.kp_info(prob)["rare_blocks"] > 0 else 0))}
    try:
        st1 = kp.kp_select_stats(prob)
        result["config"]["select_passes_last_step"] = st1[0]
    except Exception:
        pass

    # Sec. 5.4 post-processing of x = Algorithm 1 at the last lambda (after the
    # timed region): one untimed run, then three timed on fresh copies of x
    if not args.no_post:
        lam_f = lam[cur[0]]
        x_f = kp.kp_solve_users(prob, lam_f)
        x_w = torch.empty_like(x_f)
        reset = torch.zeros((), dtype=torch.int64, device=dev)
        R_a = torch.zeros(K, dtype=torch.float64, device=dev)
        pp_ms = []
        for rep in range(4):
            x_w.copy_(x_f)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kp.kp_postprocess(prob, lam_f, x_w, reset=reset, R_after=R_a)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                pp_ms.append(e0.elapsed_time(e1))
        kp.kp_device_status(prob)
        R_b = torch.empty_like(R_a)
        g_b = torch.zeros((), dtype=torch.float64, device=dev)
        pr_b = torch.zeros((), dtype=torch.float64, device=dev)
        kp.kp_reduce_consumption(prob, lam_f, R=R_b, primal_sum=pr_b, g=g_b)
        result["quality"] = quality(inst, prob, x_w, R_b, R_a, float(g_b), float(pr_b))
        result["postprocess"] = {
            "ms": statistics.mean(pp_ms), "users_reset": int(reset),
            "over_budget_before": int((R_b > inst.B).sum()),
            "over_budget_after": int((R_a > inst.B).sum()),
            "note": "Sec. 5.4 on x = Algorithm 1 at the lambda after the timed steps; "
                    "radix selection of the last user reset, no sort"}
        del x_f, x_w

    # end to end through the public API from pinned host memory: a fresh job (the
    # instance copied in, a new handle created, SCD from lambda = 0)
    if not args.no_e2e and rank == 0:
        prob.close()
        torch.cuda.empty_cache()
        host = {}
        names = ["p", "b", "user_off", "item_nnz", "val", "kidx", "B"]
        for nm in names:
            t = getattr(inst, nm)
            if t is not None:
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t)
                host[nm] = h
        h2d = sum(h.numel() * h.element_size() for h in host.values())
        lam_h = torch.zeros(K, dtype=torch.float64, pin_memory=True)
        R_h = torch.zeros(K, dtype=torch.float64, pin_memory=True)
        for nm in names:  # the device copies start out empty
            t = getattr(inst, nm)
            if t is not None:
                t.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for nm, h in host.items():
            getattr(inst, nm).copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        prob2 = kp.kp_create_from_instance(inst)   # validation scan, CSR structure, scratch
        lam[0].zero_()
        cur[0] = 0
        for i in range(args.steps):
            step(h=prob2)
        lam_h.copy_(lam[cur[0]], non_blocking=True)
        R_h.copy_(R, non_blocking=True)
        torch.cuda.synchronize()
        e_s = time.perf_counter() - t0
        kp.kp_device_status(prob2)
        prob2.close()
        result["e2e"] = {"value": N * args.steps / e_s, "unit": UNIT,
                         "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 2 * K * 8 / args.steps,
                         "seconds": e_s,
                         "note": "a fresh job of `steps` SCD iterations (+ backward) from lambda = 0 through "
                                 "the C ABI, host wall clock: the instance copied host->device from pinned "
                                 "memory, kp_create (validation scan, CSR structure, scratch) on a new "
                                 "handle whose threshold prediction starts cold, lambda and R read back; "
                                 "unlike `value` it includes the first iterations, whose thresholds lie far "
                                 "from any prediction and take re-run passes"}
    if not args.no_cpu and rank == 0:
        try:
            result["cpu_baseline"] = cpu_baseline(inst, min(args.cpu_sample, N))
        except Exception as e:  # pragma: no cover
            result["cpu_baseline"] = {"value": None, "error": str(e)}
    # batched instances (the workload of many uneven instances), after the
    # headline instance is freed
    if not args.no_batch and rank == 0 and args.workload.startswith("csr"):
        try:
            prob.close()
        except Exception:
            pass
        del inst, gp, xb
        torch.cuda.empty_cache()
        try:
            result["batched"] = batched_measure(args.batch_count, args.batch_nhi, args.batch_steps,
                                                args.batch_warmup, graph=False)
        except Exception as e:  # pragma: no cover
            result["batched"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
