"""Writes tests/golden/oracle_tiny.json from the CPU oracle only.

A tiny dense instance with explicit numbers (drawn once from numpy with a fixed
seed, rounded to 4 decimals so that they are exact in the JSON and close to
float32) and the oracle's DD and SCD trajectories on it.  The GPU tests replay
the same inputs through the C ABI and compare.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402


def main():
    rng = np.random.default_rng(20200201)
    N, M, K = 64, 6, 3
    # float32-representable inputs: the GPU path stores p and b in float32
    p = rng.uniform(0, 1, size=(N, M)).astype(np.float32).astype(np.float64)
    b = rng.uniform(0, 1, size=(N, M, K)).astype(np.float32).astype(np.float64)
    S = [0b000111, 0b111000, 0b111111]
    C = [2, 1, 2]
    B = 0.15 * b.sum(axis=(0, 1))
    lam = np.zeros(K)
    scd = [lam.tolist()]
    for _ in range(8):
        lam, _, _ = oracle.scd_step(p, b, S, C, lam, B)
        scd.append(lam.tolist())
    alpha = 2e-3
    lam = np.zeros(K)
    dd = [lam.tolist()]
    for _ in range(8):
        _, R, _, _ = oracle.user_pass(p, b, S, C, lam)
        lam = oracle.dd_update(lam, R, B, alpha)
        dd.append(lam.tolist())
    out = dict(
        source="oracle/ (tests/golden/make_golden.py)",
        N=N, M=M, K=K, S=S, C=C, B=B.tolist(), alpha=alpha,
        p=p.reshape(-1).tolist(), b=b.reshape(-1).tolist(),
        scd_lambda=scd, dd_lambda=dd,
    )
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
