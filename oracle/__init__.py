"""FP64 CPU oracle for the dual-decomposition knapsack method (arXiv 2002.00352).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never touches it, and it
shares no code with that path.

The arithmetic lives in ``kp_oracle.c`` (plain C, double precision, one
routine per step of the paper: Sec. 4.2 and Algorithm 1 for the per-user
greedy, Eq. (14) and Algorithm 2 for dual descent, Algorithms 3-4 for
synchronous coordinate descent, Algorithm 5 for its one-item-per-knapsack
special case, Sec. 5.4 for post-processing).  This module
marshals numpy arrays into those routines and converts the CSR storage of
``b`` into the dense layout the oracle reads; the bucketed Reduce of Sec. 5.2
(bucket_ids ... bucket_step), a few lines over the emitted pairs, is numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kp_oracle.c")
_HDR = os.path.join(_HERE, "kp_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libkp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.kpo_reduced_costs.argtypes = [i32, i32, P, P, P, P]
    lib.kpo_topo_order.argtypes = [i32, P, P]
    lib.kpo_is_hierarchical.argtypes = [i32, P]
    lib.kpo_is_hierarchical.restype = i32
    lib.kpo_greedy.argtypes = [i32, i32, P, P, P, P, P]
    lib.kpo_brute_force.argtypes = [i32, i32, P, P, P, P]
    lib.kpo_brute_force.restype = f64
    lib.kpo_user_pass.argtypes = [i64, i32, i32, P, P, i32, P, P, P, P, P, P, P]
    lib.kpo_dd_update.argtypes = [i32, P, P, P, f64, P]
    lib.kpo_dual_value.argtypes = [i64, i32, i32, P, P, i32, P, P, P, P]
    lib.kpo_dual_value.restype = f64
    lib.kpo_scd_map_user.argtypes = [i32, i32, P, P, i32, P, P, P, P, P, P, P, P]
    lib.kpo_scd_reduce.argtypes = [i64, P, P, f64]
    lib.kpo_scd_reduce.restype = f64
    lib.kpo_scd_step.argtypes = [i64, i32, i32, P, P, i32, P, P, P, P, P, P, P]
    lib.kpo_scd_step.restype = i64
    lib.kpo_scd_map_all.argtypes = [i64, i32, i32, P, P, i32, P, P, P, i64, P, P, P, P]
    lib.kpo_scd_map_all.restype = i64
    lib.kpo_postprocess.argtypes = [i64, i32, i32, P, P, P, P, P]
    lib.kpo_postprocess.restype = i64
    lib.kpo_alg5_map_user.argtypes = [i32, P, P, i32, P, P, P, P, P]
    lib.kpo_alg5_step.argtypes = [i64, i32, P, P, i32, P, P, P]
    lib.kpo_alg5_step.restype = i64
    lib.kpo_num_threads.restype = i32
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tree(S, C):
    S = np.ascontiguousarray(np.asarray(S, dtype=np.uint64).reshape(-1))
    C = np.ascontiguousarray(np.asarray(C, dtype=np.int32).reshape(-1))
    assert S.shape == C.shape
    return S, C


def num_threads() -> int:
    return int(_load().kpo_num_threads())


def is_hierarchical(S) -> bool:
    S, _ = _tree(S, np.zeros(len(S)))
    return bool(_load().kpo_is_hierarchical(len(S), _ptr(S)))


def topo_order(S) -> np.ndarray:
    S, _ = _tree(S, np.zeros(len(S)))
    topo = np.zeros(max(len(S), 1), dtype=np.int32)
    _load().kpo_topo_order(len(S), _ptr(S), _ptr(topo))
    return topo[: len(S)]


def reduced_costs(p_i, b_i, lam) -> np.ndarray:
    """p~_j = p_j - sum_k lam_k b_jk for one user (p_i [M], b_i [M, K])."""
    p_i, b_i, lam = _f64(p_i), _f64(b_i), _f64(lam)
    M, K = b_i.shape
    out = np.zeros(M)
    _load().kpo_reduced_costs(M, K, _ptr(p_i), _ptr(b_i), _ptr(lam), _ptr(out))
    return out


def greedy(pt, S, C) -> np.ndarray:
    """Algorithm 1 on one user's cost-adjusted profits."""
    pt = _f64(pt)
    S, C = _tree(S, C)
    topo = topo_order(S) if len(S) else np.zeros(1, dtype=np.int32)
    topo = np.ascontiguousarray(topo, dtype=np.int32)
    x = np.zeros(len(pt), dtype=np.int32)
    _load().kpo_greedy(len(pt), len(S), _ptr(S), _ptr(C), _ptr(topo), _ptr(pt), _ptr(x))
    return x


def brute_force(pt, S, C):
    """Exhaustive optimum of Eq. (11)-(13): (objective, x)."""
    pt = _f64(pt)
    S, C = _tree(S, C)
    assert len(pt) <= 24
    x = np.zeros(len(pt), dtype=np.int32)
    v = _load().kpo_brute_force(len(pt), len(S), _ptr(S), _ptr(C), _ptr(pt), _ptr(x))
    return float(v), x


def user_pass(p, b, S, C, lam, want_x: bool = True):
    """Algorithm 2 Map+Reduce at lam: (x [N,M] or None, R [K], dual, primal)."""
    p, b, lam = _f64(p), _f64(b), _f64(lam)
    S, C = _tree(S, C)
    N, M, K = b.shape
    x = np.zeros((N, M), dtype=np.int32) if want_x else None
    R = np.zeros(K)
    dual = ctypes.c_double()
    primal = ctypes.c_double()
    _load().kpo_user_pass(N, M, K, _ptr(p), _ptr(b), len(S), _ptr(S), _ptr(C), _ptr(lam),
                          _ptr(x) if x is not None else None, _ptr(R),
                          ctypes.byref(dual), ctypes.byref(primal))
    return x, R, dual.value, primal.value


def dd_update(lam, R, B, alpha) -> np.ndarray:
    """Eq. (14)."""
    lam, R, B = _f64(lam), _f64(R), _f64(B)
    out = np.zeros_like(lam)
    _load().kpo_dd_update(len(lam), _ptr(lam), _ptr(R), _ptr(B), float(alpha), _ptr(out))
    return out


def dual_value(p, b, S, C, lam, B) -> float:
    """g(lam) of Eq. (5): sum of per-user maxima plus lam . B."""
    p, b, lam, B = _f64(p), _f64(b), _f64(lam), _f64(B)
    S, C = _tree(S, C)
    N, M, K = b.shape
    return float(_load().kpo_dual_value(N, M, K, _ptr(p), _ptr(b), len(S), _ptr(S), _ptr(C),
                                        _ptr(lam), _ptr(B)))


def scd_map_user(p_i, b_i, S, C, lam):
    """Algorithms 3-4 Map for one user: arrays (k, v1, v2) of emitted pairs."""
    p_i, b_i, lam = _f64(p_i), _f64(b_i), _f64(lam)
    S, C = _tree(S, C)
    M, K = b_i.shape
    cap = K * (M + M * (M - 1) // 2) + 1
    ek = np.zeros(cap, dtype=np.int32)
    v1 = np.zeros(cap)
    v2 = np.zeros(cap)
    n = ctypes.c_int64(0)
    topo = np.ascontiguousarray(topo_order(S) if len(S) else np.zeros(1), dtype=np.int32)
    _load().kpo_scd_map_user(M, K, _ptr(p_i), _ptr(b_i), len(S), _ptr(S), _ptr(C), _ptr(topo),
                             _ptr(lam), ctypes.byref(n), _ptr(ek), _ptr(v1), _ptr(v2))
    m = n.value
    return ek[:m].copy(), v1[:m].copy(), v2[:m].copy()


def scd_map_users(p, b, S, C, lam, users=None):
    """Algorithms 3-4 Map for every user (or the listed ones): arrays (user, k, v1, v2)
    of all emitted pairs, users ascending (kpo_scd_map_all: scd_map_user per user)."""
    p, b, lam = _f64(p), _f64(b), _f64(lam)
    S, C = _tree(S, C)
    idx = None if users is None else np.asarray(users, dtype=np.int64)
    if idx is not None:
        p, b = _f64(p[idx]), _f64(b[idx])
    N, M, K = b.shape
    cap = max(1024, 4 * N * K)
    while True:
        eu = np.zeros(cap, dtype=np.int64)
        ek = np.zeros(cap, dtype=np.int32)
        v1 = np.zeros(cap)
        v2 = np.zeros(cap)
        n = _load().kpo_scd_map_all(N, M, K, _ptr(p), _ptr(b), len(S), _ptr(S), _ptr(C), _ptr(lam),
                                    cap, _ptr(eu), _ptr(ek), _ptr(v1), _ptr(v2))
        if n < 0:
            raise MemoryError("oracle scd_map_all: allocation failed")
        if n <= cap:
            break
        cap = int(n)
    eu = eu[:n]
    if idx is not None:
        eu = idx[eu]
    return eu.copy(), ek[:n].copy(), v1[:n].copy(), v2[:n].copy()


def scd_reduce(v1, v2, Bk) -> float:
    """Algorithm 4 Reduce for one knapsack."""
    v1, v2 = _f64(v1), _f64(v2)
    return float(_load().kpo_scd_reduce(len(v1), _ptr(v1), _ptr(v2), float(Bk)))


def scd_step(p, b, S, C, lam, B):
    """One Algorithm 4 iteration: (lam_next [K], emitted pairs per k, their mass per k)."""
    p, b, lam, B = _f64(p), _f64(b), _f64(lam), _f64(B)
    S, C = _tree(S, C)
    N, M, K = b.shape
    out = np.zeros(K)
    nemit = np.zeros(K, dtype=np.int64)
    mass = np.zeros(K)
    r = _load().kpo_scd_step(N, M, K, _ptr(p), _ptr(b), len(S), _ptr(S), _ptr(C), _ptr(lam),
                             _ptr(B), _ptr(out), _ptr(nemit), _ptr(mass))
    if r < 0:
        raise MemoryError("oracle scd_step: allocation failed")
    return out, nemit, mass


def bcd_step(p, b, S, C, lam, B, block):
    """One block coordinate-descent iteration (Sec. 4.3.2): the Reduce of Algorithm 4
    at lam for the knapsacks in `block` (boolean [K]), lam unchanged elsewhere
    (composition of scd_step)."""
    lam = _f64(lam)
    nxt, _, _ = scd_step(p, b, S, C, lam, B)
    block = np.asarray(block, dtype=bool)
    return np.where(block, nxt, lam)


def bucket_ids(v1, lam_k, delta_k) -> np.ndarray:
    """Sec. 5.2 bucket of each candidate v1 around lam_k (reading of the bucket
    formula: id 0 where |d| < Delta, else sign(d) (1 + floor(log2(|d| / Delta))),
    d = v1 - lam_k, clamped to [-127, 127]).  The id is an integer decided by
    floating point, so it is taken in the precision of the kernel: v1, lam_k and
    Delta rounded to FP32, d and |d| / Delta rounded to FP32 (numpy float32
    arithmetic is IEEE round-to-nearest), floor(log2) exact from frexp."""
    v = np.asarray(v1, dtype=np.float64).astype(np.float32)
    lt = np.float32(lam_k)
    dl = np.float32(delta_k)
    d = (v - lt).astype(np.float32)
    with np.errstate(over="ignore"):  # overflow to inf is part of the definition (clamped)
        a = (np.abs(d) / dl).astype(np.float32)
    ids = np.zeros(v.shape, dtype=np.int64)
    big = a >= np.float32(1.0)
    _, e = np.frexp(a[big])  # a = m 2^e with m in [0.5, 1): 1 + floor(log2 a) = e
    e = np.where(np.isinf(a[big]), 127, e).astype(np.int64)
    e = np.minimum(e, 127)
    ids[big] = np.where(d[big] < 0, -e, e)
    return ids


def bucket_delta(lam_k, delta) -> np.float32:
    """Delta_k of a bucketed step: delta * lam_k (delta where lam_k = 0), in FP32,
    at least the smallest normal FP32 value."""
    dl = np.float32(delta * lam_k if lam_k > 0 else delta)
    return max(dl, np.finfo(np.float32).tiny)


def bucket_range(id_, lam_k, delta_k):
    """[lo, hi) of bucket id_ (FP64 from the FP32 lam_k and Delta_k)."""
    lt, dl = float(np.float32(lam_k)), float(np.float32(delta_k))
    if id_ == 0:
        return lt - dl, lt + dl
    if id_ > 0:
        return lt + dl * 2.0 ** (id_ - 1), lt + dl * 2.0 ** id_
    return lt - dl * 2.0 ** (-id_), lt - dl * 2.0 ** (-id_ - 1)


def bucket_reduce(v1, v2, Bk, lam_k, delta_k, ids=None) -> float:
    """Sec. 5.2 Reduce for one knapsack: bucket the candidates around lam_k, sum
    v2 per bucket, walk down from the highest bucket to the first one whose mass
    takes the cumulative mass above Bk, and interpolate linearly inside it (its
    mass taken as uniform over its range); 0 if the whole mass is within Bk
    (Algorithm 4).  ids: the candidates' buckets if already known."""
    v2 = np.asarray(v2, dtype=np.float64)
    if ids is None:
        ids = bucket_ids(v1, lam_k, delta_k)
    mass = np.zeros(256)
    np.add.at(mass, np.asarray(ids) + 128, v2)
    A = 0.0
    for b in range(255, 0, -1):
        if A + mass[b] > Bk:
            lo, hi = bucket_range(b - 128, lam_k, delta_k)
            f = (Bk - A) / mass[b]
            lam = min(max(hi - f * (hi - lo), lo), hi)
            return max(lam, 0.0)
        A += mass[b]
    return 0.0


def bucket_step(p, b, S, C, lam, B, delta):
    """One Algorithm 4 iteration with the Sec. 5.2 bucketed Reduce: the Map at lam
    (scd_map_users), then bucket_reduce per knapsack with Delta_k = bucket_delta."""
    lam, B = _f64(lam), _f64(B)
    _, ek, v1, v2 = scd_map_users(p, b, S, C, lam)
    out = np.zeros(len(lam))
    for k in range(len(lam)):
        sel = ek == k
        out[k] = bucket_reduce(v1[sel], v2[sel], B[k], lam[k], bucket_delta(lam[k], delta))
    return out


def presolve(p, b, S, C, B, users, iters):
    """Sec. 5.3 pre-solving by sampling: `iters` steps of Algorithm 4 from lambda = 0
    on the users `users` with every budget scaled by n / N (composition of the
    routines above)."""
    users = np.asarray(users, dtype=np.int64)
    p, b = _f64(p), _f64(b)
    N = p.shape[0]
    ps, bs = p[users], b[users]
    Bs = _f64(B) * (len(users) / N)
    lam = np.zeros(b.shape[2])
    for _ in range(int(iters)):
        lam, _, _ = scd_step(ps, bs, S, C, lam, Bs)
    return lam


def postprocess(p, b, lam, B, x):
    """Sec. 5.4: returns (feasible x, number of users reset)."""
    p, b, lam, B = _f64(p), _f64(b), _f64(lam), _f64(B)
    x = np.ascontiguousarray(x, dtype=np.int32).copy()
    N, M, K = b.shape
    r = _load().kpo_postprocess(N, M, K, _ptr(p), _ptr(b), _ptr(lam), _ptr(B), _ptr(x))
    return x, int(r)


def alg5_map_user(p_i, bdiag_i, Q, lam):
    """Algorithm 5 (Sec. 5.1) for one user with M = K items, item k consuming only
    knapsack k (b_ikk = bdiag_i[k]), at most Q items: arrays (k, v1, v2)."""
    p_i, bdiag_i, lam = _f64(p_i), _f64(bdiag_i), _f64(lam)
    K = p_i.shape[0]
    ek = np.zeros(K, dtype=np.int32)
    v1 = np.zeros(K)
    v2 = np.zeros(K)
    n = ctypes.c_int64(0)
    _load().kpo_alg5_map_user(K, _ptr(p_i), _ptr(bdiag_i), int(Q), _ptr(lam), ctypes.byref(n),
                              _ptr(ek), _ptr(v1), _ptr(v2))
    m = n.value
    return ek[:m].copy(), v1[:m].copy(), v2[:m].copy()


def alg5_map_users(p, bdiag, Q, lam):
    """Algorithm 5 for every user (p, bdiag [N, K]): arrays (user, k, v1, v2)."""
    p, bdiag = _f64(p), _f64(bdiag)
    us, ks, v1s, v2s = [], [], [], []
    for i in range(p.shape[0]):
        k, v1, v2 = alg5_map_user(p[i], bdiag[i], Q, lam)
        us.append(np.full(len(k), i, dtype=np.int64))
        ks.append(k)
        v1s.append(v1)
        v2s.append(v2)
    return np.concatenate(us), np.concatenate(ks), np.concatenate(v1s), np.concatenate(v2s)


def alg5_step(p, bdiag, Q, lam, B):
    """One Algorithm 4 iteration with Algorithm 5 as Map (p, bdiag [N, K]): lam_next [K]."""
    p, bdiag, lam, B = _f64(p), _f64(bdiag), _f64(lam), _f64(B)
    N, K = p.shape
    out = np.zeros(K)
    r = _load().kpo_alg5_step(N, K, _ptr(p), _ptr(bdiag), int(Q), _ptr(lam), _ptr(B), _ptr(out))
    if r < 0:
        raise MemoryError("oracle alg5_step: allocation failed")
    return out


def densify_csr(N, M, K, user_off, item_nnz, val, kidx) -> np.ndarray:
    """Dense [N, M, K] float64 view of a CSR-stored b (layout conversion only).

    user_off [N+1] indexes val/kidx; the entries of user i are its items'
    entries in item order, item j owning item_nnz[i*M+j] consecutive entries.
    """
    user_off = np.asarray(user_off, dtype=np.int64)
    item_nnz = np.asarray(item_nnz, dtype=np.int64).reshape(N * M)
    val = np.asarray(val, dtype=np.float64)
    kidx = np.asarray(kidx, dtype=np.int64)
    e0, e1 = int(user_off[0]), int(user_off[N])
    assert int(item_nnz.sum()) == e1 - e0, "user_off inconsistent with item_nnz"
    owner = np.repeat(np.arange(N * M, dtype=np.int64), item_nnz)
    b = np.zeros((N * M, K))
    np.add.at(b, (owner, kidx[e0:e1]), val[e0:e1])
    return b.reshape(N, M, K)
