"""Thin Python binding of the C ABI in include/kp.h (argument marshalling only).

Every function has the name of the C entry point it calls, takes torch CUDA
tensors and passes their device pointers and the current CUDA stream.  All
computation happens in libkp.so; if the library is not built or not loadable
the import of this module's functions raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkp.so")

KP_OK, KP_EINVAL, KP_ENOMEM, KP_ECUDA, KP_ETIMEOUT, KP_ESTATE, KP_EDATA = range(7)
KP_B_DENSE, KP_B_CSR = 0, 1
_STATUS = {0: "KP_OK", 1: "KP_EINVAL", 2: "KP_ENOMEM", 3: "KP_ECUDA", 4: "KP_ETIMEOUT",
           5: "KP_ESTATE", 6: "KP_EDATA"}

_lib = None


class KpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class kp_desc(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64),
        ("M", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("p", ctypes.c_void_p),
        ("b_layout", ctypes.c_int32),
        ("b_dense", ctypes.c_void_p),
        ("csr_user_off", ctypes.c_void_p),
        ("csr_item_nnz", ctypes.c_void_p),
        ("csr_val", ctypes.c_void_p),
        ("csr_k", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("L", ctypes.c_int32),
        ("S", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
    ]


EXPORTS = [
    "kp_create", "kp_destroy", "kp_solve_users", "kp_reduce_consumption", "kp_dual_value",
    "kp_dd_step", "kp_scd_breakpoints", "kp_threshold_select", "kp_scd_step",
    "kp_dual_backward", "kp_device_status", "kp_select_stats", "kp_info", "kp_presolve", "kp_postprocess",
    "kp_last_error",
    "kp_version",
    "kp_reduce_consumption_noalloc", "kp_batch_create", "kp_batch_destroy", "kp_batch_layout",
    "kp_batch_reduce_consumption", "kp_batch_dd_step", "kp_batch_scd_step", "kp_batch_device_status",
    "kp_autotune", "kp_limits", "kp_bcd_step", "kp_shard_group_create", "kp_shard_group_destroy",
    "kp_shard_group_scd_step", "kp_scd_step_bucketed", "kp_set_tile", "kp_wait_selftest",
]


def load_library(path: Optional[str] = None):
    """Load libkp.so (raises OSError if it is missing: nothing falls back to the CPU)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    lib = ctypes.CDLL(path or LIB_PATH)
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.kp_create.argtypes = [ctypes.POINTER(kp_desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.kp_destroy.argtypes = [P]
    lib.kp_solve_users.argtypes = [P, P, P, P]
    lib.kp_reduce_consumption.argtypes = [P, P, P, P, P, P, P, P]
    lib.kp_dual_value.argtypes = [P, P, P, P]
    lib.kp_dd_step.argtypes = [P, P, f64, P, P, P]
    lib.kp_scd_breakpoints.argtypes = [P, P, P, P, P, P, P]
    lib.kp_threshold_select.argtypes = [P, P, P, P]
    lib.kp_scd_step.argtypes = [P, P, P, P, P, P, P]
    lib.kp_dual_backward.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.kp_device_status.argtypes = [P, P]
    lib.kp_select_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P]
    lib.kp_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.kp_presolve.argtypes = [P, P, i64, i32, P, P]
    lib.kp_postprocess.argtypes = [P, P, P, P, P, P]
    lib.kp_reduce_consumption_noalloc.argtypes = [ctypes.POINTER(kp_desc), P, P, P, P, P, P, P]
    lib.kp_batch_create.argtypes = [ctypes.POINTER(kp_desc), i32, ctypes.POINTER(ctypes.c_void_p)]
    lib.kp_batch_destroy.argtypes = [P]
    lib.kp_batch_layout.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.kp_batch_reduce_consumption.argtypes = [P, P, P, P, P, P, P]
    lib.kp_batch_dd_step.argtypes = [P, P, f64, P, P]
    lib.kp_batch_scd_step.argtypes = [P, P, P, P]
    lib.kp_batch_device_status.argtypes = [P, P]
    lib.kp_autotune.argtypes = [P, ctypes.POINTER(ctypes.c_int32), P]
    lib.kp_limits.argtypes = [ctypes.POINTER(ctypes.c_int32)]
    lib.kp_bcd_step.argtypes = [P, P, P, P, P, P, P]
    lib.kp_scd_step_bucketed.argtypes = [P, P, f64, P, P]
    lib.kp_set_tile.argtypes = [P, i32, i32]
    lib.kp_wait_selftest.argtypes = [i64, P]
    lib.kp_shard_group_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32, ctypes.POINTER(ctypes.c_void_p)]
    lib.kp_shard_group_destroy.argtypes = [P]
    lib.kp_shard_group_scd_step.argtypes = [P, P, P, P, P, P, P]
    lib.kp_last_error.restype = ctypes.c_char_p
    lib.kp_version.restype = ctypes.c_int
    for name in EXPORTS:
        if name not in ("kp_last_error", "kp_version"):
            getattr(lib, name).restype = i32
    if path is None:
        _lib = lib
    return lib


def _check(status: int):
    if status != KP_OK:
        raise KpError(status, load_library().kp_last_error().decode())


def _ptr(t: Optional[torch.Tensor], dtype=None, name=""):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Problem:
    """A kp_problem handle plus references to the borrowed instance tensors."""

    def __init__(self, handle, N, M, K, layout, keep):
        self.handle = handle
        self.N, self.M, self.K, self.layout = N, M, K, layout
        self.W = (M + 31) // 32
        self._keep = keep

    def close(self):
        if self.handle:
            load_library().kp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(N, M, K, p, B, S, C, b_dense, csr_user_off, csr_item_nnz, csr_val, csr_k):
    d = kp_desc()
    d.N, d.M, d.K = int(N), int(M), int(K)
    d.p = _ptr(p, torch.float32, "p")
    d.B = _ptr(B, torch.float64, "B")
    if b_dense is not None:
        d.b_layout = KP_B_DENSE
        d.b_dense = _ptr(b_dense, torch.float32, "b_dense")
    else:
        d.b_layout = KP_B_CSR
        d.csr_user_off = _ptr(csr_user_off, torch.int64, "csr_user_off")
        d.csr_item_nnz = _ptr(csr_item_nnz, torch.uint8, "csr_item_nnz")
        d.csr_val = _ptr(csr_val, torch.float32, "csr_val")
        d.csr_k = _ptr(csr_k, torch.int16, "csr_k")
    Sa = (ctypes.c_uint64 * max(1, len(S)))(*[int(s) for s in S])
    Ca = (ctypes.c_int32 * max(1, len(C)))(*[int(c) for c in C])
    d.L = len(S)
    d.S = ctypes.cast(Sa, ctypes.c_void_p)
    d.C = ctypes.cast(Ca, ctypes.c_void_p)
    return d, (Sa, Ca)


def kp_reduce_consumption_noalloc(N: int, M: int, K: int, p: torch.Tensor, B: torch.Tensor,
                                  S: Sequence[int], C: Sequence[int], lam: torch.Tensor,
                                  b_dense=None, csr_user_off=None, csr_item_nnz=None, csr_val=None,
                                  csr_k=None, R=None, dual_sum=None, primal_sum=None, g=None,
                                  x_bits=None, stream=None):
    """Allocation-free consumption pass (no handle; the instance is described per call)."""
    d, keep = _desc(N, M, K, p, B, S, C, b_dense, csr_user_off, csr_item_nnz, csr_val, csr_k)
    _check(load_library().kp_reduce_consumption_noalloc(
        ctypes.byref(d), _ptr(lam, torch.float64, "lambda"), _ptr(R, torch.float64, "R"),
        _ptr(dual_sum, torch.float64, "dual_sum"), _ptr(primal_sum, torch.float64, "primal_sum"),
        _ptr(g, torch.float64, "g"), _ptr(x_bits, None, "x_bits"), _stream(stream)))
    del keep


def kp_create(N: int, M: int, K: int, p: torch.Tensor, B: torch.Tensor, S: Sequence[int],
              C: Sequence[int], b_dense: Optional[torch.Tensor] = None,
              csr_user_off: Optional[torch.Tensor] = None,
              csr_item_nnz: Optional[torch.Tensor] = None,
              csr_val: Optional[torch.Tensor] = None,
              csr_k: Optional[torch.Tensor] = None) -> Problem:
    lib = load_library()
    d = kp_desc()
    d.N, d.M, d.K = int(N), int(M), int(K)
    d.p = _ptr(p, torch.float32, "p")
    d.B = _ptr(B, torch.float64, "B")
    if b_dense is not None:
        d.b_layout = KP_B_DENSE
        d.b_dense = _ptr(b_dense, torch.float32, "b_dense")
    else:
        d.b_layout = KP_B_CSR
        d.csr_user_off = _ptr(csr_user_off, torch.int64, "csr_user_off")
        d.csr_item_nnz = _ptr(csr_item_nnz, torch.uint8, "csr_item_nnz")
        d.csr_val = _ptr(csr_val, torch.float32, "csr_val")
        d.csr_k = _ptr(csr_k, torch.int16, "csr_k")
    Sa = (ctypes.c_uint64 * max(1, len(S)))(*[int(s) for s in S])
    Ca = (ctypes.c_int32 * max(1, len(C)))(*[int(c) for c in C])
    d.L = len(S)
    d.S = ctypes.cast(Sa, ctypes.c_void_p)
    d.C = ctypes.cast(Ca, ctypes.c_void_p)
    h = ctypes.c_void_p()
    _check(lib.kp_create(ctypes.byref(d), ctypes.byref(h)))
    keep = (p, B, b_dense, csr_user_off, csr_item_nnz, csr_val, csr_k)
    return Problem(h, int(N), int(M), int(K), d.b_layout, keep)


def kp_create_from_instance(inst) -> Problem:
    """kp_create for a paper_2002_00352_gb300.gen.Instance on a CUDA device."""
    if inst.layout == "dense":
        return kp_create(inst.N, inst.M, inst.K, inst.p, inst.B, inst.S, inst.C, b_dense=inst.b)
    return kp_create(inst.N, inst.M, inst.K, inst.p, inst.B, inst.S, inst.C,
                     csr_user_off=inst.user_off, csr_item_nnz=inst.item_nnz, csr_val=inst.val,
                     csr_k=inst.kidx)


def _x_bits(prob: Problem, x_bits):
    if x_bits is None:
        x_bits = torch.empty(prob.N * prob.W, dtype=torch.int32, device="cuda")
    return x_bits


def kp_solve_users(prob: Problem, lam: torch.Tensor, x_bits=None, stream=None) -> torch.Tensor:
    x_bits = _x_bits(prob, x_bits)
    _check(load_library().kp_solve_users(prob.handle, _ptr(lam, torch.float64, "lambda"),
                                         _ptr(x_bits, None, "x_bits"), _stream(stream)))
    return x_bits


def kp_reduce_consumption(prob: Problem, lam, R=None, dual_sum=None, primal_sum=None, g=None,
                          x_bits=None, stream=None):
    _check(load_library().kp_reduce_consumption(
        prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(R, torch.float64, "R"),
        _ptr(dual_sum, torch.float64, "dual_sum"), _ptr(primal_sum, torch.float64, "primal_sum"),
        _ptr(g, torch.float64, "g"), _ptr(x_bits, None, "x_bits"), _stream(stream)))


def kp_dual_value(prob: Problem, lam, g, stream=None):
    _check(load_library().kp_dual_value(prob.handle, _ptr(lam, torch.float64, "lambda"),
                                        _ptr(g, torch.float64, "g"), _stream(stream)))


def kp_dd_step(prob: Problem, lam, alpha: float, lam_next, R=None, stream=None):
    _check(load_library().kp_dd_step(prob.handle, _ptr(lam, torch.float64, "lambda"), float(alpha),
                                     _ptr(lam_next, torch.float64, "lambda_next"),
                                     _ptr(R, torch.float64, "R"), _stream(stream)))


def kp_scd_breakpoints(prob: Problem, lam, R=None, dual_sum=None, primal_sum=None, x_bits=None,
                       stream=None):
    _check(load_library().kp_scd_breakpoints(
        prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(R, torch.float64, "R"),
        _ptr(dual_sum, torch.float64, "dual_sum"), _ptr(primal_sum, torch.float64, "primal_sum"),
        _ptr(x_bits, None, "x_bits"), _stream(stream)))


def kp_threshold_select(prob: Problem, lam, lam_next, stream=None):
    _check(load_library().kp_threshold_select(prob.handle, _ptr(lam, torch.float64, "lambda"),
                                              _ptr(lam_next, torch.float64, "lambda_next"),
                                              _stream(stream)))


def kp_scd_step(prob: Problem, lam, lam_next, R=None, dual_sum=None, primal_sum=None, stream=None):
    _check(load_library().kp_scd_step(
        prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(lam_next, torch.float64, "lambda_next"),
        _ptr(R, torch.float64, "R"), _ptr(dual_sum, torch.float64, "dual_sum"),
        _ptr(primal_sum, torch.float64, "primal_sum"), _stream(stream)))


def kp_bcd_step(prob: Problem, lam, block, lam_next, dual_sum=None, primal_sum=None, stream=None):
    """Block / cyclic coordinate descent (Sec. 4.3.2): block = uint8 [K] device flags."""
    _check(load_library().kp_bcd_step(prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(block, torch.uint8, "block"),
                                      _ptr(lam_next, torch.float64, "lambda_next"),
                                      _ptr(dual_sum, torch.float64, "dual_sum"),
                                      _ptr(primal_sum, torch.float64, "primal_sum"), _stream(stream)))


def kp_scd_step_bucketed(prob: Problem, lam, delta: float, lam_next, stream=None):
    """Algorithm 4 with the bucketed, interpolated Reduce of Sec. 5.2 (bucket
    width delta * lambda_k, or delta where lambda_k = 0)."""
    _check(load_library().kp_scd_step_bucketed(prob.handle, _ptr(lam, torch.float64, "lambda"), float(delta),
                                               _ptr(lam_next, torch.float64, "lambda_next"), _stream(stream)))


def kp_set_tile(prob: Problem, users: int, staging: int):
    """Dense instances: users per shared-memory tile and staging mode (0 loads by the
    threads, 1 double-buffered bulk asynchronous copies)."""
    _check(load_library().kp_set_tile(prob.handle, int(users), int(staging)))


def kp_wait_selftest(limit_ns: int, stream=None):
    """Runs the bounded-wait self-test; raises KpError with status KP_ETIMEOUT (expected)."""
    _check(load_library().kp_wait_selftest(int(limit_ns), _stream(stream)))


def kp_dual_backward(prob: Problem, lam, x_bits, R, upstream, grad_lambda=None, grad_p=None,
                     grad_B=None, stream=None):
    _check(load_library().kp_dual_backward(
        prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(x_bits, None, "x_bits"),
        _ptr(R, torch.float64, "R"), _ptr(upstream, torch.float64, "upstream"),
        _ptr(grad_lambda, torch.float64, "grad_lambda"), _ptr(grad_p, torch.float32, "grad_p"),
        _ptr(grad_B, torch.float64, "grad_B"), _stream(stream)))


def kp_device_status(prob: Problem, stream=None):
    _check(load_library().kp_device_status(prob.handle, _stream(stream)))


def kp_select_stats(prob: Problem, stream=None):
    out = (ctypes.c_int64 * 3)()
    _check(load_library().kp_select_stats(prob.handle, out, _stream(stream)))
    return list(out)


def kp_presolve(prob: Problem, users, iters: int, lambda0=None, stream=None):
    """Sec. 5.3: SCD on the sampled users (device int64 tensor) with budgets scaled by
    n / N; returns (or fills) lambda0, a float64 device tensor of K entries."""
    if lambda0 is None:
        lambda0 = torch.empty(prob.K, dtype=torch.float64, device="cuda")
    users = users.contiguous()
    _check(load_library().kp_presolve(prob.handle, _ptr(users, torch.int64, "users"), users.numel(),
                                      int(iters), _ptr(lambda0, torch.float64, "lambda0"), _stream(stream)))
    return lambda0


def kp_postprocess(prob: Problem, lam, x_bits, reset=None, R_after=None, stream=None):
    """Sec. 5.4: resets users in order of their cost-adjusted group profit until x
    (int32 words, modified in place) fits every budget.  Returns (reset, R_after):
    a device int64 scalar tensor and a float64 [K] device tensor."""
    if reset is None:
        reset = torch.empty((), dtype=torch.int64, device="cuda")
    if R_after is None:
        R_after = torch.empty(prob.K, dtype=torch.float64, device="cuda")
    _check(load_library().kp_postprocess(
        prob.handle, _ptr(lam, torch.float64, "lambda"), _ptr(x_bits, None, "x_bits"),
        _ptr(reset, torch.int64, "reset"), _ptr(R_after, torch.float64, "R_after"), _stream(stream)))
    return reset, R_after


def kp_info(prob: Problem) -> dict:
    """Launch layout of a handle (see include/kp.h)."""
    out = (ctypes.c_int64 * 4)()
    _check(load_library().kp_info(prob.handle, out))
    return {"pass_blocks": out[0], "rare_users": out[1], "rare_blocks": out[2], "buffer_per_block": out[3]}


def kp_limits() -> dict:
    """Limits of the library (include/kp.h: KP_MAX_M, KP_MAX_L, KP_MAX_K)."""
    out = (ctypes.c_int32 * 3)()
    _check(load_library().kp_limits(out))
    return {"max_m": out[0], "max_l": out[1], "max_k": out[2]}


def kp_autotune(prob: Problem, stream=None) -> int:
    """Tile-size autotuner of the dense pass; returns the chosen users per tile."""
    out = ctypes.c_int32(0)
    _check(load_library().kp_autotune(prob.handle, ctypes.byref(out), _stream(stream)))
    return int(out.value)


def kp_version() -> int:
    return int(load_library().kp_version())


def unpack_x(x_bits: torch.Tensor, N: int, M: int) -> torch.Tensor:
    """x bits (int32 words, W per user) -> uint8 [N, M] tensor on the same device."""
    W = (M + 31) // 32
    w = x_bits.view(N, W).to(torch.int64) & 0xFFFFFFFF
    j = torch.arange(M, device=x_bits.device)
    return ((w[:, j // 32] >> (j % 32)) & 1).to(torch.uint8)


class Batch:
    """A kp_batch handle: many dense instances solved by shared launches."""

    def __init__(self, handle, insts, koff):
        self.handle = handle
        self.insts = insts
        self.koff = koff                    # python list, len count + 1
        self.count = len(insts)
        self.totK = koff[-1]
        self.xoff = [0]
        for inst in insts:
            self.xoff.append(self.xoff[-1] + inst.N * ((inst.M + 31) // 32))

    def close(self):
        if self.handle:
            load_library().kp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kp_batch_create(insts) -> Batch:
    """kp_batch_create over a list of dense gen.Instance on the GPU."""
    lib = load_library()
    arr = (kp_desc * len(insts))()
    keep = []
    for q, inst in enumerate(insts):
        d, k = _desc(inst.N, inst.M, inst.K, inst.p, inst.B, inst.S, inst.C, inst.b, None, None, None, None)
        arr[q] = d
        keep.append(k)
    h = ctypes.c_void_p()
    _check(lib.kp_batch_create(arr, len(insts), ctypes.byref(h)))
    koff = (ctypes.c_int64 * (len(insts) + 1))()
    _check(lib.kp_batch_layout(h, koff))
    return Batch(h, list(insts), list(koff))


def kp_batch_reduce_consumption(batch: Batch, lam, R=None, dual_sum=None, primal_sum=None, x_bits=None,
                                stream=None):
    _check(load_library().kp_batch_reduce_consumption(
        batch.handle, _ptr(lam, torch.float64, "lambda"), _ptr(R, torch.float64, "R"),
        _ptr(dual_sum, torch.float64, "dual_sum"), _ptr(primal_sum, torch.float64, "primal_sum"),
        _ptr(x_bits, None, "x_bits"), _stream(stream)))


def kp_batch_dd_step(batch: Batch, lam, alpha, lam_next, stream=None):
    _check(load_library().kp_batch_dd_step(batch.handle, _ptr(lam, torch.float64, "lambda"), float(alpha),
                                           _ptr(lam_next, torch.float64, "lambda_next"), _stream(stream)))


def kp_batch_scd_step(batch: Batch, lam, lam_next, stream=None):
    _check(load_library().kp_batch_scd_step(batch.handle, _ptr(lam, torch.float64, "lambda"),
                                            _ptr(lam_next, torch.float64, "lambda_next"), _stream(stream)))


def kp_batch_device_status(batch: Batch, stream=None):
    _check(load_library().kp_batch_device_status(batch.handle, _stream(stream)))


class ShardGroup:
    """A kp_shard_group: one instance whose users are split over several handles."""

    def __init__(self, handle, shards):
        self.handle = handle
        self.shards = shards    # keeps the handles (and their instances) alive
        self.K = shards[0].K

    def close(self):
        if self.handle:
            load_library().kp_shard_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kp_shard_group_create(shards) -> ShardGroup:
    arr = (ctypes.c_void_p * len(shards))(*[s.handle for s in shards])
    out = ctypes.c_void_p()
    _check(load_library().kp_shard_group_create(arr, len(shards), ctypes.byref(out)))
    return ShardGroup(out, list(shards))


def kp_shard_group_scd_step(group: ShardGroup, lam, lam_next, R=None, dual_sum=None, primal_sum=None,
                            stream=None):
    _check(load_library().kp_shard_group_scd_step(group.handle, _ptr(lam, torch.float64, "lambda"),
                                                  _ptr(lam_next, torch.float64, "lambda_next"),
                                                  _ptr(R, torch.float64, "R"),
                                                  _ptr(dual_sum, torch.float64, "dual_sum"),
                                                  _ptr(primal_sum, torch.float64, "primal_sum"), _stream(stream)))


def kp_create_user_range(inst, u0: int, u1: int) -> Problem:
    """A handle over the users [u0, u1) of an instance (a shard): views of their rows."""
    M, K = inst.M, inst.K
    p = inst.p[u0 * M:u1 * M]
    if inst.layout == "dense":
        return kp_create(u1 - u0, M, K, p, inst.B, inst.S, inst.C, b_dense=inst.b[u0 * M * K:u1 * M * K])
    return kp_create(u1 - u0, M, K, p, inst.B, inst.S, inst.C, csr_user_off=inst.user_off[u0:u1 + 1],
                     csr_item_nnz=inst.item_nnz[u0 * M:u1 * M], csr_val=inst.val, csr_k=inst.kidx)
