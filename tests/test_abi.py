"""The C-ABI library: builds for sm_103a, loads, and exports every entry point that
include/kp.h declares (no compute calls: no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2002_00352_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["kp_create", "kp_solve_users", "kp_reduce_consumption", "kp_scd_breakpoints",
                 "kp_threshold_select", "kp_dd_step", "kp_dual_value", "kp_dual_backward"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(kp_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_exports(lib_path):
    from paper_2002_00352_gb300 import kp
    lib = kp.load_library(lib_path)
    for n in _declared():
        assert hasattr(lib, n)
        assert n in kp.EXPORTS
    assert lib.kp_version() >= 100


def test_sm103a_only(lib_path):
    from paper_2002_00352_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_limits_match_header(lib_path):
    """kp_limits reports the enum of include/kp.h (host values, no device work)."""
    src = open(os.path.join(ROOT, "include", "kp.h")).read()
    want = {n: int(v) for n, v in re.findall(r"\b(KP_MAX_[MLK])\s*=\s*(\d+)", src)}
    from paper_2002_00352_gb300 import kp
    got = kp.kp_limits()
    assert (got["max_m"], got["max_l"], got["max_k"]) == (want["KP_MAX_M"], want["KP_MAX_L"], want["KP_MAX_K"])
