"""The C-ABI library builds, loads and exports every entry point that
include/hqn.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hqn.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sim_create", "sim_step", "sim_energy_grad", "sim_solve_A0", "sim_direction",
              "sim_set_state", "sim_get_state", "sim_get_info", "sim_destroy", "sim_strerror"):
        assert n in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs the CUDA toolkit to build")
def test_library_exports_every_declared_symbol():
    from paper_1604_07378_gb300 import build
    lib = ctypes.CDLL(build.build_library())
    for n in _declared():
        assert hasattr(lib, n), n
    # host-only entry points work without a device
    from paper_1604_07378_gb300 import hqn
    p = hqn.default_params()
    assert abs(p.h - 1.0 / 30.0) < 1e-15 and p.iters == 10 and p.history_m == 5
    assert abs(p.gamma - 0.3) < 1e-15 and abs(p.backtrack - 0.5) < 1e-15
    assert hqn.library().sim_strerror(hqn.HQN_ERR_NOT_SPD) == b"A0 is not positive definite"
