"""The norm-fold slot schedule of the low passes (host logic, no GPU).

fold_for (paper_1103_1399_gb300/csrc/qaa_internal.cuh) decides, for every low
pass, which per-CTA partial-sum slots it reads and writes.  The exact
evolution is unitary (Eq. (1) is Hermitian), so the fold only removes FP32
rounding drift; a wrong schedule would read a slot while another CTA of the
same launch writes it, or correct with a stale or missing measurement.
tests/fold_slots_check.cpp compiles the header with the host compiler and
checks every period and run length, with the step numbering of per-pass
launches and of launch graphs (see its header).
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_fold_slot_schedule(tmp_path):
    gxx = shutil.which("g++")
    inc = cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "fold_slots_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1103_1399_gb300", "csrc"), "-I", inc,
                    os.path.join(ROOT, "tests", "fold_slots_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
