"""The observables kernel's clamps keep every access in bounds on corrupted tables.

mpo_observables_static runs k_obs on bond tables (chi, charge, segoff) held in the
caller's device buffers.  k_obs clamps every size and index it reads from them with
the helpers of csrc/mpo_internal.cuh.  tests/c_abi/obs_clamp_walk.cpp includes those
helpers, walks the kernel's loops over random tables with out-of-range values and
checks every buffer index; here it is built with the host compiler and run.  No GPU
is involved: bad inputs are never sent to a device.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = "/usr/local/cuda/include"


def test_obs_clamps_keep_accesses_in_bounds(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ and the CUDA headers are needed to build the walker")
    exe = str(tmp_path / "obs_clamp_walk")
    src = os.path.join(HERE, "c_abi", "obs_clamp_walk.cpp")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CUDA_INC,
                    "-I", os.path.join(ROOT, "paper_2301_12814_gb300", "csrc"), src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert " 0 out of bounds" in out.stdout
