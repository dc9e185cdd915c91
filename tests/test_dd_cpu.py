"""Accuracy of the double-float arithmetic (csrc/dd.cuh) that the FP64 path's block
refinement runs in: tests/c_abi/dd_check.cpp includes the header, compares sums,
products, complex products and 512-term compensated dot products (32 lanes x 16 terms,
combined pairwise) with long double on random inputs, some near cancellation, and
fails if an error exceeds a small multiple of u^2 = 2^-48 (relative to the operands'
magnitudes); tests/c_abi/dd_rot_check.cpp does the same for the one-sided Jacobi
rotation of a complex double-float column pair (parameters on the FP32 pipe, both
rotation forms, carried norms), and tests/c_abi/dd_ns_check.cpp for the two
Newton-Schulz steps that orthonormalise the FP32 seed.  Built here with the host
compiler, FMA contraction off."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_double_float_arithmetic_accuracy(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is needed to build the check")
    exe = str(tmp_path / "dd_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_2301_12814_gb300", "csrc"),
                    os.path.join(HERE, "c_abi", "dd_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout


def _build_and_run(tmp_path, name):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is needed to build the check")
    exe = str(tmp_path / name)
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_2301_12814_gb300", "csrc"),
                    os.path.join(HERE, "c_abi", name + ".cpp"), "-o", exe], check=True)
    return subprocess.run([exe], capture_output=True, text=True)


def test_double_float_jacobi_rotation(tmp_path):
    """c^2 + s^2 = 1 and |e| = 1 to a few u^2, the pair's inner product annihilated up
    to the FP32-rounded angle (1e-6 relative), the pair's total norm kept, and the
    carried norms equal to the rotated columns' norms, for large and small angles."""
    out = _build_and_run(tmp_path, "dd_rot_check")
    assert out.returncode == 0, out.stdout


def test_double_float_newton_schulz(tmp_path):
    """Two Newton-Schulz steps (S in double-float, the correction product in FP32) take
    an FP32 seed with 1e-6 non-orthogonality to |V^dag V - I| <= 5e-14, within 1e-11 of
    the same steps in long double."""
    out = _build_and_run(tmp_path, "dd_ns_check")
    assert out.returncode == 0, out.stdout

