"""The C ABI used from plain C (tests/c_abi/mesh_demo.c, built with gcc against
include/gbs_mpo.h and libgbsmpo.so): it compiles and links on any machine; on a GPU
it runs a truncated mesh, a checkpoint round trip and one App. C estimate, and prints
the same numbers the Python binding computes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "mesh_demo.c")


def _compile(tmp_path):
    from paper_2301_12814_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "mesh_demo")
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
           "-L", libdir, "-lgbsmpo", f"-Wl,-rpath,{libdir}"]
    # the library is named libgbsmpo.so in the package directory
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_consumer_compiles_and_links(tmp_path):
    exe = _compile(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_consumer_matches_python(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import gbs_workloads as w
    from paper_2301_12814_gb300 import mpo
    exe = _compile(tmp_path)
    M, d, chi, r, eta = 8, 5, 16, 0.8, 0.4
    m = w.dialled_mesh(M, 2)
    lines = [f"{M} {d} {chi} {r!r} {eta!r} {m.n_gates}"]
    lines += [f"{int(k)} {float(t)!r} {float(p)!r}" for k, t, p in zip(m.k, m.theta, m.phi)]
    lines.append(" ".join(repr(float(x)) for x in m.final_phase))
    mesh_file = tmp_path / "mesh.txt"
    mesh_file.write_text("\n".join(lines) + "\n")
    out = subprocess.run([exe, str(mesh_file)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        parts = line.split()
        got[" ".join(p for p in parts if not _isnum(p))] = [float(p) for p in parts if _isnum(p)]
    G = mpo.MPO(M, d, [r] * M, [eta] * M, chi_max=chi)
    disc = G.sweep_mesh([m.n_gates], m.k, m.theta, m.phi, m.final_phase)
    tr, n1, _ = G.observables()
    _, _, smax = G.operator_entropy()
    G.close()
    assert got["trace"][0] == tr[0]
    assert np.array_equal(np.array(got["n_mean"]), n1[0])
    assert got["S_max"][0] == smax[0]
    dsum = 0.0
    for x in disc:  # the C program adds in gate order
        dsum += float(x)
    assert got["discarded_sum"][0] == dsum
    assert got["checkpoint cursor trace"] == [m.n_gates, tr[0]]
    a = mpo.asymptotic_ee([0.88], [0.3], [0.78539816339744831], 8)["S1"][0]
    assert got["asymptotic_S1"][0] == a


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False
