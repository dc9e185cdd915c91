"""The large-block SVD on a thread-block cluster, exercised on every block.

By default a block goes to a cluster only when it would be its layer's critical
path, which the small parity workloads reach for a few blocks at most.  Here a child
process routes every block with a Gram side >= 1 through it
(GBS_MPO_SVD_CLUSTER_MIN_N=1): many ragged column blocks, empty blocks, self-mirror
blocks in the mirror-real basis.  The results must meet
the same bars as the single-CTA path against the FP64 oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", params=["gram_seed", "fp32_phase"])
def results(request):
    """Every block on a cluster; cluster blocks of Gram side <= 64 seeded by the
    single-CTA Gram eigensolver (GBS_MPO_SVD_CLUSTER_SEED_MAX=64, the FP32 path's
    default), or all of them by the FP32 cluster phase (=0, the FP64 path's default)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, GBS_MPO_SVD_CLUSTER_MIN_N="1")
    env["GBS_MPO_SVD_CLUSTER_SEED_MAX"] = "0" if request.param == "fp32_phase" else "64"
    out = subprocess.run([sys.executable, os.path.join(HERE, "cluster_route_check.py")], env=env,
                         capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("case", ["exact_fp64", "chi64_fp64", "chi256_fp64_prefix"])
def test_cluster_path_fp64_vs_oracle(results, case):
    r = results[case]
    assert r["chi_equal"], r
    assert r["bitwise_replay"], r
    assert r["tr"] <= 1e-10 and r["n1"] <= 1e-10 and r["n2"] <= 1e-10, r
    # per-gate discarded weights: 1e-10 relative to the largest, absolute floor 1e-12
    # (an untruncated gate's weight is a difference of two sums, zero up to rounding)
    assert r["S"] <= 1e-10 and r["disc_abs"] <= 1e-12 + 1e-10 * r["disc_max"], r


def test_cluster_path_mixed_vs_oracle(results):
    r = results["chi64_mixed"]
    assert r["bitwise_replay"], r
    assert r["n1"] <= 1e-4 and r["n2"] <= 1e-4 and r["S"] <= 1e-3 and r["tr"] <= 1e-4, r
    assert r["disc_abs"] <= 1e-12 + 1e-2 * r["disc_max"], r
