"""The App. C asymptotic estimator on the GPU (mpo_asymptotic_ee) against the oracle
(oracle/asymptotic.py) on the same points: the whole normalised spectrum element by
element, S_1 and Renyi entropies, across photon cutoffs from 1 to the largest the
kernel takes, the Fig. 1 protocol, the device entry point, and argument errors.

Tolerances (FP64 on both sides): the kernel's one-sided Jacobi gives every squared
singular value to a few ulps of the largest, LAPACK's SVD likewise, so a normalised
eigenvalue differs by at most ~(n_max+1)^2 * 1e-16 < 1e-13; the entropies are sums of
p log p over at most 576 values, bounded by 1e-11 absolute plus 1e-10 relative."""
import math

import numpy as np
import pytest

from oracle import asymptotic as asy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    return mpo


def _points(seed, n):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, 1.5, n)
    mu = rng.uniform(0.0, 1.0, n)
    th = rng.uniform(0.0, math.pi / 2, n)
    # special cases: vacuum input, no loss, full loss, no split, the asymptotic angle
    r[:5] = [0.0, 0.88, 0.88, 0.88, 0.88]
    mu[:5] = [0.5, 1.0, 0.0, 0.5, 0.3]
    th[:5] = [math.pi / 4, 0.3, math.pi / 4, 0.0, math.pi / 4]
    return r, mu, th


@pytest.mark.parametrize("n_max", [1, 2, 5, 8, 12])
def test_spectrum_and_entropies_match_oracle(lib, n_max):
    r, mu, th = _points(n_max, 24)
    K = (n_max + 1) ** 2
    g = lib.asymptotic_ee(r, mu, th, n_max, alpha=2.0, spectrum=True)
    g_half = lib.asymptotic_ee(r, mu, th, n_max, alpha=0.5)
    for i in range(r.size):
        p = asy.mode_spectrum(r[i], mu[i], n_max, th[i])
        assert g["spectrum"][i].shape == (K,)
        assert np.max(np.abs(g["spectrum"][i] - p)) < 1e-13, (i, r[i], mu[i], th[i])
        for got, alpha in ((g["S1"][i], None), (g["S_alpha"][i], 2.0), (g_half["S_alpha"][i], 0.5)):
            want = asy.entropy(p, alpha)
            assert abs(got - want) <= 1e-11 + 1e-10 * abs(want), (i, alpha, got, want)
    assert np.array_equal(g["S1"], g_half["S1"])


def test_largest_cutoff(lib):
    n_max = lib.ASYM_NMAX
    r = np.array([0.88, 0.4]); mu = np.array([0.3, 1.0]); th = np.array([math.pi / 4, 0.3])
    g = lib.asymptotic_ee(r, mu, th, n_max, spectrum=True)
    for i in range(2):
        p = asy.mode_spectrum(r[i], mu[i], n_max, th[i])
        assert np.max(np.abs(g["spectrum"][i] - p)) < 1e-13
        assert abs(g["S1"][i] - asy.entropy(p)) <= 1e-11 + 1e-10 * asy.entropy(p)


def test_fig1_protocol_vs_oracle(lib):
    from paper_2301_12814_gb300 import experiments as ex
    Ns = np.array([10, 40, 160, 640, 2560])
    for gamma in (0.25, 0.5, 1.0):
        beta = 0.5 if gamma == 1.0 else 1.0
        got = ex.asymptotic_ee(Ns, beta, gamma, r=0.88, n_max=8)["S1"]
        want = [asy.system_entropy(int(N), beta, gamma, 0.88, 8) for N in Ns]
        assert np.allclose(got, want, rtol=1e-10, atol=1e-10)
    conv = ex.n_max_convergence(N=50, n_maxes=(4, 6, 8))
    for n, v in conv:
        assert abs(v - asy.system_entropy(50, 1.0, 0.5, 0.88, n)) <= 1e-9 * v


def test_device_entry_equals_host(lib):
    import torch
    n_max = 8
    r, mu, th = _points(3, 40)
    K = (n_max + 1) ** 2
    dev = torch.device("cuda:0")
    tr, tm, tt = (torch.tensor(x, dtype=torch.float64, device=dev) for x in (r, mu, th))
    S1 = torch.empty(40, dtype=torch.float64, device=dev)
    Sa = torch.empty(40, dtype=torch.float64, device=dev)
    sp = torch.empty(40 * K, dtype=torch.float64, device=dev)
    sw = torch.zeros(160, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    lib.asymptotic_ee_device(tr, tm, tt, n_max, S1, sp, alpha=2.0, S_alpha=Sa, sweeps=sw, stream=stream)
    torch.cuda.synchronize()
    h = lib.asymptotic_ee(r, mu, th, n_max, alpha=2.0, spectrum=True)
    assert np.array_equal(S1.cpu().numpy(), h["S1"])
    assert np.array_equal(Sa.cpu().numpy(), h["S_alpha"])
    assert np.array_equal(sp.cpu().numpy().reshape(40, K), h["spectrum"])
    s = sw.cpu().numpy()
    assert s.min() >= 1 and s.max() <= 40


def test_argument_errors(lib):
    one = np.array([0.5])
    for n_max in (0, lib.ASYM_NMAX + 1):
        with pytest.raises(lib.MPOError):
            lib.asymptotic_ee(one, one, one, n_max)
    with pytest.raises(lib.MPOError):
        lib.asymptotic_ee(one, np.array([1.5]), one, 8)
    with pytest.raises(lib.MPOError):
        lib.asymptotic_ee(np.array([-0.1]), one, one, 8)
    with pytest.raises(lib.MPOError):
        lib.asymptotic_ee(one, one, one, 8, alpha=-1.0)
    g = lib.asymptotic_ee(np.zeros(0), np.zeros(0), np.zeros(0), 8)
    assert g["S1"].size == 0
