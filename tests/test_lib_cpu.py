"""CPU checks of the C-ABI library: it builds, loads, and exports every symbol that
include/gbs_mpo.h declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gbs_mpo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpo_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_12814_gb300 import build
    path = build.build()
    from paper_2301_12814_gb300 import mpo
    return mpo.load_library(path)


def test_header_and_binding_agree():
    from paper_2301_12814_gb300 import mpo
    assert _declared() == sorted(mpo.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(10):
        assert lib.mpo_status_string(s)


def test_host_argument_checks(lib):
    from paper_2301_12814_gb300 import mpo
    h = ctypes.c_void_p()
    r = np.zeros(4); eta = np.ones(4)
    # null params
    assert lib.mpo_init_lossy_squeezed(ctypes.byref(h), None, mpo._d(r), mpo._d(eta)) == 1
    bad = [dict(M=1), dict(d=1), dict(n_cap=9), dict(batch=0), dict(prec=7)]
    for kw in bad:
        base = dict(M=4, d=4, n_cap=0, batch=1, prec=0)
        base.update(kw)
        prm = mpo._Params(M=base["M"], d=base["d"], n_cap=base["n_cap"], batch=base["batch"],
                          prec=base["prec"], chi_max=None, cuda_stream=None)
        assert lib.mpo_init_lossy_squeezed(ctypes.byref(h), ctypes.byref(prm), mpo._d(r),
                                           mpo._d(eta)) == 1, kw
    # out-of-range physics parameters
    prm = mpo._Params(M=4, d=4, n_cap=0, batch=1, prec=0, chi_max=None, cuda_stream=None)
    assert lib.mpo_init_lossy_squeezed(ctypes.byref(h), ctypes.byref(prm), mpo._d(np.full(4, -1.0)),
                                       mpo._d(eta)) == 1
    assert lib.mpo_init_lossy_squeezed(ctypes.byref(h), ctypes.byref(prm), mpo._d(r),
                                       mpo._d(np.full(4, 1.5))) == 1
    # null handles
    assert lib.mpo_apply_bs(None, 0, 0, 0.1, 0.2, None) == 1
    assert lib.mpo_sync(None) == 1
    assert lib.mpo_bond_capacity(None) == 0


def test_no_gpu_is_reported_not_faked(lib):
    """Without a GPU the library refuses (MPO_ERR_NOT_BUILT) instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2301_12814_gb300 import MPO, MPOError
    with pytest.raises(MPOError) as ei:
        MPO(4, 4, [0.5] * 4, [0.5] * 4)
    assert ei.value.status == 9
    from paper_2301_12814_gb300 import mpo
    with pytest.raises(MPOError) as ei:
        mpo.asymptotic_ee([0.88], [0.3], [0.7853981633974483], 8)
    assert ei.value.status == 9


def test_asymptotic_argument_checks(lib):
    """mpo_asymptotic_ee validates sizes and ranges on the host before any CUDA call."""
    from paper_2301_12814_gb300 import mpo
    one = np.array([0.5]); K = 81
    out = np.zeros(1); sp = np.zeros(K)
    call = lambda n, r, mu, th, alpha=0.0, Sa=None, ld=K: lib.mpo_asymptotic_ee(
        1, n, mpo._d(r), mpo._d(mu), mpo._d(th), alpha, mpo._d(out), mpo._d(Sa), mpo._d(sp), ld)
    assert call(0, one, one, one) == 1
    assert call(24, one, one, one) == 1
    assert call(8, np.array([3.5]), one, one) == 1
    assert call(8, one, np.array([1.01]), one) == 1
    assert call(8, one, one, np.array([np.inf])) == 1
    assert call(8, one, one, one, alpha=0.0, Sa=np.zeros(1)) == 1
    assert call(8, one, one, one, ld=80) == 1
    assert lib.mpo_asymptotic_ee(0, 8, None, None, None, 0.0, None, None, None, 0) == 0
    assert lib.mpo_asymptotic_ee_device(1, 8, None, None, None, 0.0, None, None, None, K, None, None) == 1


def test_checkpoint_argument_checks(lib):
    import ctypes as ct
    n = ct.c_size_t()
    assert lib.mpo_checkpoint_bytes(None, ct.byref(n)) == 1
    assert lib.mpo_save(None, None, 0, 0) == 1
    assert lib.mpo_load(None, None, 0, None) == 1


def test_allocator_argument_checks(lib):
    from paper_2301_12814_gb300 import mpo
    a = mpo._ALLOC_FN(lambda n, st, ctx: None)
    f = mpo._FREE_FN(lambda p, st, ctx: None)
    assert lib.mpo_set_allocator(a, mpo._FREE_FN(), None) == 1
    assert lib.mpo_set_allocator(mpo._ALLOC_FN(), f, None) == 1
    assert lib.mpo_set_allocator(a, f, None) == 0
    assert lib.mpo_set_allocator(mpo._ALLOC_FN(), mpo._FREE_FN(), None) == 0
