"""Python binding of libgbsmpo.so (argument marshalling only; every step runs in CUDA).

Names follow the C ABI of include/gbs_mpo.h.  The library is loaded from this
package directory; if it is missing or cannot be loaded the binding raises
instead of falling back to anything else.

* ``MPO``: a handle (mpo_init_lossy_squeezed) with gates (apply_bs, sweep_mesh,
  plan_mesh), observables, entropies, bonds, the truncated probability, checkpoints
  (save / load) and reset.
* ``Plan``: a mesh captured in a CUDA graph, with per-stage times and an instrumented
  profile.
* ``asymptotic_ee`` / ``asymptotic_ee_device``: the App. C estimator.
* ``set_allocator`` / ``use_torch_allocator``: device memory of later handles from a
  caller's allocator (mpo_set_allocator).
* ``svd_cluster_shape``: the block SVD's launch shape on this GPU.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgbsmpo.so")

MPO_FP64, MPO_MIXED_TF32, MPO_MIXED_BF16 = 0, 1, 2
PRECISIONS = {"fp64": MPO_FP64, "mixed_tf32": MPO_MIXED_TF32, "mixed_bf16": MPO_MIXED_BF16}

# every symbol declared in include/gbs_mpo.h
EXPORTS = [
    "mpo_init_lossy_squeezed", "mpo_reset", "mpo_apply_bs", "mpo_sweep_mesh", "mpo_plan_mesh",
    "mpo_plan_run", "mpo_plan_discarded", "mpo_plan_launches", "mpo_plan_profile", "mpo_plan_stage_times",
    "mpo_plan_destroy",
    "mpo_observables", "mpo_truncated_probability", "mpo_operator_entropy", "mpo_get_bonds", "mpo_bond_capacity",
    "mpo_sync", "mpo_destroy", "mpo_status_string", "mpo_observables_static", "mpo_svd_cluster_shape",
    "mpo_asymptotic_ee", "mpo_asymptotic_ee_device", "mpo_checkpoint_bytes", "mpo_save", "mpo_load",
    "mpo_set_allocator", "mpo_measure_peaks", "mpo_set_tuning", "mpo_get_tuning",
]
ASYM_NMAX = 23  # MPO_ASYM_NMAX


class MPOError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().mpo_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class Tuning(ctypes.Structure):
    """Launch choices of a handle (mpo_tuning in include/gbs_mpo.h)."""
    _fields_ = [("theta_form", ctypes.c_int), ("gram_tc_min", ctypes.c_int), ("svd_cluster_size", ctypes.c_int),
                ("svd_cluster_min_n", ctypes.c_int), ("svd_cluster_seed_max", ctypes.c_int)]
    NAMES = ("theta_form", "gram_tc_min", "svd_cluster_size", "svd_cluster_min_n", "svd_cluster_seed_max")

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k in self.NAMES}


class _Params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("d", ctypes.c_int), ("n_cap", ctypes.c_int),
                ("batch", ctypes.c_int), ("prec", ctypes.c_int),
                ("chi_max", ctypes.POINTER(ctypes.c_int)), ("cuda_stream", ctypes.c_void_p)]


_LIB = None
_i = ctypes.c_int
_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libgbsmpo.so and declare its signatures.  Raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgbsmpo.so not built at {path}: call __graft_entry__.build() "
                           "or python -m paper_2301_12814_gb300.build")
    lib = ctypes.CDLL(path)
    sig = {
        "mpo_init_lossy_squeezed": (_i, [ctypes.POINTER(_p), ctypes.POINTER(_Params), _dp, _dp]),
        "mpo_reset": (_i, [_p]),
        "mpo_apply_bs": (_i, [_p, _i, _i, ctypes.c_double, ctypes.c_double, _dp]),
        "mpo_sweep_mesh": (_i, [_p, _ip, _ip, _dp, _dp, _dp, _dp]),
        "mpo_plan_mesh": (_i, [_p, _ip, _ip, _dp, _dp, _dp, ctypes.POINTER(_p)]),
        "mpo_plan_run": (_i, [_p]),
        "mpo_plan_discarded": (_i, [_p, _dp]),
        "mpo_plan_launches": (_i, [_p]),
        "mpo_plan_profile": (_i, [_p, _dp, _ip, _dp, _dp]),
        "mpo_plan_stage_times": (_i, [_p, _dp]),
        "mpo_svd_cluster_shape": (_i, [_ip, _ip, _ip, _ip]),
        "mpo_checkpoint_bytes": (_i, [_p, ctypes.POINTER(ctypes.c_size_t)]),
        "mpo_set_allocator": (_i, [_ALLOC_FN, _FREE_FN, _p]),
        "mpo_save": (_i, [_p, _p, ctypes.c_size_t, ctypes.c_longlong]),
        "mpo_load": (_i, [_p, _p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_longlong)]),
        "mpo_asymptotic_ee": (_i, [_i, _i, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _i]),
        "mpo_asymptotic_ee_device": (_i, [_i, _i, _p, _p, _p, ctypes.c_double, _p, _p, _p, _i, _p, _p]),
        "mpo_plan_destroy": (None, [_p]),
        "mpo_observables": (_i, [_p, _dp, _dp, _dp, _i]),
        "mpo_truncated_probability": (_i, [_p, _dp]),
        "mpo_operator_entropy": (_i, [_p, _dp, _dp, _dp]),
        "mpo_get_bonds": (_i, [_p, _i, _i, _ip, _dp, _ip]),
        "mpo_bond_capacity": (_i, [_p]),
        "mpo_sync": (_i, [_p]),
        "mpo_destroy": (None, [_p]),
        "mpo_status_string": (ctypes.c_char_p, [_i]),
        "mpo_observables_static": (_i, [_i, _i, _i, _p, _p, _p, _p, _p, _p, _p]),
        "mpo_measure_peaks": (_i, [_dp, _dp]),
        "mpo_set_tuning": (_i, [_p, ctypes.POINTER(Tuning)]),
        "mpo_get_tuning": (_i, [_p, ctypes.POINTER(Tuning)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _lib() -> ctypes.CDLL:
    return load_library()


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_ALLOCATOR_REFS = []  # keeps the installed ctypes callbacks alive


def set_allocator(alloc=None, free=None) -> None:
    """Install a device allocator for handles created afterwards (mpo_set_allocator):
    ``alloc(bytes, stream) -> int`` and ``free(ptr, stream)``, stream being the raw
    cudaStream_t as an int; None, None restores the CUDA runtime."""
    if alloc is None and free is None:
        _check(_lib().mpo_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "mpo_set_allocator")
        return
    a = _ALLOC_FN(lambda n, st, ctx: int(alloc(int(n), int(st or 0))) or None)
    f = _FREE_FN(lambda ptr, st, ctx: free(int(ptr), int(st or 0)))
    _ALLOCATOR_REFS.append((a, f))
    _check(_lib().mpo_set_allocator(a, f, None), "mpo_set_allocator")


def use_torch_allocator() -> None:
    """Route handle memory through PyTorch's CUDA caching allocator on each handle's
    stream (torch.cuda.caching_allocator_alloc / caching_allocator_delete)."""
    import torch
    dev = torch.cuda.current_device()
    set_allocator(lambda n, st: torch.cuda.caching_allocator_alloc(n, device=dev, stream=st),
                  lambda ptr, st: torch.cuda.caching_allocator_delete(ptr))


def _d(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_dp)


def _ip_of(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_ip)


def _check(st: int, where: str) -> None:
    if st != 0:
        raise MPOError(st, where)


def measure_peaks() -> dict:
    """Measured peaks of the current GPU in TFLOP/s (mpo_measure_peaks): FP64 and FP32
    FMA chains, TF32 and BF16 tcgen05 MMA on shared-memory operands."""
    t = np.zeros(4)
    ms = np.zeros(4)
    _check(_lib().mpo_measure_peaks(_d(t), _d(ms)), "mpo_measure_peaks")
    return {"fp64": float(t[0]), "fp32": float(t[1]), "tf32": float(t[2]), "bf16": float(t[3]),
            "ms": [float(x) for x in ms]}


def svd_cluster_shape() -> dict:
    """Launch shape of the block SVD on this GPU (mpo_svd_cluster_shape)."""
    v = np.zeros(4, dtype=np.int32)
    _check(_lib().mpo_svd_cluster_shape(*[v[i:].ctypes.data_as(_ip) for i in range(4)]), "mpo_svd_cluster_shape")
    return {"cluster_size": int(v[0]), "clusters_fp64": int(v[1]), "clusters_fp32": int(v[2]), "min_n": int(v[3])}


def asymptotic_ee(r, mu, theta, n_max: int, alpha: Optional[float] = None, spectrum: bool = False) -> dict:
    """App. C estimator for a batch of points (mpo_asymptotic_ee): one squeezed mode of
    squeezing r, transmission mu, split angle theta, cut at n_max photons.  Returns
    ``{"S1": [npts], "S_alpha": [npts] or None, "spectrum": [npts, (n_max+1)^2] or None}``."""
    r, mu, theta = (np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64))) for x in (r, mu, theta))
    r, mu, theta = (np.ascontiguousarray(x) for x in np.broadcast_arrays(r, mu, theta))
    n = r.size
    K = (int(n_max) + 1) ** 2
    S1 = np.zeros(n)
    Sa = np.zeros(n) if alpha is not None else None
    sp = np.zeros((n, K)) if spectrum else None
    _check(_lib().mpo_asymptotic_ee(n, int(n_max), _d(r), _d(mu), _d(theta),
                                    float(alpha) if alpha is not None else 0.0, _d(S1), _d(Sa), _d(sp), K),
           "mpo_asymptotic_ee")
    return {"S1": S1, "S_alpha": Sa, "spectrum": sp}


def asymptotic_ee_device(r, mu, theta, n_max: int, S1, spectrum, alpha: Optional[float] = None, S_alpha=None,
                         sweeps=None, stream=None) -> None:
    """mpo_asymptotic_ee_device on caller-owned device buffers (objects exposing
    ``data_ptr()``, e.g. torch CUDA tensors of float64; ``sweeps`` int32).  Asynchronous
    on ``stream`` (an object with ``cuda_stream`` or a raw handle; None = default)."""
    n = int(r.numel())
    K = (int(n_max) + 1) ** 2
    ptr = (lambda t: None if t is None else t.data_ptr())
    sp = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib().mpo_asymptotic_ee_device(n, int(n_max), ptr(r), ptr(mu), ptr(theta),
                                           float(alpha) if alpha is not None else 0.0, ptr(S1), ptr(S_alpha),
                                           ptr(spectrum), K, ptr(sweeps), sp), "mpo_asymptotic_ee_device")


class Plan:
    """A mesh uploaded once and captured in a CUDA graph (mpo_plan_*)."""

    def __init__(self, owner: "MPO", n_gates, k, theta, phi, final_phase):
        self._owner = owner
        self.n_total = int(np.sum(n_gates))
        h = _p()
        _check(_lib().mpo_plan_mesh(owner._h, _ip_of(n_gates), _ip_of(k), _d(theta), _d(phi),
                                    _d(final_phase), ctypes.byref(h)), "mpo_plan_mesh")
        self._h = h
        owner._plans.add(self)
        self.launches = int(_lib().mpo_plan_launches(h))

    def run(self) -> None:
        _check(_lib().mpo_plan_run(self._h), "mpo_plan_run")

    def discarded(self) -> np.ndarray:
        out = np.zeros(max(self.n_total, 1))
        _check(_lib().mpo_plan_discarded(self._h, _d(out)), "mpo_plan_discarded")
        return out[:self.n_total]

    STAGES = ("setup", "theta", "gram", "order", "svd", "select", "resplit", "phases")

    def profile(self, with_jacobi: bool = False):
        """One instrumented replay: {stage: (ms, launches, flops)} (and, if asked,
        {blocks, two-sided sweeps, one-sided sweeps})."""
        ms = np.zeros(8); nl = np.zeros(8, dtype=np.int32); fl = np.zeros(8); jb = np.zeros(14)
        _check(_lib().mpo_plan_profile(self._h, _d(ms), _ip_of(nl), _d(fl), _d(jb)), "mpo_plan_profile")
        out = {s: (float(ms[i]), int(nl[i]), float(fl[i])) for i, s in enumerate(self.STAGES)}
        if with_jacobi:
            return out, {"blocks": int(jb[0]), "sweeps": int(jb[1]), "refine_sweeps": int(jb[2]),
                         "seed_flops": float(jb[3]), "refine_flops": float(jb[4]), "cluster_blocks": int(jb[5]),
                         "cluster_cycles": float(jb[6]), "cta_cycles": float(jb[7]),
                         "cluster_seed_cycles": float(jb[8]), "cluster_ns_cycles": float(jb[9]),
                         "cluster_polish_cycles": float(jb[10]), "warp_blocks": int(jb[11]),
                         "warp_cycles": float(jb[12]), "theta_F_flops": float(jb[13])}
        return out

    def stage_times(self) -> dict:
        """{stage: ms} of the most recent run(), from the events inside the graph."""
        ms = np.zeros(8)
        _check(_lib().mpo_plan_stage_times(self._h, _d(ms)), "mpo_plan_stage_times")
        return {s: float(ms[i]) for i, s in enumerate(self.STAGES)}

    def close(self) -> None:
        # the owning handle frees its plans itself when it is destroyed first
        if getattr(self, "_h", None) and getattr(self._owner, "_h", None):
            _lib().mpo_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPO:
    """A batch of lossy-GBS U(1) MPOs on the GPU (mpo_init_lossy_squeezed and friends)."""

    def __init__(self, M: int, d: int, r, eta, chi_max=None, batch: int = 1,
                 n_cap: Optional[int] = None, precision: str = "fp64", stream=None):
        lib = _lib()
        self.M, self.d, self.batch = int(M), int(d), int(batch)
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(r, dtype=np.float64), (batch, M)))
        eta = np.ascontiguousarray(np.broadcast_to(np.asarray(eta, dtype=np.float64), (batch, M)))
        if chi_max is None:
            chis = np.zeros(batch, dtype=np.int32)
        else:
            chis = np.ascontiguousarray(np.broadcast_to(
                np.asarray([0 if c is None else c for c in np.atleast_1d(chi_max)], dtype=np.int32),
                (batch,)))
        self._chis = chis
        sp = None
        if stream is not None:
            sp = int(getattr(stream, "cuda_stream", stream))
        prm = _Params(M=self.M, d=self.d, n_cap=0 if n_cap is None else int(n_cap), batch=self.batch,
                      prec=PRECISIONS[precision], chi_max=_ip_of(chis), cuda_stream=sp)
        self._plans = weakref.WeakSet()
        h = _p()
        _check(lib.mpo_init_lossy_squeezed(ctypes.byref(h), ctypes.byref(prm), _d(r), _d(eta)),
               "mpo_init_lossy_squeezed")
        self._h = h
        self.D = int(lib.mpo_bond_capacity(h))

    # --------------------------------------------------------------- updates
    def reset(self) -> None:
        _check(_lib().mpo_reset(self._h), "mpo_reset")

    def apply_bs(self, k: int, theta: float, phi: float, inst: int = 0,
                 want_discarded: bool = True) -> Optional[float]:
        out = np.zeros(1)
        _check(_lib().mpo_apply_bs(self._h, int(inst), int(k), float(theta), float(phi),
                                   _d(out) if want_discarded else None), "mpo_apply_bs")
        return float(out[0]) if want_discarded else None

    @staticmethod
    def _mesh_arrays(n_gates, k, theta, phi, final_phase):
        n_gates = np.ascontiguousarray(np.atleast_1d(n_gates), dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        fp = None if final_phase is None else np.ascontiguousarray(final_phase, dtype=np.float64)
        return n_gates, k, theta, phi, fp

    def sweep_mesh(self, n_gates, k, theta, phi, final_phase=None) -> np.ndarray:
        n_gates, k, theta, phi, fp = self._mesh_arrays(n_gates, k, theta, phi, final_phase)
        out = np.zeros(max(int(n_gates.sum()), 1))
        _check(_lib().mpo_sweep_mesh(self._h, _ip_of(n_gates), _ip_of(k), _d(theta), _d(phi),
                                     _d(fp), _d(out)), "mpo_sweep_mesh")
        return out[:int(n_gates.sum())]

    def set_tuning(self, **kw) -> dict:
        """Change launch choices (mpo_set_tuning): theta_form, gram_tc_min,
        svd_cluster_size, svd_cluster_min_n, svd_cluster_seed_max; unnamed ones keep
        their current values.  Plans made afterwards use them.  Returns the new set."""
        t = Tuning()
        _check(_lib().mpo_get_tuning(self._h, ctypes.byref(t)), "mpo_get_tuning")
        for key, v in kw.items():
            if key not in Tuning.NAMES:
                raise KeyError(key)
            setattr(t, key, int(v))
        _check(_lib().mpo_set_tuning(self._h, ctypes.byref(t)), "mpo_set_tuning")
        return t.as_dict()

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(_lib().mpo_get_tuning(self._h, ctypes.byref(t)), "mpo_get_tuning")
        return t.as_dict()

    def plan_mesh(self, n_gates, k, theta, phi, final_phase=None) -> Plan:
        n_gates, k, theta, phi, fp = self._mesh_arrays(n_gates, k, theta, phi, final_phase)
        return Plan(self, n_gates, k, theta, phi, fp)

    # ----------------------------------------------------------- observables
    def observables(self, normalize: bool = True):
        B, M = self.batch, self.M
        tr = np.zeros(B); n1 = np.zeros(B * M); n2 = np.zeros(B * M)
        _check(_lib().mpo_observables(self._h, _d(tr), _d(n1), _d(n2), 1 if normalize else 0),
               "mpo_observables")
        return tr, n1.reshape(B, M), n2.reshape(B, M)

    def save(self, cursor: int = 0) -> np.ndarray:
        """Checkpoint of the current state (mpo_save) as a uint8 array; ``cursor`` is
        stored with it (for example the number of gates applied so far)."""
        n = ctypes.c_size_t()
        _check(_lib().mpo_checkpoint_bytes(self._h, ctypes.byref(n)), "mpo_checkpoint_bytes")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(_lib().mpo_save(self._h, buf.ctypes.data_as(_p), n.value, int(cursor)), "mpo_save")
        return buf

    def load(self, buf) -> int:
        """Replace the state by a checkpoint from ``save`` (mpo_load); returns its cursor."""
        buf = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray))
                                   else buf, dtype=np.uint8)
        cur = ctypes.c_longlong()
        _check(_lib().mpo_load(self._h, buf.ctypes.data_as(_p), buf.size, ctypes.byref(cur)), "mpo_load")
        return int(cur.value)

    def truncated_probability(self) -> np.ndarray:
        """[batch] probability cut from the initial state by the local dimension d and
        the photon-number cap (mpo_truncated_probability)."""
        tail = np.zeros(self.batch)
        _check(_lib().mpo_truncated_probability(self._h, _d(tail)), "mpo_truncated_probability")
        return tail

    def operator_entropy(self):
        B, M = self.batch, self.M
        S = np.zeros(B * (M + 1)); pur = np.zeros(B * (M + 1)); smax = np.zeros(B)
        _check(_lib().mpo_operator_entropy(self._h, _d(S), _d(pur), _d(smax)), "mpo_operator_entropy")
        return S.reshape(B, M + 1), pur.reshape(B, M + 1), smax

    def bonds(self, inst: int = 0):
        """(chi[M+1], [lambda_b], [charges_b (chi_b x 2)]) of one instance."""
        M, ld = self.M, self.D
        chi = np.zeros(M + 1, dtype=np.int32)
        lam = np.zeros((M + 1) * ld)
        ch = np.zeros((M + 1) * ld * 2, dtype=np.int32)
        _check(_lib().mpo_get_bonds(self._h, int(inst), ld, _ip_of(chi), _d(lam), _ip_of(ch)),
               "mpo_get_bonds")
        lam = lam.reshape(M + 1, ld)
        ch = ch.reshape(M + 1, ld, 2)
        return chi, [lam[b, :chi[b]].copy() for b in range(M + 1)], \
            [ch[b, :chi[b]].copy() for b in range(M + 1)]

    def sync(self) -> None:
        _check(_lib().mpo_sync(self._h), "mpo_sync")

    def close(self) -> None:
        if getattr(self, "_h", None):
            for pl in list(getattr(self, "_plans", ())):
                pl.close()
            _lib().mpo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
