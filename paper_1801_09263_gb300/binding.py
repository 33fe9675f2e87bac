"""ctypes binding of liblace (names follow the C calls of include/lace.h).

Arguments are marshalled to plain pointers and sizes; results come back in
caller-owned numpy arrays (host calls) or torch CUDA tensors (``_dev``
calls, where torch only provides the device memory and the stream).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

LACE_OK = 0
LACE_FP64, LACE_MIXED = 0, 1
LACE_SYM_AVG, LACE_SYM_UPPER, LACE_SYM_LOWER = 0, 1, 2
MAT_OVERLAP_MODULI, MAT_EXCHANGE, MAT_CHOLESKY, MAT_PAIR_ENERGY, MAT_SCDM_U = 0, 1, 2, 3, 4
ORB_PSI, ORB_W, ORB_XI = 0, 1, 2
REQ_REBUILD, REQ_APPLY = 0, 1
KERNEL_COULOMB, KERNEL_ERFC = 0, 1
SYSTEM_ALIGN = 1
STAGES = ("load", "localize", "screen", "exchange", "ace_build", "ace_apply", "pairconv_kernels")

_HERE = os.path.dirname(os.path.abspath(__file__))
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "lace.h")
_LIB = None


class LaceError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


def library_path() -> str:
    return os.path.join(_HERE, "liblace.so")


def exported_symbols() -> list[str]:
    """Function names declared in include/lace.h."""
    txt = open(_HEADER).read()
    return sorted(set(re.findall(r"\b(lace_[a-z_]+)\s*\(", txt)))


def load_library(build_if_missing: bool = False):
    """Load liblace.so from the package directory (in-tree build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            from .build import build
            build()
        else:
            raise RuntimeError(f"liblace.so not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    P, I, D, LL, V = C.c_void_p, C.c_int, C.c_double, C.c_longlong, None
    sig = {
        "lace_create": ([C.POINTER(P), I, I], I),
        "lace_destroy": ([P], I),
        "lace_set_stream": ([P, P], I),
        "lace_set_wait_limit": ([P, D], I),
        "lace_set_cell": ([P, P, I, I, I, D], I),
        "lace_load_orbitals": ([P, P, I, I, I], I),
        "lace_load_orbitals_dev": ([P, P, I, I, I], I),
        "lace_localize": ([P, I, P], I),
        "lace_set_pivots": ([P, P, I], I),
        "lace_screen": ([P, D, P], I),
        "lace_apply_exchange": ([P, P, P], I),
        "lace_exchange_energy": ([P, D, P], I),
        "lace_build_ace": ([P, I], I),
        "lace_apply_ace": ([P, P, I, P], I),
        "lace_apply_ace_dev": ([P, P, I, P], I),
        "lace_get_matrix": ([P, I, P, LL], I),
        "lace_get_orbitals": ([P, I, P, LL], I),
        "lace_get_pairs": ([P, P, LL, P], I),
        "lace_get_pivots": ([P, P, I], I),
        "lace_get_timings": ([P, P, I], I),
        "lace_get_launch_count": ([P, P], I),
        "lace_get_device_bytes": ([P, P], I),
        "lace_set_kernel": ([P, I, D, D], I),
        "lace_align_to_previous": ([P, P], I),
        "lace_pw_basis": ([P, D, P, LL, P], I),
        "lace_grid_for_cutoff": ([P, D, P], I),
        "lace_load_orbitals_pw": ([P, P, LL, I, I, I], I),
        "lace_get_orbitals_pw": ([P, I, P, LL], I),
        "lace_server_create": ([C.POINTER(P), I, I, I, I, C.c_ulonglong], I),
        "lace_server_destroy": ([P], I),
        "lace_server_add_system": ([P, P, I, I, I, D, I, I, D, I, P], I),
        "lace_server_submit": ([P, I, I, P, I, P, P], I),
        "lace_server_poll": ([P, LL, I, P, P, P, P, P], I),
        "lace_server_remove_system": ([P, I], I),
        "lace_server_request_error": ([P, LL], C.c_char_p),
        "lace_batch_create": ([C.POINTER(P), I, I, P], I),
        "lace_batch_destroy": ([P], I),
        "lace_batch_set_orbitals": ([P, I, P], I),
        "lace_batch_run": ([P, P, P], I),
        "lace_batch_context": ([P, I], P),
        "lace_batch_info": ([P, P, P, P, P, P, P, P, I], I),
        "lace_batch_mode": ([P, P], I),
        "lace_batch_last_error": ([P], C.c_char_p),
        "lace_server_stats": ([P, P, P, P], I),
        "lace_server_set_pair_merging": ([P, I, D], I),
        "lace_server_merge_stats": ([P, P, P, P], I),
        "lace_server_set_rebuild_tolerance": ([P, I, D], I),
        "lace_server_apply_info": ([P, LL, P, P], I),
        "lace_get_ace_energy": ([P, P], I),
        "lace_exchange_pairs_noalloc": ([P, I, I, I, P, I, I, P, LL, P, P, P], I),
        "lace_probe_peak_rates": ([I, P, I], I),
        "lace_status_string": ([I], C.c_char_p),
        "lace_last_error": ([P], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _LIB = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Lace:
    """One liblace context (one device, one precision)."""

    def __init__(self, device: int = 0, precision: int = LACE_FP64):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.lace_create(C.byref(h), int(device), int(precision))
        if st != LACE_OK:
            raise LaceError(st, "lace_create", self.lib.lace_status_string(st).decode())
        self.h = h
        self.precision = precision
        self.shape = None
        self.n_occ = self.n_extra = 0

    # -- helpers
    def _check(self, st: int, where: str):
        if st != LACE_OK:
            detail = self.lib.lace_last_error(self.h).decode()
            raise LaceError(st, where, detail or self.lib.lace_status_string(st).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lace_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_p(self) -> int:
        return self.n_occ + self.n_extra

    @property
    def ng(self) -> int:
        return int(np.prod(self.shape))

    # -- the C calls
    def set_stream(self, stream_ptr: int | None):
        self._check(self.lib.lace_set_stream(self.h, C.c_void_p(stream_ptr or 0)), "lace_set_stream")

    def set_wait_limit(self, seconds: float):
        self._check(self.lib.lace_set_wait_limit(self.h, float(seconds)), "lace_set_wait_limit")

    def set_cell(self, cell, shape, ecut: float):
        c = _f64(cell)
        self._check(self.lib.lace_set_cell(self.h, _ptr(c), int(shape[0]), int(shape[1]), int(shape[2]),
                                           float(ecut)), "lace_set_cell")
        self.shape = tuple(int(s) for s in shape)

    def set_kernel(self, kind: int = KERNEL_COULOMB, omega: float = 0.0, alpha: float = 1.0):
        """Coulomb (Eq. 2) or erfc-screened short-range kernel, times the exchange fraction alpha."""
        self._check(self.lib.lace_set_kernel(self.h, int(kind), float(omega), float(alpha)), "lace_set_kernel")

    def load_orbitals(self, phi, n_occ: int, n_extra: int = 0, orthonormalize: bool = True):
        a = _f64(phi)
        assert a.shape == (n_occ + n_extra,) + self.shape
        self._check(self.lib.lace_load_orbitals(self.h, _ptr(a), n_occ, n_extra, int(orthonormalize)),
                    "lace_load_orbitals")
        self.n_occ, self.n_extra = n_occ, n_extra

    def load_orbitals_pw(self, coef, n_occ: int, n_extra: int = 0, orthonormalize: bool = True):
        """coef: complex array [n_occ + n_extra, n_pw] in the basis of pw_basis(cell, ecut)."""
        c = np.ascontiguousarray(coef, dtype=np.complex128)
        self._check(self.lib.lace_load_orbitals_pw(self.h, c.ctypes.data_as(C.c_void_p), c.shape[1], n_occ, n_extra,
                                                   int(orthonormalize)), "lace_load_orbitals_pw")
        self.n_occ, self.n_extra = n_occ, n_extra

    def get_orbitals_pw(self, which: int, n_pw: int) -> np.ndarray:
        out = np.empty((self.n_p, n_pw), dtype=np.complex128)
        self._check(self.lib.lace_get_orbitals_pw(self.h, int(which), out.ctypes.data_as(C.c_void_p), int(n_pw)),
                    "lace_get_orbitals_pw")
        return out

    def load_orbitals_dev(self, phi_dev, n_occ: int, n_extra: int = 0, orthonormalize: bool = True):
        """phi_dev: a contiguous float64 CUDA torch tensor [(n_occ+n_extra), n1, n2, n3]."""
        assert phi_dev.is_cuda and phi_dev.is_contiguous() and str(phi_dev.dtype) == "torch.float64"
        self._check(self.lib.lace_load_orbitals_dev(self.h, C.c_void_p(phi_dev.data_ptr()), n_occ, n_extra,
                                                    int(orthonormalize)), "lace_load_orbitals_dev")
        self.n_occ, self.n_extra = n_occ, n_extra

    def localize(self, stride: int = 2) -> np.ndarray:
        piv = np.zeros(self.n_occ, dtype=np.int64)
        self._check(self.lib.lace_localize(self.h, int(stride), _ptr(piv)), "lace_localize")
        return piv

    def set_pivots(self, pivots):
        p = np.ascontiguousarray(pivots, dtype=np.int64)
        self._check(self.lib.lace_set_pivots(self.h, _ptr(p), len(p)), "lace_set_pivots")

    def align_to_previous(self) -> bool:
        """Rotate the localised orbitals to the previous call's set (True when rotated)."""
        a = C.c_int(0)
        self._check(self.lib.lace_align_to_previous(self.h, C.byref(a)), "lace_align_to_previous")
        return bool(a.value)

    def screen(self, s_thr: float) -> int:
        n = C.c_longlong(0)
        self._check(self.lib.lace_screen(self.h, float(s_thr), C.byref(n)), "lace_screen")
        return int(n.value)

    def apply_exchange(self, want_W: bool = True):
        ex = C.c_double(0.0)
        want_W = want_W and self.shape is not None and self.n_p > 0
        W = np.empty((self.n_p,) + self.shape, dtype=np.float64) if want_W else None
        self._check(self.lib.lace_apply_exchange(self.h, _ptr(W) if want_W else None, C.byref(ex)),
                    "lace_apply_exchange")
        return W, float(ex.value)

    def exchange_energy(self, f_spin: float = 1.0) -> float:
        ex = C.c_double(0.0)
        self._check(self.lib.lace_exchange_energy(self.h, float(f_spin), C.byref(ex)), "lace_exchange_energy")
        return float(ex.value)

    def build_ace(self, sym: int = LACE_SYM_AVG):
        self._check(self.lib.lace_build_ace(self.h, int(sym)), "lace_build_ace")

    def apply_ace(self, psi) -> np.ndarray:
        a = _f64(psi)
        n = a.shape[0]
        out = np.empty_like(a)
        self._check(self.lib.lace_apply_ace(self.h, _ptr(a), n, _ptr(out)), "lace_apply_ace")
        return out

    def apply_ace_dev(self, psi_dev, out_dev):
        assert psi_dev.is_cuda and out_dev.is_cuda and psi_dev.is_contiguous() and out_dev.is_contiguous()
        self._check(self.lib.lace_apply_ace_dev(self.h, C.c_void_p(psi_dev.data_ptr()), int(psi_dev.shape[0]),
                                                C.c_void_p(out_dev.data_ptr())), "lace_apply_ace_dev")

    def get_matrix(self, which: int) -> np.ndarray:
        n = self.n_p if which in (MAT_EXCHANGE, MAT_CHOLESKY) else self.n_occ
        out = np.empty((n, n), dtype=np.float64)
        self._check(self.lib.lace_get_matrix(self.h, int(which), _ptr(out), out.size), "lace_get_matrix")
        return out

    def get_orbitals(self, which: int) -> np.ndarray:
        out = np.empty((self.n_p,) + self.shape, dtype=np.float64)
        self._check(self.lib.lace_get_orbitals(self.h, int(which), _ptr(out), out.size), "lace_get_orbitals")
        return out

    def get_pairs(self) -> np.ndarray:
        n = C.c_longlong(0)
        self._check(self.lib.lace_get_pairs(self.h, None, 0, C.byref(n)), "lace_get_pairs")
        out = np.empty((max(n.value, 1), 2), dtype=np.int32)
        self._check(self.lib.lace_get_pairs(self.h, _ptr(out), n.value, C.byref(n)), "lace_get_pairs")
        return out[: n.value]

    def ace_energy(self) -> float:
        """sum_j <psi_j|K_ACE|psi_j> of the last ACE application's block."""
        e = C.c_double(0)
        self._check(self.lib.lace_get_ace_energy(self.h, C.byref(e)), "lace_get_ace_energy")
        return e.value

    def get_pivots(self) -> np.ndarray:
        out = np.empty(self.n_occ, dtype=np.int64)
        self._check(self.lib.lace_get_pivots(self.h, _ptr(out), int(self.n_occ)), "lace_get_pivots")
        return out

    def get_timings(self) -> dict:
        ms = np.zeros(len(STAGES), dtype=np.float64)
        self._check(self.lib.lace_get_timings(self.h, _ptr(ms), len(STAGES)), "lace_get_timings")
        return dict(zip(STAGES, ms.tolist()))

    def launch_count(self) -> int:
        n = C.c_longlong(0)
        self._check(self.lib.lace_get_launch_count(self.h, C.byref(n)), "lace_get_launch_count")
        return int(n.value)

    def device_bytes(self) -> int:
        n = C.c_ulonglong(0)
        self._check(self.lib.lace_get_device_bytes(self.h, C.byref(n)), "lace_get_device_bytes")
        return int(n.value)


class Server:
    """lace_server_*: requests against resident systems, run by `slots`
    worker threads (at most `rebuild_slots` of them on rebuilds; 0 = all)
    under a device-memory budget (0 = 90% of free memory).

    submit() keeps the request's arrays alive until its poll(wait=True) (or
    a done poll) has returned, as the C call borrows them until completion.
    """

    def __init__(self, device: int = 0, precision: int = LACE_MIXED, slots: int = 4, rebuild_slots: int = 0,
                 mem_bytes: int = 0):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.lace_server_create(C.byref(h), int(device), int(precision), int(slots), int(rebuild_slots),
                                         int(mem_bytes))
        if st != LACE_OK:
            raise LaceError(st, "lace_server_create", self.lib.lace_status_string(st).decode())
        self.h = h
        self._systems = {}
        self._live = {}

    def _check(self, st: int, where: str):
        if st != LACE_OK:
            raise LaceError(st, where, self.lib.lace_status_string(st).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lace_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_system(self, cell, shape, ecut: float, n_occ: int, n_extra: int = 0, s_thr: float = 1e-3,
                   align: bool = False) -> int:
        c = _f64(cell)
        sid = C.c_int(-1)
        self._check(self.lib.lace_server_add_system(self.h, _ptr(c), int(shape[0]), int(shape[1]), int(shape[2]),
                                                    float(ecut), int(n_occ), int(n_extra), float(s_thr),
                                                    SYSTEM_ALIGN if align else 0, C.byref(sid)),
                    "lace_server_add_system")
        self._systems[sid.value] = (tuple(int(x) for x in shape), int(n_occ) + int(n_extra))
        return sid.value

    def submit_rebuild(self, system: int, phi) -> int:
        a = _f64(phi)
        shape, n_p = self._systems[system]
        assert a.shape == (n_p,) + shape
        rid = C.c_longlong(0)
        self._check(self.lib.lace_server_submit(self.h, int(system), REQ_REBUILD, _ptr(a), n_p, None,
                                                C.byref(rid)), "lace_server_submit")
        self._live[rid.value] = (a, None)
        return rid.value

    def submit_apply(self, system: int, psi, out=None) -> int:
        """K_ACE psi into `out` (a new array unless given, e.g. a pinned buffer)."""
        a = _f64(psi)
        shape, _ = self._systems[system]
        assert a.shape[1:] == shape
        if out is None:
            out = np.empty_like(a)
        assert out.shape == a.shape and out.dtype == np.float64 and out.flags.c_contiguous
        rid = C.c_longlong(0)
        self._check(self.lib.lace_server_submit(self.h, int(system), REQ_APPLY, _ptr(a), a.shape[0], _ptr(out),
                                                C.byref(rid)), "lace_server_submit")
        self._live[rid.value] = (a, out)
        return rid.value

    def poll(self, request: int, wait: bool = True) -> dict | None:
        """None while running; else {status, latency_ms, ex, n_pairs, out}."""
        done, res, lat, ex, npairs = C.c_int(0), C.c_int(0), C.c_double(0), C.c_double(0), C.c_longlong(0)
        self._check(self.lib.lace_server_poll(self.h, int(request), int(wait), C.byref(done), C.byref(res),
                                              C.byref(lat), C.byref(ex), C.byref(npairs)), "lace_server_poll")
        if not done.value:
            return None
        _, out = self._live.pop(request, (None, None))
        err = self.lib.lace_server_request_error(self.h, int(request)) if res.value else b""
        eb, due = C.c_double(0), C.c_int(0)
        self._check(self.lib.lace_server_apply_info(self.h, int(request), C.byref(eb), C.byref(due)),
                    "lace_server_apply_info")
        return dict(status=res.value, latency_ms=lat.value, ex=ex.value, n_pairs=npairs.value, out=out,
                    error=(err or b"").decode(), e_block=eb.value, rebuild_due=bool(due.value))

    def remove_system(self, system: int):
        self._check(self.lib.lace_server_remove_system(self.h, int(system)), "lace_server_remove_system")

    def stats(self) -> dict:
        b, r, q = C.c_ulonglong(0), C.c_int(0), C.c_int(0)
        self._check(self.lib.lace_server_stats(self.h, C.byref(b), C.byref(r), C.byref(q)), "lace_server_stats")
        return dict(bytes_resident=int(b.value), running=r.value, queued=q.value)

    def set_rebuild_tolerance(self, system: int, tol: float):
        self._check(self.lib.lace_server_set_rebuild_tolerance(self.h, int(system), float(tol)),
                    "lace_server_set_rebuild_tolerance")

    def set_pair_merging(self, enable: bool = True, window_ms: float = 50.0):
        self._check(self.lib.lace_server_set_pair_merging(self.h, int(bool(enable)), float(window_ms)),
                    "lace_server_set_pair_merging")

    def merge_stats(self) -> dict:
        b, mb, mr = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
        self._check(self.lib.lace_server_merge_stats(self.h, C.byref(b), C.byref(mb), C.byref(mr)),
                    "lace_server_merge_stats")
        return dict(batches=b.value, merged_batches=mb.value, merged_requests=mr.value)


class _Instance(C.Structure):
    _fields_ = [("cell", C.c_double * 3), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int),
                ("ecut_ha", C.c_double), ("n_occ", C.c_int), ("s_thr", C.c_double)]


TUNE_SHAPES = ((128, 1), (128, 2), (128, 3), (128, 4), (256, 1), (256, 2), (512, 1), (512, 2))


class Batch:
    """lace_batch_*: independent systems run together (mixed precision).

    instances: sequence of (cell, shape, ecut, n_occ, s_thr).  set_orbitals()
    keeps the arrays alive: the library reads them on every run().
    """

    def __init__(self, instances, device: int = 0):
        self.lib = load_library()
        arr = (_Instance * len(instances))()
        self.shapes = []
        for k, (cell, shape, ecut, n_occ, s_thr) in enumerate(instances):
            arr[k].cell[:] = [float(x) for x in cell]
            arr[k].n1, arr[k].n2, arr[k].n3 = (int(x) for x in shape)
            arr[k].ecut_ha, arr[k].n_occ, arr[k].s_thr = float(ecut), int(n_occ), float(s_thr)
            self.shapes.append(((int(n_occ),) + tuple(int(x) for x in shape)))
        h = C.c_void_p()
        st = self.lib.lace_batch_create(C.byref(h), int(device), len(instances), C.cast(arr, C.c_void_p))
        if st != LACE_OK:
            raise LaceError(st, "lace_batch_create", self.lib.lace_status_string(st).decode())
        self.h = h
        self.n = len(instances)
        self._phi = [None] * self.n

    def _check(self, st: int, where: str):
        if st != LACE_OK:
            detail = self.lib.lace_batch_last_error(self.h).decode() if self.h else ""
            raise LaceError(st, where, detail or self.lib.lace_status_string(st).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lace_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_orbitals(self, inst: int, phi):
        a = _f64(phi)
        assert a.shape == self.shapes[inst]
        self._phi[inst] = a
        self._check(self.lib.lace_batch_set_orbitals(self.h, int(inst), _ptr(a)), "lace_batch_set_orbitals")

    def run(self):
        """(E_x per instance, status per instance)."""
        ex = np.zeros(self.n, dtype=np.float64)
        st = np.zeros(self.n, dtype=np.int32)
        self._check(self.lib.lace_batch_run(self.h, _ptr(ex), _ptr(st)), "lace_batch_run")
        return ex, st

    def context(self, inst: int) -> "Lace":
        """A non-owning Lace view of an instance's context (for the getters)."""
        h = self.lib.lace_batch_context(self.h, int(inst))
        if not h:
            raise LaceError(1, "lace_batch_context", "bad instance")
        view = Lace.__new__(Lace)
        view.lib, view.h, view.precision = self.lib, C.c_void_p(h), LACE_MIXED
        n_occ = self.shapes[inst][0]
        view.shape, view.n_occ, view.n_extra = self.shapes[inst][1:], n_occ, 0
        view.close = lambda: None  # owned by the batch
        return view

    def info(self) -> dict:
        th, ct, ch = C.c_int(0), C.c_int(0), C.c_int(0)
        rp, ln = C.c_longlong(0), C.c_longlong(0)
        ms = np.zeros(4, dtype=np.float64)
        tune = np.zeros(len(TUNE_SHAPES) + 1, dtype=np.float64)
        self._check(self.lib.lace_batch_info(self.h, C.byref(th), C.byref(ct), C.byref(ch), C.byref(rp), C.byref(ln),
                                             _ptr(ms), _ptr(tune), len(tune)), "lace_batch_info")
        pi = C.c_int(0)
        self._check(self.lib.lace_batch_mode(self.h, C.byref(pi)), "lace_batch_mode")
        per_instance = pi.value != 0
        tune_ms = {f"{a}x{b}": round(float(t), 3) for (a, b), t in zip(TUNE_SHAPES, tune)}
        tune_ms["per_instance"] = round(float(tune[-1]), 3)
        return dict(threads=th.value, ctas_per_sm=ct.value, chunks=ch.value, graph_replays=rp.value,
                    launches=ln.value, setup_ms=ms[0], pairconv_ms=ms[1], hot_ms=ms[2], call_ms=ms[3],
                    mode="per_instance" if per_instance else "persistent", tune_ms=tune_ms)


def probe_peak_rates(device: int = 0) -> dict:
    """Measured FP32 (scalar and packed-pair FMA) and FP64 FMA rates of a device, in TFLOP/s."""
    lib = load_library()
    r = np.zeros(3, dtype=np.float64)
    st = lib.lace_probe_peak_rates(int(device), _ptr(r), 3)
    if st != LACE_OK:
        raise LaceError(st, "lace_probe_peak_rates", lib.lace_status_string(st).decode())
    return {"fp32_tflops": r[0] / 1e12, "fp32x2_tflops": r[1] / 1e12, "fp64_tflops": r[2] / 1e12}


def pw_basis(cell, ecut: float) -> np.ndarray:
    """lace_pw_basis: the (m1, m2, m3) of the half-sphere basis, int [n_pw, 3]."""
    lib = load_library()
    c = _f64(cell)
    n = C.c_longlong(0)
    st = lib.lace_pw_basis(_ptr(c), float(ecut), None, 0, C.byref(n))
    if st != LACE_OK:
        raise LaceError(st, "lace_pw_basis", lib.lace_status_string(st).decode())
    m = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    lib.lace_pw_basis(_ptr(c), float(ecut), _ptr(m), n.value, C.byref(n))
    return m[: n.value]


def grid_for_cutoff(cell, ecut: float) -> tuple:
    """lace_grid_for_cutoff: the smallest 2/3/5-smooth grid holding the sphere."""
    lib = load_library()
    c = _f64(cell)
    d = np.zeros(3, dtype=np.int32)
    st = lib.lace_grid_for_cutoff(_ptr(c), float(ecut), _ptr(d))
    if st != LACE_OK:
        raise LaceError(st, "lace_grid_for_cutoff", lib.lace_status_string(st).decode())
    return tuple(int(x) for x in d)
