"""Thin ctypes binding of the C ABI in ``include/qhp.h`` (argument marshalling only).

Every function mirrors the C entry point of the same name; a nonzero return
code raises :class:`QHPError` carrying ``qhp_last_error()``.  Host arrays are
numpy; the ``_device`` variants take torch CUDA tensors (their data_ptr()).
There is no CPU fallback: if ``libqhp.so`` is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# QHP_LIBRARY selects another build of the library (the bounds-checked libqhp_check.so)
LIB_PATH = os.environ.get("QHP_LIBRARY") or os.path.join(_HERE, "libqhp.so")

QHP_OK = 0
ERRORS = {-1: "QHP_ERR_ARG", -2: "QHP_ERR_CUDA", -3: "QHP_ERR_TIMEOUT", -4: "QHP_ERR_NONFINITE",
          -5: "QHP_ERR_LIST_OVERFLOW", -6: "QHP_ERR_STATE", -7: "QHP_ERR_NOMEM", -8: "QHP_ERR_BOUNDS"}
QHP_FP64, QHP_MIXED = 0, 1
QHP_THERMO_PILE, QHP_THERMO_ADQTB, QHP_THERMO_NVE = 0, 1, 2
QHP_ADAPT_NONE, QHP_ADAPT_SIMPLE, QHP_ADAPT_RATIO = 0, 1, 2
QHP_INTEGRATOR_BAOAB, QHP_INTEGRATOR_BCOCB = 0, 1


class QHPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class qhp_ff(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eps", "sigma", "q_O", "k_b", "r0", "k_theta", "theta0",
                                          "alpha", "rc", "skin", "m_O", "m_H")]


class qhp_thermo(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma0", C.c_double), ("dt_fs", C.c_double), ("n_seg", C.c_int),
                ("omega_cut_cm", C.c_double), ("a_gamma", C.c_double), ("gamma_min_frac", C.c_double),
                ("adapt", C.c_int), ("tau_ratio_ps", C.c_double), ("integrator", C.c_int)]


class qhp_energy(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("potential", "spring", "kinetic_nm", "kinetic_cv", "fdt_delta",
                                          "bonded", "nonbonded", "reserved")]


class qhp_info(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("P", C.c_int), ("precision", C.c_int), ("list_mode", C.c_int),
                ("step", C.c_int64), ("rebuilds", C.c_int64), ("list_entries", C.c_int64),
                ("list_capacity", C.c_int64), ("kernel_launches", C.c_int64),
                ("n_cells_per_edge", C.c_int), ("reserved", C.c_int)]


_lib = None
_VP, _DP, _FP, _IP = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int)
_SIGS = {
    "qhp_create_system": [C.POINTER(C.c_void_p), C.c_int, _IP, _IP, _DP, C.c_double, C.c_int],
    "qhp_destroy_system": [_VP],
    "qhp_set_forcefield": [_VP, C.POINTER(qhp_ff)],
    "qhp_set_beads": [_VP, C.c_int, C.c_double, C.c_uint64],
    "qhp_set_thermostat": [_VP, C.POINTER(qhp_thermo)],
    "qhp_step_rpmd": [_VP, C.c_int],
    "qhp_step_adqtb": [_VP, C.c_int],
    "qhp_compute_forces": [_VP],
    "qhp_sync": [_VP],
    "qhp_get_energy": [_VP, C.POINTER(qhp_energy)],
    "qhp_get_forces": [_VP, _DP],
    "qhp_get_centroid": [_VP, _DP],
    "qhp_get_beads": [_VP, _DP],
    "qhp_get_modes": [_VP, _DP, _DP],
    "qhp_set_modes": [_VP, _DP, _DP],
    "qhp_set_modes_device": [_VP, _VP, _VP],
    "qhp_get_modes_device": [_VP, _VP, _VP],
    "qhp_get_forces_device": [_VP, _VP],
    "qhp_get_state": [_VP, _VP, C.POINTER(C.c_size_t)],
    "qhp_set_state": [_VP, _VP, C.c_size_t],
    "qhp_get_gamma": [_VP, _DP],
    "qhp_set_gamma": [_VP, _DP],
    "qhp_get_qtb_noise": [_VP, _FP],
    "qhp_get_qtb_records": [_VP, _FP, _FP],
    "qhp_build_list": [_VP],
    "qhp_get_cells": [_VP, _IP, _IP],
    "qhp_get_list_pairs": [_VP, C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64)],
    "qhp_get_info": [_VP, C.POINTER(qhp_info)],
    "qhp_set_stream": [_VP, _VP],
    "qhp_set_profiling": [_VP, C.c_int],
    "qhp_set_graph_mode": [_VP, C.c_int],
    "qhp_set_respa": [_VP, C.c_int, C.c_int],
    "qhp_get_profile": [_VP, _VP],
    "qhp_count_pairs": [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "qhp_estimators_noalloc": [C.c_int, C.c_int, C.c_double, _VP, _VP, _VP, _VP, _VP, _VP],
    "qhp_get_list_row": [_VP, C.c_int, _IP, C.c_int, _IP],
    "qhp_create_batch": [C.POINTER(_VP), C.c_int, C.POINTER(_VP)],
    "qhp_destroy_batch": [_VP],
    "qhp_batch_step": [_VP, C.c_int],
    "qhp_batch_sync": [_VP],
    "qhp_batch_set_stream": [_VP, _VP],
    "qhp_batch_autotune": [_VP, C.c_int, _IP],
    "qhp_batch_get_info": [_VP, _VP],
    "qhp_batch_get_profile": [_VP, _VP],
    "qhp_batch_set_wait_limit": [_VP, C.c_longlong],
    "qhp_selftest_grid_barrier": [C.c_longlong, C.POINTER(C.c_uint)],
    "qhp_autotune": [_VP, C.c_int, _IP],
    "qhp_set_pair_warps": [_VP, C.c_int],
    "qhp_set_pair_skip": [_VP, C.c_int],
    "qhp_state_energies": [_VP, _DP, _DP, _DP],
    "qhp_bar": [_DP, C.c_int, _DP, C.c_int, C.c_double, C.c_double, _DP, _IP],
    "qhp_energy_grad": [_VP, _DP, _DP, _DP],
    "qhp_energy_grad_device": [_VP, _VP, _DP, _VP, _DP],
    "qhp_segment_grad": [_VP, C.c_int, C.c_int, C.c_int, _DP, _DP],
}


class qhp_profile(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("integrate_ms", "list_ms", "pair_ms", "bonded_ms", "project_ms",
                                         "step_ms")]


def lib():
    """Load libqhp.so (raises if it was not built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing (run paper_2212_03137_b300.build)")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.qhp_last_error.argtypes = []
        L.qhp_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != QHP_OK:
        raise QHPError(rc, lib().qhp_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(_DP)


def _fp(a):
    return a.ctypes.data_as(_FP)


def _ip(a):
    return a.ctypes.data_as(_IP)


# ------------------------------------------------------------------ C mirrors

def qhp_create_system(types, molecule, pos, box, precision) -> C.c_void_p:
    t = np.ascontiguousarray(types, dtype=np.int32)
    m = np.ascontiguousarray(molecule, dtype=np.int32)
    p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    h = C.c_void_p()
    _check(lib().qhp_create_system(C.byref(h), int(len(t)), _ip(t), _ip(m), _dp(p), float(box), int(precision)))
    return h


def qhp_destroy_system(h) -> None:
    _check(lib().qhp_destroy_system(h))


def qhp_set_forcefield(h, ff: qhp_ff) -> None:
    _check(lib().qhp_set_forcefield(h, C.byref(ff)))


def qhp_set_beads(h, P: int, temperature: float, seed: int) -> None:
    _check(lib().qhp_set_beads(h, int(P), float(temperature), int(seed)))


def qhp_set_thermostat(h, th: qhp_thermo) -> None:
    _check(lib().qhp_set_thermostat(h, C.byref(th)))


def qhp_step_rpmd(h, n: int) -> None:
    _check(lib().qhp_step_rpmd(h, int(n)))


def qhp_step_adqtb(h, n: int) -> None:
    _check(lib().qhp_step_adqtb(h, int(n)))


def qhp_compute_forces(h) -> None:
    _check(lib().qhp_compute_forces(h))


def qhp_sync(h) -> None:
    _check(lib().qhp_sync(h))


def qhp_get_energy(h) -> qhp_energy:
    e = qhp_energy()
    _check(lib().qhp_get_energy(h, C.byref(e)))
    return e


def qhp_get_info(h) -> qhp_info:
    i = qhp_info()
    _check(lib().qhp_get_info(h, C.byref(i)))
    return i


def _dims(h):
    i = qhp_get_info(h)
    return i.n_atoms, i.P


def qhp_get_forces(h, out=None) -> np.ndarray:
    N, P = _dims(h)
    out = np.empty((P, N, 3)) if out is None else out
    _check(lib().qhp_get_forces(h, _dp(out)))
    return out


def qhp_get_centroid(h) -> np.ndarray:
    N, _ = _dims(h)
    out = np.empty((N, 3))
    _check(lib().qhp_get_centroid(h, _dp(out)))
    return out


def qhp_get_beads(h) -> np.ndarray:
    N, P = _dims(h)
    out = np.empty((P, N, 3))
    _check(lib().qhp_get_beads(h, _dp(out)))
    return out


def qhp_get_modes(h):
    N, P = _dims(h)
    Q, Pm = np.empty((N, 3, P)), np.empty((N, 3, P))
    _check(lib().qhp_get_modes(h, _dp(Q), _dp(Pm)))
    return Q, Pm


def qhp_set_modes(h, Q, Pm) -> None:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    Pm = np.ascontiguousarray(Pm, dtype=np.float64)
    _check(lib().qhp_set_modes(h, _dp(Q), _dp(Pm)))


def qhp_set_modes_device(h, Q, Pm) -> None:
    """Q, Pm: contiguous float64 CUDA tensors [N, 3, P] (or None)."""
    _check(lib().qhp_set_modes_device(h, C.c_void_p(Q.data_ptr() if Q is not None else 0),
                                      C.c_void_p(Pm.data_ptr() if Pm is not None else 0)))


def qhp_get_modes_device(h, Q, Pm) -> None:
    _check(lib().qhp_get_modes_device(h, C.c_void_p(Q.data_ptr() if Q is not None else 0),
                                      C.c_void_p(Pm.data_ptr() if Pm is not None else 0)))


def qhp_get_forces_device(h, out) -> None:
    _check(lib().qhp_get_forces_device(h, C.c_void_p(out.data_ptr())))


def qhp_get_state(h) -> bytes:
    size = C.c_size_t(0)
    _check(lib().qhp_get_state(h, None, C.byref(size)))
    buf = C.create_string_buffer(size.value)
    _check(lib().qhp_get_state(h, C.cast(buf, C.c_void_p), C.byref(size)))
    return buf.raw


def qhp_set_state(h, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().qhp_set_state(h, C.cast(buf, C.c_void_p), len(blob)))


def qhp_get_gamma(h, n_seg: int) -> np.ndarray:
    out = np.empty((2, n_seg + 1))
    _check(lib().qhp_get_gamma(h, _dp(out)))
    return out


def qhp_set_gamma(h, g) -> None:
    g = np.ascontiguousarray(g, dtype=np.float64)
    _check(lib().qhp_set_gamma(h, _dp(g)))


def qhp_get_qtb_noise(h, n_seg: int) -> np.ndarray:
    N, _ = _dims(h)
    out = np.empty((n_seg, 3 * N), dtype=np.float32)
    _check(lib().qhp_get_qtb_noise(h, _fp(out)))
    return out


def qhp_get_qtb_records(h, n_seg: int):
    N, _ = _dims(h)
    v = np.empty((n_seg, 3 * N), dtype=np.float32)
    F = np.empty((n_seg, 3 * N), dtype=np.float32)
    _check(lib().qhp_get_qtb_records(h, _fp(v), _fp(F)))
    return v, F


def qhp_build_list(h) -> None:
    _check(lib().qhp_build_list(h))


def qhp_get_cells(h):
    N, _ = _dims(h)
    cell = np.empty(N, dtype=np.int32)
    order = np.empty(N, dtype=np.int32)
    _check(lib().qhp_get_cells(h, _ip(cell), _ip(order)))
    return cell, order


def qhp_get_list_pairs(h) -> np.ndarray:
    cnt = C.c_int64(0)
    _check(lib().qhp_get_list_pairs(h, None, 0, C.byref(cnt)))
    out = np.empty((max(cnt.value, 1), 2), dtype=np.int64)
    _check(lib().qhp_get_list_pairs(h, out.ctypes.data_as(C.POINTER(C.c_int64)), cnt.value, C.byref(cnt)))
    return out[: cnt.value]


def qhp_get_list_row(h, atom: int) -> np.ndarray:
    cnt = C.c_int(0)
    buf = np.empty(4096, dtype=np.int32)
    _check(lib().qhp_get_list_row(h, int(atom), _ip(buf), len(buf), C.byref(cnt)))
    if cnt.value > len(buf):
        buf = np.empty(cnt.value, dtype=np.int32)
        _check(lib().qhp_get_list_row(h, int(atom), _ip(buf), len(buf), C.byref(cnt)))
    return buf[: cnt.value].copy()


def qhp_set_stream(h, stream_ptr: int | None) -> None:
    _check(lib().qhp_set_stream(h, C.c_void_p(stream_ptr or 0)))


def qhp_set_profiling(h, on: bool) -> None:
    _check(lib().qhp_set_profiling(h, 1 if on else 0))


def qhp_set_respa(h, n_alt: int, contracted_beads: int = 0) -> None:
    _check(lib().qhp_set_respa(h, int(n_alt), int(contracted_beads)))


def qhp_set_graph_mode(h, use_graphs: bool) -> None:
    _check(lib().qhp_set_graph_mode(h, 1 if use_graphs else 0))


def qhp_get_profile(h) -> qhp_profile:
    p = qhp_profile()
    _check(lib().qhp_get_profile(h, C.cast(C.byref(p), C.c_void_p)))
    return p


def qhp_estimators_noalloc(n_atoms: int, P: int, temperature: float, Q, Pm, F, mass, out, stream: int = 0) -> None:
    """Device tensors in, device tensor out (see include/qhp.h); allocates nothing."""
    def ptr(t):
        return C.c_void_p(t.data_ptr() if t is not None else 0)
    _check(lib().qhp_estimators_noalloc(int(n_atoms), int(P), float(temperature), ptr(Q), ptr(Pm), ptr(F), ptr(mass),
                                        ptr(out), C.c_void_p(stream or 0)))


def qhp_count_pairs(h) -> tuple[int, int]:
    a, b = C.c_int64(0), C.c_int64(0)
    _check(lib().qhp_count_pairs(h, C.byref(a), C.byref(b)))
    return a.value, b.value


# ------------------------------------------------------------------ convenience

class qhp_batch_info(C.Structure):
    _fields_ = [("n_sys", C.c_int), ("kernels_per_step", C.c_int), ("atom_beads", C.c_int64), ("steps", C.c_int64),
                ("rebuilds", C.c_int64), ("kernel_launches", C.c_int64), ("grid_integrate", C.c_int),
                ("grid_pair", C.c_int), ("grid_bonded", C.c_int), ("grid_project", C.c_int), ("items_pair", C.c_int),
                ("reserved", C.c_int)]


def qhp_create_batch(handles) -> int:
    arr = (_VP * len(handles))(*handles)
    b = _VP()
    _check(lib().qhp_create_batch(C.byref(b), len(handles), arr))
    return b


def qhp_destroy_batch(b) -> None:
    _check(lib().qhp_destroy_batch(b))


def qhp_batch_step(b, n: int) -> None:
    _check(lib().qhp_batch_step(b, int(n)))


def qhp_batch_sync(b) -> None:
    _check(lib().qhp_batch_sync(b))


def qhp_batch_set_stream(b, stream_ptr: int | None) -> None:
    _check(lib().qhp_batch_set_stream(b, C.c_void_p(stream_ptr or 0)))


def qhp_batch_autotune(b, reps: int = 5) -> dict:
    """Tuned warps per atom by bead count, {P: W}."""
    out = (C.c_int * 7)()
    _check(lib().qhp_batch_autotune(b, int(reps), out))
    return {1 << k: out[k] for k in range(7) if out[k]}


def qhp_batch_get_info(b) -> qhp_batch_info:
    info = qhp_batch_info()
    _check(lib().qhp_batch_get_info(b, C.cast(C.byref(info), C.c_void_p)))
    return info


def qhp_batch_get_profile(b):
    p = qhp_profile()
    _check(lib().qhp_batch_get_profile(b, C.cast(C.byref(p), C.c_void_p)))
    return p


def qhp_batch_set_wait_limit(b, wait_ns: int) -> None:
    _check(lib().qhp_batch_set_wait_limit(b, int(wait_ns)))


def qhp_selftest_grid_barrier(wait_ns: int) -> tuple[int, int]:
    """(return code, status word) of the grid barrier's time-limit self-test; not raised."""
    st = C.c_uint(0)
    rc = lib().qhp_selftest_grid_barrier(int(wait_ns), C.byref(st))
    return rc, st.value


def qhp_autotune(h, reps: int = 5) -> int:
    w = C.c_int(0)
    _check(lib().qhp_autotune(h, int(reps), C.byref(w)))
    return w.value


def qhp_set_pair_warps(h, w: int) -> None:
    _check(lib().qhp_set_pair_warps(h, int(w)))


def qhp_set_pair_skip(h, enabled: bool) -> None:
    _check(lib().qhp_set_pair_skip(h, 1 if enabled else 0))


class Batch:
    """Owns one qhp_batch over caller-owned System objects (kept alive here)."""

    def __init__(self, systems):
        self.systems = list(systems)
        self.h = qhp_create_batch([s.h for s in self.systems])

    def step(self, n: int) -> None:
        qhp_batch_step(self.h, n)

    def sync(self) -> None:
        qhp_batch_sync(self.h)

    def close(self):
        if self.h is not None:
            qhp_destroy_batch(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PARAM_NAMES = ("eps", "sigma", "q_O", "k_b", "k_theta")


def qhp_energy_grad(h):
    """(U_P, dU_P/dx [P, N, 3], dU_P/dtheta [5]) at the current bead positions."""
    N, P = _dims(h)
    e = C.c_double(0.0)
    gx = np.empty((P, N, 3))
    gt = np.empty(5)
    _check(lib().qhp_energy_grad(h, C.byref(e), _dp(gx), _dp(gt)))
    return e.value, gx, gt


def qhp_energy_grad_device(h, x_ptr: int | None, gx_ptr: int | None, want_theta: bool = True):
    """Device variant: x_ptr / gx_ptr are device addresses of [P, N, 3] FP64 arrays (or None)."""
    e = C.c_double(0.0)
    gt = np.empty(5)
    _check(lib().qhp_energy_grad_device(h, C.c_void_p(x_ptr or 0), C.byref(e), C.c_void_p(gx_ptr or 0),
                                        _dp(gt) if want_theta else None))
    return e.value, gt


def qhp_segment_grad(h, K: int, block: int, observable: int):
    """(J, dJ/dtheta [5]) of the K-step time average of observable 0 (centroid V) or 1 (mean O-H)."""
    J = C.c_double(0.0)
    g = np.empty(5)
    _check(lib().qhp_segment_grad(h, int(K), int(block), int(observable), C.byref(J), _dp(g)))
    return J.value, g


def qhp_state_energies(h, theta_A, theta_B) -> np.ndarray:
    """[U_P(A), U_P(B), V_A(x_0), V_B(x_0)] at the current beads (kcal/mol)."""
    a = np.ascontiguousarray(theta_A, dtype=np.float64)
    b = np.ascontiguousarray(theta_B, dtype=np.float64)
    out = np.empty(4)
    _check(lib().qhp_state_energies(h, _dp(a), _dp(b), _dp(out)))
    return out


def qhp_bar(dU_A, dU_B, beta: float, tol: float = 1e-12):
    """(Dlt F_AB, iterations) by (PI-)BAR from dU = U_B - U_A sampled in A and in B."""
    a = np.ascontiguousarray(dU_A, dtype=np.float64)
    b = np.ascontiguousarray(dU_B, dtype=np.float64)
    dF = C.c_double(0.0)
    it = C.c_int(0)
    _check(lib().qhp_bar(_dp(a), len(a), _dp(b), len(b), float(beta), float(tol), C.byref(dF), C.byref(it)))
    return dF.value, it.value


def ff_with_params(ff: qhp_ff, theta) -> qhp_ff:
    """Copy of ff with (eps, sigma, q_O, k_b, k_theta) replaced."""
    out = qhp_ff()
    C.pointer(out)[0] = ff
    for n, v in zip(PARAM_NAMES, theta):
        setattr(out, n, float(v))
    return out


def ff_params(ff: qhp_ff) -> np.ndarray:
    return np.array([getattr(ff, n) for n in PARAM_NAMES], dtype=float)


def make_ff(rc: float, skin: float = 2.0, **kw) -> qhp_ff:
    from .workloads import WATER_FF as W
    p = dict(eps=W["eps"], sigma=W["sigma"], q_O=W["q_O"], k_b=W["k_b"], r0=W["r0"], k_theta=W["k_theta"],
             theta0=math.radians(W["theta0_deg"]), alpha=W["alpha"], rc=rc, skin=skin, m_O=W["m_O"], m_H=W["m_H"])
    p.update(kw)
    return qhp_ff(**p)


def make_thermo(kind: int = QHP_THERMO_PILE, gamma0: float = 1.0, dt_fs: float = 0.5, n_seg: int = 1024,
                omega_cut_cm: float = 15000.0, a_gamma: float = 10.0, gamma_min_frac: float = 0.01,
                adapt: int = QHP_ADAPT_SIMPLE, tau_ratio_ps: float = 1.0,
                integrator: int = QHP_INTEGRATOR_BAOAB) -> qhp_thermo:
    return qhp_thermo(kind, gamma0, dt_fs, n_seg, omega_cut_cm, a_gamma, gamma_min_frac, adapt, tau_ratio_ps,
                      integrator)


class System:
    """Owns one qhp_sys handle (create, force field, beads, thermostat)."""

    def __init__(self, box, types, molecule, pos, precision, ff: qhp_ff, P, temperature, seed,
                 thermo: qhp_thermo | None = None):
        self.h = qhp_create_system(types, molecule, pos, box, precision)
        try:
            qhp_set_forcefield(self.h, ff)
            if thermo is not None and thermo.kind != QHP_THERMO_ADQTB:
                qhp_set_thermostat(self.h, thermo)
            qhp_set_beads(self.h, P, temperature, seed)
            if thermo is not None and thermo.kind == QHP_THERMO_ADQTB:
                qhp_set_thermostat(self.h, thermo)
        except Exception:
            qhp_destroy_system(self.h)
            raise
        self.n_atoms, self.P = len(types), P
        self.thermo = thermo
        self.ff = ff

    def set_params(self, theta) -> None:
        """Replace (eps, sigma, q_O, k_b, k_theta) of the force field."""
        self.ff = ff_with_params(self.ff, theta)
        qhp_set_forcefield(self.h, self.ff)

    @classmethod
    def from_config(cls, cfg, precision=None, **over):
        w = cfg.system()
        prec = {"fp64": QHP_FP64, "mixed": QHP_MIXED}[precision or cfg.precision]
        kind = QHP_THERMO_ADQTB if cfg.thermostat == "adqtb" else QHP_THERMO_PILE
        th = make_thermo(kind=kind, gamma0=cfg.gamma0, dt_fs=cfg.dt_fs, n_seg=cfg.n_seg,
                         omega_cut_cm=cfg.omega_cut_cm, a_gamma=cfg.a_gamma, gamma_min_frac=cfg.gamma_min_frac,
                         integrator=QHP_INTEGRATOR_BCOCB if cfg.extra.get("integrator") == "bcocb"
                         else QHP_INTEGRATOR_BAOAB)
        return cls(w.box, w.types, w.molecule, w.pos, prec, make_ff(cfg.rc, cfg.skin), cfg.P, cfg.temperature,
                   over.get("seed", cfg.seed), th)

    def close(self):
        if self.h is not None:
            qhp_destroy_system(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
