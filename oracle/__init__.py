"""FP64 CPU oracle for the RK4IP step of the coupled multimode NLSE (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark; the CUDA path never imports it and it never
imports the CUDA path.  The arithmetic lives in rk4ip.c (plain C, FP64); this
file only compiles it with gcc and marshals numpy arrays.

Every function follows the paper's equations: Eq. 1 (the linear operator and the
Kerr term, the latter in overlap-tensor form) and Eq. 4a-4f (the RK4IP step).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rk4ip.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rk4ip.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP, IEEE FP64)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp, cp, i64 = C.POINTER(C.c_double), C.c_void_p, C.c_int64
        lib.orc_fft.argtypes = [cp, i64, C.c_int]
        lib.orc_lin.argtypes = [C.c_int, i64, C.c_double, dp, C.c_double, C.c_double, cp, cp]
        lib.orc_kerr_build.argtypes = [C.c_int, C.c_int, dp]
        lib.orc_kerr_build.restype = C.c_void_p
        lib.orc_kerr_free.argtypes = [C.c_void_p]
        lib.orc_kerr_nnz.argtypes = [C.c_void_p]
        lib.orc_kerr_nnz.restype = i64
        lib.orc_kerr.argtypes = [C.c_void_p, i64, C.c_double, cp, cp]
        lib.orc_kerr_at.argtypes = [C.c_void_p, i64, C.c_double, cp, C.POINTER(C.c_int64), i64, cp]
        lib.orc_kerr_dense.argtypes = [C.c_int, C.c_int, dp, i64, C.c_double, cp, cp]
        lib.orc_propagate.argtypes = [C.c_int, C.c_int, dp, dp, C.c_double, C.c_double, i64,
                                      C.c_double, cp, C.c_double, C.c_int]
        lib.orc_energy.argtypes = [C.c_int, i64, C.c_double, cp, dp]
        lib.orc_kerr_kappa.argtypes = [C.c_int, i64, dp, C.c_double, cp, cp]
        lib.orc_propagate_method.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_double, C.c_double, i64,
                                             C.c_double, cp, C.c_double, C.c_int]
        lib.orc_propagate_kappa.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, i64, C.c_double, cp,
                                            C.c_double, C.c_int]
        lib.orc_num_threads.restype = C.c_int
        lib.orc_set_num_threads.argtypes = [C.c_int]
        _lib = lib
        return lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def fft(x, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT of one row (sign -1 forward, +1 inverse without 1/N)."""
    y = _c128(x).copy()
    if _load().orc_fft(y.ctypes.data, y.size, int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return y


def lin(fields, betas, alpha: float, dt: float, z: float) -> np.ndarray:
    """exp(z * Lhat) applied to every field (Eq. 1 linear part, exact in the frequency domain)."""
    A = _c128(fields)
    P, Nt = A.shape
    b = _f64(betas).reshape(P, 4)
    out = np.empty_like(A)
    if _load().orc_lin(P, Nt, dt, _dp(b), alpha, z, A.ctypes.data, out.ctypes.data) != 0:
        raise ValueError("orc_lin failed")
    return out


class KerrList:
    """Nonzero entries of the spatial overlap tensor S; evaluates the Kerr term of Eq. 1."""

    def __init__(self, S, n_pol: int):
        S = _f64(S)
        M = S.shape[0]
        self.M, self.n_pol = M, n_pol
        self._S = S
        self._h = _load().orc_kerr_build(M, n_pol, _dp(S))
        if not self._h:
            raise MemoryError("orc_kerr_build failed")

    @property
    def nnz(self) -> int:
        return _load().orc_kerr_nnz(self._h)

    def __call__(self, fields, scale: float) -> np.ndarray:
        """i * scale * sum Sfull A_l A_m conj(A_n) at every sample."""
        A = _c128(fields)
        out = np.empty_like(A)
        if _load().orc_kerr(self._h, A.shape[1], scale, A.ctypes.data, out.ctypes.data) != 0:
            raise MemoryError("orc_kerr failed")
        return out

    def at(self, fields, scale: float, samples) -> np.ndarray:
        """Kerr term at the given sample indices only -> [P, len(samples)]."""
        A = _c128(fields)
        s = np.ascontiguousarray(samples, dtype=np.int64)
        out = np.empty((A.shape[0], s.size), dtype=np.complex128)
        if _load().orc_kerr_at(self._h, A.shape[1], scale, A.ctypes.data,
                               s.ctypes.data_as(C.POINTER(C.c_int64)), s.size, out.ctypes.data) != 0:
            raise MemoryError("orc_kerr_at failed")
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_kerr_free(h)
            self._h = None


def kerr_dense(S, n_pol: int, fields, scale: float) -> np.ndarray:
    """Brute-force Kerr term over all P^4 index combinations (small P only)."""
    S = _f64(S)
    A = _c128(fields)
    out = np.empty_like(A)
    _load().orc_kerr_dense(S.shape[0], n_pol, _dp(S), A.shape[1], scale, A.ctypes.data, out.ctypes.data)
    return out


METHODS = {"rk4ip": 0, "ssfm-rk4": 1, "ssfm-agrawal": 2}


def propagate(S, n_pol: int, betas, alpha: float, gamma: float, dt: float, fields,
              L: float, n_steps: int, method: str = "rk4ip") -> np.ndarray:
    """RK4IP (Eq. 4) -- or SSFM-RK4 (Section 3.1) -- over length L in n_steps fixed steps."""
    S = _f64(S)
    A = _c128(fields).copy()
    P, Nt = A.shape
    b = _f64(betas).reshape(P, 4)
    if method != "rk4ip":
        rc = _load().orc_propagate_method(METHODS[method], S.shape[0], n_pol, _dp(S), None, _dp(b), alpha, gamma,
                                          Nt, dt, A.ctypes.data, L, int(n_steps))
        if rc != 0:
            raise ValueError("orc_propagate_method failed")
        return A
    rc = _load().orc_propagate(S.shape[0], n_pol, _dp(S), _dp(b), alpha, gamma, Nt, dt,
                               A.ctypes.data, L, int(n_steps))
    if rc != 0:
        raise ValueError("orc_propagate failed")
    return A


def propagate_workload(wl, n_steps: int | None = None, L: float | None = None) -> np.ndarray:
    """Convenience: propagate a workloads.Workload (optionally fewer steps / shorter L)."""
    n = wl.n_steps if n_steps is None else n_steps
    length = wl.L if L is None else L
    return propagate(wl.S, wl.n_pol, wl.betas, wl.alpha, wl.gamma, wl.dt, wl.fields, length, n)


def kerr_kappa(kappa, fields, scale: float) -> np.ndarray:
    """Kappa form of Eq. 1's Kerr term: i * scale * (sum_g kappa_fg |A_g|^2) A_f at every sample."""
    K = _f64(kappa)
    A = _c128(fields)
    P, Nt = A.shape
    if K.shape != (P, P):
        raise ValueError("kappa must be [P, P]")
    out = np.empty_like(A)
    if _load().orc_kerr_kappa(P, Nt, _dp(K), scale, A.ctypes.data, out.ctypes.data) != 0:
        raise MemoryError("orc_kerr_kappa failed")
    return out


def propagate_kappa(kappa, betas, alpha: float, gamma: float, dt: float, fields, L: float,
                    n_steps: int, method: str = "rk4ip") -> np.ndarray:
    """RK4IP (Eq. 4) -- or SSFM-RK4 -- with the kappa form of Eq. 1's Kerr term."""
    K = _f64(kappa)
    A = _c128(fields).copy()
    P, Nt = A.shape
    b = _f64(betas).reshape(P, 4)
    if method != "rk4ip":
        rc = _load().orc_propagate_method(METHODS[method], P, 1, None, _dp(K), _dp(b), alpha, gamma, Nt, dt,
                                          A.ctypes.data, L, int(n_steps))
    else:
        rc = _load().orc_propagate_kappa(P, _dp(K), _dp(b), alpha, gamma, Nt, dt, A.ctypes.data, L, int(n_steps))
    if rc != 0:
        raise ValueError("orc_propagate_kappa failed")
    return A


def energy(fields, dt: float) -> np.ndarray:
    A = _c128(fields)
    out = np.empty(A.shape[0])
    _load().orc_energy(A.shape[0], A.shape[1], dt, A.ctypes.data, _dp(out))
    return out
