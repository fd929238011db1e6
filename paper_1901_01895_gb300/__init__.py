"""GB300 RK4IP propagator for the coupled multimode NLSE -- Python binding of libmmf.

The functions below carry the names of the C ABI in include/mmf.h and only
marshal arguments (ctypes); every step of the propagation runs in the CUDA
kernels of the library.  PyTorch is used by callers for device memory and
streams: pass ``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``.

Importing this module does not load the library; the first call does, and it
raises if the compiled library is missing (build it with
``python -m paper_1901_01895_gb300.build`` or ``__graft_entry__.build()``).
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmmf.so")

MMF_OK, MMF_EINVAL, MMF_ENOMEM, MMF_ECUDA, MMF_ETIMEOUT, MMF_EBUSY = 0, -1, -2, -3, -4, -5
MMF_KERR_FP32, MMF_KERR_BF16X3, MMF_KERR_BF16, MMF_KERR_TF32X3 = 0, 1, 2, 3
MMF_KERR_AUTO, MMF_KERR_LIST, MMF_KERR_PAIRS = 0 << 3, 1 << 3, 2 << 3
MMF_METHOD_RK4IP, MMF_METHOD_SSFM_RK4, MMF_METHOD_SSFM_AGRAWAL = 0 << 7, 1 << 7, 2 << 7
KERR_PATH_NAMES = {0: "list", 1: "pairs-simt", 3: "pairs-tcgen05", 4: "kappa", 5: "kappa-tcgen05"}

_lock = threading.Lock()
_lib = None

RQ_PENDING, RQ_RUNNING, RQ_DONE, RQ_FAILED = 0, 1, 2, 3


class MMFRequest(C.Structure):
    """mmf_request of include/mmf.h."""
    _fields_ = [("fiber", C.c_int), ("betas", C.POINTER(C.c_double)), ("alpha", C.c_double),
                ("N_t", C.c_int64), ("dt", C.c_double), ("L", C.c_double), ("n_steps", C.c_int),
                ("fields_in", C.c_void_p), ("fields_out", C.c_void_p)]


class MMFServerStats(C.Structure):
    """mmf_server_stats_t of include/mmf.h."""
    _fields_ = [("completed", C.c_uint64), ("failed", C.c_uint64), ("pending", C.c_uint64),
                ("running", C.c_int), ("peak_running", C.c_int), ("pools", C.c_int),
                ("bytes_in_use", C.c_size_t), ("field_sample_steps", C.c_double),
                ("graph_launches", C.c_uint64), ("kernel_launches", C.c_uint64)]


class MMFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mmf error {code}: {msg}")
        self.code = code


def lib() -> C.CDLL:
    """Load libmmf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1901_01895_gb300.build)")
        L = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        L.mmf_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, dp, C.POINTER(C.c_int32), dp, C.c_double,
                                 C.c_double, i64, C.c_double, C.c_uint, vp]
        L.mmf_create_kappa.argtypes = [C.POINTER(vp), C.c_int, dp, dp, C.c_double, C.c_double, i64, C.c_double,
                                       C.c_uint, vp]
        L.mmf_propagate.argtypes = [vp, vp, C.c_double, C.c_int]
        L.mmf_propagate_host.argtypes = [vp, vp, vp, C.c_double, C.c_int]
        L.mmf_energy.argtypes = [vp, vp, dp]
        L.mmf_kerr.argtypes = [vp, vp, vp, C.c_double]
        L.mmf_linear.argtypes = [vp, vp, vp, C.c_double]
        L.mmf_kerr_stage.argtypes = [vp, vp, vp, C.c_double, vp, C.c_double]
        L.mmf_linear_stage.argtypes = [vp, C.c_int, C.POINTER(vp), dp, vp, C.c_double, vp, C.c_double]
        L.mmf_amplify.argtypes = [vp, vp, C.c_double, vp]
        L.mmf_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(i64), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        L.mmf_destroy.argtypes = [vp]
        L.mmf_energy_noalloc.argtypes = [vp, C.c_int, i64, C.c_double, vp, vp]
        L.mmf_device_status.argtypes = [vp, C.POINTER(C.c_int)]
        L.mmf_last_error.restype = C.c_char_p
        u64 = C.c_uint64
        L.mmf_server_create.argtypes = [C.POINTER(vp), C.c_size_t, C.c_int]
        L.mmf_server_add_fiber.argtypes = [vp, C.c_int, C.c_int, dp, C.POINTER(C.c_int32), C.c_double, C.c_uint,
                                           C.POINTER(C.c_int)]
        L.mmf_server_submit.argtypes = [vp, C.POINTER(MMFRequest), C.POINTER(u64)]
        L.mmf_server_poll.argtypes = [vp, u64, C.POINTER(C.c_int), dp]
        L.mmf_server_wait.argtypes = [vp, u64, C.c_double, dp]
        L.mmf_server_release.argtypes = [vp, u64]
        L.mmf_server_stats.argtypes = [vp, C.POINTER(MMFServerStats)]
        L.mmf_server_destroy.argtypes = [vp]
        for name in ("mmf_create", "mmf_create_kappa", "mmf_propagate", "mmf_propagate_host", "mmf_energy", "mmf_kerr",
                     "mmf_linear", "mmf_kerr_stage", "mmf_linear_stage", "mmf_amplify", "mmf_info", "mmf_destroy", "mmf_energy_noalloc",
                     "mmf_device_status", "mmf_server_create", "mmf_server_add_fiber", "mmf_server_submit",
                     "mmf_server_poll", "mmf_server_wait", "mmf_server_release", "mmf_server_stats",
                     "mmf_server_destroy"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(rc: int) -> None:
    if rc != MMF_OK:
        raise MMFError(rc, lib().mmf_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---- the C ABI, one Python function per entry point ------------------------------

def mmf_create(n_modes: int, n_pol: int, S_plmn, parity_class, betas, alpha: float, gamma: float,
               N_t: int, dt: float, flags: int = 0, stream: int = 0) -> int:
    S = np.ascontiguousarray(S_plmn, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    if S.size != n_modes ** 4:
        raise ValueError("S_plmn must have n_modes^4 entries")
    if b.size != 4 * n_modes * n_pol:
        raise ValueError("betas must be [P][4]")
    par = None
    if parity_class is not None:
        par = np.ascontiguousarray(parity_class, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().mmf_create(C.byref(h), int(n_modes), int(n_pol), _dp(S),
                            par.ctypes.data_as(C.POINTER(C.c_int32)) if par is not None else None,
                            _dp(b), float(alpha), float(gamma), int(N_t), float(dt), int(flags),
                            C.c_void_p(int(stream))))
    return h.value


def mmf_create_kappa(n_fields: int, kappa, betas, alpha: float, gamma: float, N_t: int, dt: float,
                     flags: int = 0, stream: int = 0) -> int:
    K = np.ascontiguousarray(kappa, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    if K.shape != (n_fields, n_fields):
        raise ValueError("kappa must be [P][P]")
    if b.size != 4 * n_fields:
        raise ValueError("betas must be [P][4]")
    h = C.c_void_p()
    _check(lib().mmf_create_kappa(C.byref(h), int(n_fields), _dp(K), _dp(b), float(alpha), float(gamma), int(N_t),
                                  float(dt), int(flags), C.c_void_p(int(stream))))
    return h.value


def mmf_propagate(h: int, fields_ptr: int, L: float, n_steps: int) -> None:
    _check(lib().mmf_propagate(C.c_void_p(h), C.c_void_p(int(fields_ptr)), float(L), int(n_steps)))


def mmf_propagate_host(h: int, fields_in: np.ndarray, fields_out: np.ndarray, L: float, n_steps: int) -> None:
    for a in (fields_in, fields_out):
        if a.dtype != np.complex64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous complex64")
    _check(lib().mmf_propagate_host(C.c_void_p(h), C.c_void_p(fields_in.ctypes.data),
                                    C.c_void_p(fields_out.ctypes.data), float(L), int(n_steps)))


def mmf_energy(h: int, fields_ptr: int, P: int) -> np.ndarray:
    out = np.empty(P, dtype=np.float64)
    _check(lib().mmf_energy(C.c_void_p(h), C.c_void_p(int(fields_ptr)), _dp(out)))
    return out


def mmf_kerr(h: int, in_ptr: int, out_ptr: int, scale: float) -> None:
    _check(lib().mmf_kerr(C.c_void_p(h), C.c_void_p(int(in_ptr)), C.c_void_p(int(out_ptr)), float(scale)))


def mmf_linear(h: int, in_ptr: int, out_ptr: int, z: float) -> None:
    _check(lib().mmf_linear(C.c_void_p(h), C.c_void_p(int(in_ptr)), C.c_void_p(int(out_ptr)), float(z)))


def mmf_kerr_stage(h: int, in0_ptr: int, in1_ptr: int, c1: float, out_ptr: int, scale: float) -> None:
    """out = i * scale * gamma * Kerr(in0 + c1 * in1); in1_ptr may be 0."""
    _check(lib().mmf_kerr_stage(C.c_void_p(h), C.c_void_p(int(in0_ptr)), C.c_void_p(int(in1_ptr)) if in1_ptr else None,
                                float(c1), C.c_void_p(int(out_ptr)), float(scale)))


def mmf_linear_stage(h: int, in_ptrs, coefs, add_ptr: int, add_coef: float, out_ptr: int, z: float) -> None:
    """out = exp(z Lhat)[sum coefs[i] * in[i]] + add_coef * add; add_ptr may be 0."""
    n = len(in_ptrs)
    arr = (C.c_void_p * n)(*[C.c_void_p(int(p)) for p in in_ptrs])
    cf = np.ascontiguousarray(coefs, dtype=np.float64)
    if cf.size != n:
        raise ValueError("one coefficient per input")
    _check(lib().mmf_linear_stage(C.c_void_p(h), n, arr, _dp(cf), C.c_void_p(int(add_ptr)) if add_ptr else None,
                                  float(add_coef), C.c_void_p(int(out_ptr)), float(z)))


def mmf_amplify(h: int, fields_ptr: int, power_gain: float, noise_ptr: int = 0) -> None:
    _check(lib().mmf_amplify(C.c_void_p(h), C.c_void_p(int(fields_ptr)), float(power_gain),
                             C.c_void_p(int(noise_ptr)) if noise_ptr else None))


def mmf_info(h: int) -> dict:
    P, N, path, sb = C.c_int(), C.c_int64(), C.c_int(), C.c_size_t()
    _check(lib().mmf_info(C.c_void_p(h), C.byref(P), C.byref(N), C.byref(path), C.byref(sb)))
    return {"P": P.value, "N_t": N.value, "kerr_path": KERR_PATH_NAMES.get(path.value, str(path.value)),
            "scratch_bytes": sb.value}


def mmf_energy_noalloc(fields_ptr: int, P: int, N_t: int, dt: float, out_ptr: int, stream: int = 0) -> None:
    """Per-field energies into a device float64 [P] array without allocating device memory."""
    _check(lib().mmf_energy_noalloc(C.c_void_p(int(fields_ptr)), int(P), int(N_t), float(dt),
                                    C.c_void_p(int(out_ptr)), C.c_void_p(int(stream))))


def mmf_device_status(h: int) -> int:
    """Synchronise and return the device status word (raises MMFError if a device wait gave up)."""
    code = C.c_int(0)
    _check(lib().mmf_device_status(C.c_void_p(h), C.byref(code)))
    return code.value


def mmf_destroy(h: int) -> None:
    _check(lib().mmf_destroy(C.c_void_p(h)))


def mmf_last_error() -> str:
    return lib().mmf_last_error().decode()


# ---- request server ----------------------------------------------------------------

def mmf_server_create(hbm_budget_bytes: int = 0, max_slots: int = 0) -> int:
    s = C.c_void_p()
    _check(lib().mmf_server_create(C.byref(s), int(hbm_budget_bytes), int(max_slots)))
    return s.value


def mmf_server_add_fiber(s: int, n_modes: int, n_pol: int, S_plmn, parity_class, gamma: float,
                         flags: int = 0) -> int:
    S = np.ascontiguousarray(S_plmn, dtype=np.float64)
    if S.size != n_modes ** 4:
        raise ValueError("S_plmn must have n_modes^4 entries")
    par = None if parity_class is None else np.ascontiguousarray(parity_class, dtype=np.int32)
    fid = C.c_int()
    _check(lib().mmf_server_add_fiber(C.c_void_p(s), int(n_modes), int(n_pol), _dp(S),
                                      par.ctypes.data_as(C.POINTER(C.c_int32)) if par is not None else None,
                                      float(gamma), int(flags), C.byref(fid)))
    return fid.value


def mmf_server_submit(s: int, fiber: int, betas, alpha: float, N_t: int, dt: float, L: float, n_steps: int,
                      in_ptr: int, out_ptr: int) -> int:
    """Queue one request; in_ptr/out_ptr are host (pinned or pageable) or device addresses."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    req = MMFRequest(int(fiber), _dp(b), float(alpha), int(N_t), float(dt), float(L), int(n_steps),
                     C.c_void_p(int(in_ptr)), C.c_void_p(int(out_ptr)))
    rid = C.c_uint64()
    _check(lib().mmf_server_submit(C.c_void_p(s), C.byref(req), C.byref(rid)))
    return rid.value


def mmf_server_poll(s: int, rid: int) -> tuple[int, float]:
    """(state, latency_ms); raises MMFError for a failed request."""
    st, lat = C.c_int(), C.c_double()
    _check(lib().mmf_server_poll(C.c_void_p(s), C.c_uint64(rid), C.byref(st), C.byref(lat)))
    return st.value, lat.value


def mmf_server_wait(s: int, rid: int, timeout_s: float = -1.0) -> float:
    """Block until the request finishes; returns its latency in ms."""
    lat = C.c_double()
    _check(lib().mmf_server_wait(C.c_void_p(s), C.c_uint64(rid), float(timeout_s), C.byref(lat)))
    return lat.value


def mmf_server_release(s: int, rid: int) -> None:
    _check(lib().mmf_server_release(C.c_void_p(s), C.c_uint64(rid)))


def mmf_server_stats(s: int) -> dict:
    st = MMFServerStats()
    _check(lib().mmf_server_stats(C.c_void_p(s), C.byref(st)))
    return {k: getattr(st, k) for k, _ in MMFServerStats._fields_}


def mmf_server_destroy(s: int) -> None:
    _check(lib().mmf_server_destroy(C.c_void_p(s)))


class Fiber:
    """Owns one handle; a convenience wrapper over the functions above."""

    def __init__(self, n_modes, n_pol, S_plmn, parity_class, betas, alpha, gamma, N_t, dt, flags=0, stream=0):
        self.P = n_modes * n_pol
        self.N_t = N_t
        self.handle = mmf_create(n_modes, n_pol, S_plmn, parity_class, betas, alpha, gamma, N_t, dt, flags, stream)

    @classmethod
    def from_kappa(cls, kappa, betas, alpha, gamma, N_t, dt, flags=0, stream=0) -> "Fiber":
        """A handle whose Kerr term is the kappa form of Eq. 1 (mmf_create_kappa)."""
        self = cls.__new__(cls)
        self.P = int(np.asarray(kappa).shape[0])
        self.N_t = N_t
        self.handle = mmf_create_kappa(self.P, kappa, betas, alpha, gamma, N_t, dt, flags, stream)
        return self

    @classmethod
    def from_workload(cls, wl, flags: int = 0, stream: int = 0) -> "Fiber":
        return cls(wl.n_modes, wl.n_pol, wl.S, wl.parity, wl.betas, wl.alpha, wl.gamma, wl.N_t, wl.dt, flags, stream)

    def propagate(self, fields_ptr: int, L: float, n_steps: int) -> None:
        mmf_propagate(self.handle, fields_ptr, L, n_steps)

    def propagate_host(self, fields_in: np.ndarray, fields_out: np.ndarray, L: float, n_steps: int) -> None:
        mmf_propagate_host(self.handle, fields_in, fields_out, L, n_steps)

    def energy(self, fields_ptr: int) -> np.ndarray:
        return mmf_energy(self.handle, fields_ptr, self.P)

    def kerr(self, in_ptr: int, out_ptr: int, scale: float) -> None:
        mmf_kerr(self.handle, in_ptr, out_ptr, scale)

    def linear(self, in_ptr: int, out_ptr: int, z: float) -> None:
        mmf_linear(self.handle, in_ptr, out_ptr, z)

    def kerr_stage(self, in0_ptr: int, in1_ptr: int, c1: float, out_ptr: int, scale: float) -> None:
        mmf_kerr_stage(self.handle, in0_ptr, in1_ptr, c1, out_ptr, scale)

    def linear_stage(self, in_ptrs, coefs, add_ptr: int, add_coef: float, out_ptr: int, z: float) -> None:
        mmf_linear_stage(self.handle, in_ptrs, coefs, add_ptr, add_coef, out_ptr, z)

    def amplify(self, fields_ptr: int, power_gain: float, noise_ptr: int = 0) -> None:
        mmf_amplify(self.handle, fields_ptr, power_gain, noise_ptr)

    def info(self) -> dict:
        return mmf_info(self.handle)

    def device_status(self) -> int:
        return mmf_device_status(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            mmf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Owns one request server; a convenience wrapper over the mmf_server_* functions.

    Host buffers handed to submit() must stay alive until the request is done; the
    wrapper keeps a reference to them until then.
    """

    def __init__(self, hbm_budget_bytes: int = 0, max_slots: int = 0):
        self.handle = mmf_server_create(hbm_budget_bytes, max_slots)
        self._keep = {}

    def add_fiber(self, n_modes, n_pol, S_plmn, parity_class, gamma, flags=0) -> int:
        return mmf_server_add_fiber(self.handle, n_modes, n_pol, S_plmn, parity_class, gamma, flags)

    def submit(self, fiber, betas, alpha, N_t, dt, L, n_steps, fields_in, fields_out) -> int:
        """fields_in/fields_out: complex64 numpy arrays (host) or integer device addresses."""
        def addr(a):
            if isinstance(a, np.ndarray):
                if a.dtype != np.complex64 or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("host buffers must be C-contiguous complex64")
                return a.ctypes.data
            return int(a)
        rid = mmf_server_submit(self.handle, fiber, betas, alpha, N_t, dt, L, n_steps, addr(fields_in),
                                addr(fields_out))
        self._keep[rid] = (fields_in, fields_out)
        return rid

    def poll(self, rid) -> tuple[int, float]:
        return mmf_server_poll(self.handle, rid)

    def wait(self, rid, timeout_s: float = -1.0) -> float:
        return mmf_server_wait(self.handle, rid, timeout_s)

    def release(self, rid) -> None:
        mmf_server_release(self.handle, rid)
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        return mmf_server_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            mmf_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
