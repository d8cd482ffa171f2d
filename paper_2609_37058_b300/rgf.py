"""ctypes binding of the C ABI in include/rgf.h (argument marshalling only).

Every function below has the name of the C entry point it calls and does no
arithmetic of its own: it turns numpy arrays (host memory) or torch tensors
(device memory) into pointers and raises ``RGFError`` on a non-OK status.
The compiled library ``librgf.so`` must exist next to this file; there is no
fallback when it does not.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# RGF_DEBUG_LIB=1 in the environment loads the debug build (device-side
# index checks, see rgf_debug_flags in include/rgf_kernels.h).
LIB_PATH = os.path.join(HERE, "librgf_debug.so" if os.environ.get("RGF_DEBUG_LIB") == "1" else "librgf.so")

RGF_OK, RGF_E_INVALID, RGF_E_OOM, RGF_E_CUDA, RGF_E_NOT_READY, RGF_E_NOCONV, RGF_E_TIMEOUT, \
    RGF_E_REJECTED, RGF_E_STATE = range(9)
STATUS_NAMES = ["RGF_OK", "RGF_E_INVALID", "RGF_E_OOM", "RGF_E_CUDA", "RGF_E_NOT_READY",
                "RGF_E_NOCONV", "RGF_E_TIMEOUT", "RGF_E_REJECTED", "RGF_E_STATE"]
RGF_FP64, RGF_MIXED = 0, 1
RGF_MEM_HOST, RGF_MEM_DEVICE = 0, 1
RGF_LEAD_LEFT, RGF_LEAD_RIGHT = 0, 1
RGF_FLAG_NOCONV_L, RGF_FLAG_NOCONV_R, RGF_FLAG_SINGULAR, RGF_FLAG_REFINE, RGF_FLAG_LEAD_NEWTON = 1, 2, 4, 8, 16


class RGFError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")


class rgf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eta", ctypes.c_double), ("dec_tol", ctypes.c_double),
                ("dec_max_iter", ctypes.c_int), ("ns_steps", ctypes.c_int),
                ("energy_wave", ctypes.c_int)]


class rgf_server_options(ctypes.Structure):
    _fields_ = [("dec_tol", ctypes.c_double), ("dec_max_iter", ctypes.c_int), ("ns_steps", ctypes.c_int),
                ("slots", ctypes.c_int), ("class_step", ctypes.c_int), ("capacity_bytes", ctypes.c_size_t)]


class rgf_request(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("b", ctypes.c_int), ("eta", ctypes.c_double),
                ("H_diag", ctypes.c_void_p), ("S_diag", ctypes.c_void_p), ("H_lower", ctypes.c_void_p),
                ("S_lower", ctypes.c_void_p), ("lead", (ctypes.c_void_p * 6) * 2), ("E", ctypes.c_void_p),
                ("n_E", ctypes.c_int), ("mem", ctypes.c_int)]


class rgf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("energies_done", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("decimations", ctypes.c_longlong),
                ("fp64_reseeds", ctypes.c_longlong), ("engines", ctypes.c_int),
                ("resident_bytes", ctypes.c_size_t), ("peak_resident_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("busy_s", ctypes.c_double),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load librgf.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_37058_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "rgf_options_default": (None, [ctypes.POINTER(rgf_options)]),
        "rgf_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(rgf_options), _P]),
        "rgf_set_device_blocks": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
        "rgf_set_leads": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
        "rgf_transmission": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int]),
        "rgf_submit": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
        "rgf_poll": (ctypes.c_int, [ctypes.c_uint64, _P, _P, _P, ctypes.c_int]),
        "rgf_plan_device_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
        "rgf_plan_energy_wave": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
        "rgf_plan_destroy": (ctypes.c_int, [_P]),
        "rgf_last_error": (ctypes.c_char_p, []),
        "rgf_version": (ctypes.c_char_p, []),
        "rgf_kernel_zgemm_f64": (ctypes.c_int, [ctypes.c_int] * 4 + [_P, _P, _P]),
        "rgf_kernel_inverse_f64": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P]),
        "rgf_kernel_inverse_c64": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P]),
        "rgf_kernel_zgemm_mixed": (ctypes.c_int, [ctypes.c_int] * 4 + [_P, _P, _P, ctypes.c_int]),
        "rgf_launch_count": (ctypes.c_ulonglong, []),
        "rgf_debug_build": (ctypes.c_int, []),
        "rgf_debug_flags": (ctypes.c_uint, []),
        "rgf_kernel_zgemm_hp": (ctypes.c_int, [ctypes.c_int] * 4 + [_P, _P, _P]),
        "rgf_kernel_zgemm_slices": (ctypes.c_int, [ctypes.c_int] * 4 + [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
        "rgf_kernel_tc_timeout_probe": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "rgf_inverse_f64_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P]),
        "rgf_inverse_f64_noalloc_limit": (ctypes.c_size_t, []),
        "rgf_plan_stats": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_longlong)] * 2),
        "rgf_plan_phase_ms": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_double)] * 2),
        "rgf_peak_fma": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]),
        "rgf_gemm_timing": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
        "rgf_server_options_default": (None, [ctypes.POINTER(rgf_server_options)]),
        "rgf_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(rgf_server_options)]),
        "rgf_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(rgf_request), ctypes.POINTER(ctypes.c_uint64)]),
        "rgf_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int]),
        "rgf_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(rgf_server_stats)]),
        "rgf_server_destroy": (ctypes.c_int, [_P]),
        "rgf_server_set_class": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "rgf_bloch_sum": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
        "rgf_kmesh_mean": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
        "rgf_kmesh_transmission": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_int, _P, _P, _P]),
        "rgf_current": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_double,
                                       _P, _P]),
        "rgf_ldos": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int]),
        "rgf_kpm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                          ctypes.c_int, _P]),
        "rgf_kpm_scale": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, _D, _D]),
        "rgf_kpm_moments": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int, _P, ctypes.c_int,
                                           _P]),
        "rgf_kpm_fermi": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _P, _P]),
        "rgf_kpm_destroy": (ctypes.c_int, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status, where):
    if status != RGF_OK:
        raise RGFError(status, where, rgf_last_error())


def _ptr(x, dtype):
    """(pointer, memspace) for a numpy array (host) or torch tensor (device)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data, RGF_MEM_HOST
    import torch  # device memory comes from torch tensors
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected numpy array or torch tensor")
    tmap = {np.complex128: torch.complex128, np.float64: torch.float64, np.int32: torch.int32}
    if x.dtype != tmap[dtype] or not x.is_contiguous():
        raise TypeError(f"expected a contiguous {tmap[dtype]} tensor")
    return x.data_ptr(), (RGF_MEM_DEVICE if x.is_cuda else RGF_MEM_HOST)


def _mem_of(*ptrs):
    spaces = {m for _, m in ptrs if m is not None}
    if len(spaces) > 1:
        raise TypeError("all arrays of one call must live in the same memory space")
    return spaces.pop() if spaces else RGF_MEM_HOST


# ----------------------------------------------------------------- C entry points
def rgf_version() -> str:
    return lib().rgf_version().decode()


def rgf_last_error() -> str:
    return lib().rgf_last_error().decode(errors="replace")


def rgf_options_default() -> rgf_options:
    o = rgf_options()
    lib().rgf_options_default(ctypes.byref(o))
    return o


def rgf_plan_create(n_layers: int, b: int, opt: rgf_options | None = None, cuda_stream: int = 0):
    h = _P()
    s = lib().rgf_plan_create(ctypes.byref(h), int(n_layers), int(b),
                              ctypes.byref(opt) if opt is not None else None,
                              _P(cuda_stream) if cuda_stream else None)
    _check(s, "rgf_plan_create")
    return h


def rgf_set_device_blocks(plan, H_diag, S_diag, H_lower, S_lower):
    ps = [_ptr(a, np.complex128) for a in (H_diag, S_diag, H_lower, S_lower)]
    mem = _mem_of(*ps)
    _check(lib().rgf_set_device_blocks(plan, *[p for p, _ in ps], mem), "rgf_set_device_blocks")


def rgf_set_leads(plan, side, H00, S00, H10, S10, Hc, Sc):
    ps = [_ptr(a, np.complex128) for a in (H00, S00, H10, S10, Hc, Sc)]
    mem = _mem_of(*ps)
    _check(lib().rgf_set_leads(plan, int(side), *[p for p, _ in ps], mem), "rgf_set_leads")


def rgf_transmission(plan, E, T, err=None, flags=None):
    pe, pt = _ptr(E, np.float64), _ptr(T, np.float64)
    pr, pf = _ptr(err, np.float64), _ptr(flags, np.int32)
    mem = _mem_of(pe, pt, pr, pf)
    n = int(E.shape[0])
    _check(lib().rgf_transmission(plan, pe[0], n, pt[0], pr[0], pf[0], mem), "rgf_transmission")


def rgf_submit(plan, E: np.ndarray) -> int:
    pe = _ptr(E, np.float64)
    if pe[1] != RGF_MEM_HOST:
        raise TypeError("rgf_submit takes host energies")
    t = ctypes.c_uint64()
    _check(lib().rgf_submit(plan, pe[0], int(E.shape[0]), ctypes.byref(t)), "rgf_submit")
    return t.value


def rgf_poll(ticket: int, T, err=None, flags=None, timeout_us: int = -1) -> int:
    """Returns the status (RGF_OK, RGF_E_NOT_READY, RGF_E_TIMEOUT); raises on errors."""
    pt, pr, pf = _ptr(T, np.float64), _ptr(err, np.float64), _ptr(flags, np.int32)
    s = lib().rgf_poll(ctypes.c_uint64(ticket), pt[0], pr[0], pf[0], int(timeout_us))
    if s in (RGF_OK, RGF_E_NOT_READY, RGF_E_TIMEOUT):
        return s
    _check(s, "rgf_poll")
    return s


def rgf_plan_device_bytes(plan) -> int:
    v = ctypes.c_size_t()
    _check(lib().rgf_plan_device_bytes(plan, ctypes.byref(v)), "rgf_plan_device_bytes")
    return v.value


def rgf_plan_energy_wave(plan) -> int:
    v = ctypes.c_int()
    _check(lib().rgf_plan_energy_wave(plan, ctypes.byref(v)), "rgf_plan_energy_wave")
    return v.value


def rgf_plan_stats(plan):
    """(waves, fp64_reseeds) counted since the plan was created."""
    w, r = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().rgf_plan_stats(plan, ctypes.byref(w), ctypes.byref(r)), "rgf_plan_stats")
    return w.value, r.value


def rgf_plan_phase_ms(plan):
    """(lead_ms, sweep_ms) of the mixed path since the plan's creation."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().rgf_plan_phase_ms(plan, ctypes.byref(a), ctypes.byref(b)), "rgf_plan_phase_ms")
    return a.value, b.value


def rgf_plan_destroy(plan):
    if plan:
        _check(lib().rgf_plan_destroy(plan), "rgf_plan_destroy")


# ----------------------------------------------------------------- kernel-level calls
def _host(a, dtype):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} host array")
    return a.ctypes.data


def rgf_kernel_zgemm_f64(A, B):
    """C[i] = A[i] B[i] for complex128 arrays of shape (batch, m, k), (batch, k, n)."""
    batch, m, k = A.shape
    n = B.shape[2]
    C = np.empty((batch, m, n), dtype=np.complex128)
    _check(lib().rgf_kernel_zgemm_f64(batch, m, n, k, _host(A, np.complex128), _host(B, np.complex128),
                                      C.ctypes.data), "rgf_kernel_zgemm_f64")
    return C


def rgf_kernel_zgemm_mixed(A, B, core=0):
    batch, m, k = A.shape
    n = B.shape[2]
    C = np.empty((batch, m, n), dtype=np.complex128)
    _check(lib().rgf_kernel_zgemm_mixed(batch, m, n, k, _host(A, np.complex128), _host(B, np.complex128),
                                        C.ctypes.data, int(core)), "rgf_kernel_zgemm_mixed")
    return C


def rgf_kernel_zgemm_hp(A, B):
    """C[i] = A[i] B[i] with the seven-slice (FP64-class) tensor-core GEMM."""
    batch, m, k = A.shape
    n = B.shape[2]
    C = np.empty((batch, m, n), dtype=np.complex128)
    _check(lib().rgf_kernel_zgemm_hp(batch, m, n, k, _host(A, np.complex128), _host(B, np.complex128),
                                     C.ctypes.data), "rgf_kernel_zgemm_hp")
    return C


def rgf_kernel_zgemm_slices(A, B, fp64_operands, nsl):
    """C[i] = A[i] B[i] with nsl slices per operand (see the header)."""
    batch, m, k = A.shape
    n = B.shape[2]
    C = np.empty((batch, m, n), dtype=np.complex128)
    _check(lib().rgf_kernel_zgemm_slices(batch, m, n, k, _host(A, np.complex128), _host(B, np.complex128),
                                         C.ctypes.data, int(bool(fp64_operands)), int(nsl)),
           "rgf_kernel_zgemm_slices")
    return C


def rgf_kernel_tc_timeout_probe(wait_us=20000):
    """Returns (status, status_bits) of the bounded-wait probe (see header)."""
    bits = ctypes.c_int(0)
    st = lib().rgf_kernel_tc_timeout_probe(int(wait_us), ctypes.byref(bits))
    return st, bits.value


def rgf_kernel_inverse_f64(A):
    """Inverse of each complex128 (b x b) matrix of A (batch, b, b); returns (inv, flags)."""
    X = np.ascontiguousarray(A, dtype=np.complex128).copy()
    flags = np.zeros(X.shape[0], dtype=np.int32)
    _check(lib().rgf_kernel_inverse_f64(X.shape[0], X.shape[1], X.ctypes.data, flags.ctypes.data),
           "rgf_kernel_inverse_f64")
    return X, flags


def rgf_kernel_inverse_c64(A):
    X = np.ascontiguousarray(A, dtype=np.complex64).copy()
    flags = np.zeros(X.shape[0], dtype=np.int32)
    _check(lib().rgf_kernel_inverse_c64(X.shape[0], X.shape[1], X.ctypes.data, flags.ctypes.data),
           "rgf_kernel_inverse_c64")
    return X, flags


def rgf_inverse_f64_noalloc(A, flags=None, cuda_stream=None):
    """In-place FP64 inverses of the complex128 CUDA tensor A (batch, b, b)
    with the library's fixed scratch array (no device allocation); flags is
    an int32 CUDA tensor of at least batch entries or None.  cuda_stream is a
    torch.cuda.Stream on A's device, a raw cudaStream_t handle (int, taken to
    be on A's device) or None (the legacy default stream).  Asynchronous on
    the stream; the call runs with A's device current."""
    import torch
    if not (torch.is_tensor(A) and A.is_cuda and A.dtype == torch.complex128 and A.dim() == 3
            and A.shape[1] == A.shape[2] and A.is_contiguous()):
        raise TypeError("rgf_inverse_f64_noalloc: A must be a contiguous complex128 CUDA tensor (batch, b, b)")
    batch, b = int(A.shape[0]), int(A.shape[1])
    if flags is not None:
        if not (torch.is_tensor(flags) and flags.is_cuda and flags.dtype == torch.int32 and flags.is_contiguous()):
            raise TypeError("rgf_inverse_f64_noalloc: flags must be a contiguous int32 CUDA tensor")
        if flags.device != A.device:
            raise ValueError("rgf_inverse_f64_noalloc: flags and A are on different devices")
        if flags.numel() < batch:
            raise ValueError(f"rgf_inverse_f64_noalloc: flags has {flags.numel()} entries, need {batch}")
    handle = None
    if isinstance(cuda_stream, torch.cuda.Stream):
        if cuda_stream.device != A.device:
            raise ValueError("rgf_inverse_f64_noalloc: the stream belongs to another device than A")
        handle = cuda_stream.cuda_stream
    elif cuda_stream:
        handle = int(cuda_stream)
    with torch.cuda.device(A.device):
        _check(lib().rgf_inverse_f64_noalloc(batch, b, _P(A.data_ptr()),
                                             _P(flags.data_ptr()) if flags is not None else None,
                                             _P(handle) if handle else None),
               "rgf_inverse_f64_noalloc")


def rgf_inverse_f64_noalloc_limit() -> int:
    return int(lib().rgf_inverse_f64_noalloc_limit())


def rgf_launch_count() -> int:
    return int(lib().rgf_launch_count())


def rgf_peak_fma(kind: int, blocks_per_sm: int = 8, iters: int = 1 << 16):
    """(TFLOP/s, ms) of the library's FMA-loop probe: kind 0 = FP64, 1 = FP32."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().rgf_peak_fma(kind, blocks_per_sm, iters, ctypes.byref(tf), ctypes.byref(ms)), "rgf_peak_fma")
    return tf.value, ms.value


def rgf_gemm_timing(enable: bool):
    """Returns (total_ms, launches, flops) recorded since the last call and
    sets recording on/off for what follows."""
    ms, n, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(lib().rgf_gemm_timing(int(bool(enable)), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)),
           "rgf_gemm_timing")
    return ms.value, n.value, fl.value


# ----------------------------------------------------------------- server (include/rgf_server.h)
def rgf_server_options_default() -> rgf_server_options:
    o = rgf_server_options()
    lib().rgf_server_options_default(ctypes.byref(o))
    return o


def rgf_server_create(opt: rgf_server_options | None = None):
    h = _P()
    _check(lib().rgf_server_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None),
           "rgf_server_create")
    return h


def rgf_server_set_class(server, block_class: int, slots: int = 0, tile_n: int = 0, panel: int = 0):
    _check(lib().rgf_server_set_class(server, int(block_class), int(slots), int(tile_n), int(panel)),
           "rgf_server_set_class")


def rgf_server_submit(server, req: rgf_request) -> int:
    t = ctypes.c_uint64()
    _check(lib().rgf_server_submit(server, ctypes.byref(req), ctypes.byref(t)), "rgf_server_submit")
    return t.value


def rgf_server_poll(server, ticket: int, T, err=None, flags=None, timeout_us: int = -1):
    """Returns (status, latency_ms); raises on errors other than not-ready/timeout."""
    pt, mt = _ptr(T, np.float64)
    pe, me = _ptr(err, np.float64)
    pf, mf = _ptr(flags, np.int32)
    lat = ctypes.c_double(0.0)
    st = lib().rgf_server_poll(server, int(ticket), pt, pe, pf, ctypes.byref(lat), int(timeout_us))
    if st in (RGF_E_NOT_READY, RGF_E_TIMEOUT):
        return st, None
    _check(st, "rgf_server_poll")
    return st, lat.value


def rgf_server_stats_get(server) -> dict:
    s = rgf_server_stats()
    _check(lib().rgf_server_stats_get(server, ctypes.byref(s)), "rgf_server_stats_get")
    return {name: getattr(s, name) for name, _ in s._fields_}


def rgf_server_destroy(server):
    if server:
        _check(lib().rgf_server_destroy(server), "rgf_server_destroy")


TUNING_PATH = os.path.join(HERE, "tuning_b300.json")


def tuning_path() -> str:
    """The tuning table to load: $RGF_TUNE_CACHE when set (a table written by
    ``autotune --out``), else the one shipped with the package."""
    return os.environ.get("RGF_TUNE_CACHE") or TUNING_PATH


def load_tuning(path: str = None) -> dict:
    """Per-class settings written by ``autotune`` ({} when the file is absent)."""
    import json
    path = path or tuning_path()
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return {int(k): v for k, v in json.load(f)["classes"].items()}


class Server:
    """Owns one rgf_server_t.  ``submit(dev, E, eta)`` takes a device
    description (as ``Plan.set_device``) and keeps its arrays alive until the
    ticket is polled; ``poll`` returns (T, err, flags, latency_ms)."""

    def __init__(self, slots=148, class_step=32, capacity_bytes=0, ns_steps=6, dec_tol=1e-14,
                 dec_max_iter=100, tuning=None):
        """``tuning``: {block_class: {"slots", "tile_n", "panel"}} (as written
        by ``autotune``), "default" for the table at $RGF_TUNE_CACHE (else the
        one shipped with the package), or None."""
        o = rgf_server_options_default()
        o.slots, o.class_step, o.capacity_bytes = slots, class_step, capacity_bytes
        o.ns_steps, o.dec_tol, o.dec_max_iter = ns_steps, dec_tol, dec_max_iter
        self.handle = rgf_server_create(o)
        self._keep = {}
        if tuning == "default":
            tuning = load_tuning()
        for bc, cfg in (tuning or {}).items():
            rgf_server_set_class(self.handle, int(bc), cfg.get("slots", 0), cfg.get("tile_n", 0),
                                 cfg.get("panel", 0))

    def submit(self, dev, E, eta) -> int:
        """Queue one device.  Host devices (numpy arrays) are read from host
        memory; devices whose arrays are CUDA tensors (synth.gpu_devices) are
        read in place from device memory (synchronise their producer first)."""
        N, b = int(dev.H_diag.shape[0]), int(dev.H_diag.shape[1])
        on_gpu = hasattr(dev.H_diag, "data_ptr")
        if on_gpu:
            import torch
            chk = lambda t: t if (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()) else None
            arrs = {"H_diag": chk(dev.H_diag), "S_diag": chk(dev.S_diag)}
            if N > 1:
                arrs["H_lower"], arrs["S_lower"] = chk(dev.H_lower), chk(dev.S_lower)
            leads = [[chk(t) for t in L] for L in (dev.lead_L, dev.lead_R)]
            if any(v is None for v in arrs.values()) or any(v is None for L in leads for v in L):
                raise TypeError("device arrays must be contiguous complex128 CUDA tensors")
            E = torch.as_tensor(np.asarray(E, dtype=np.float64)).to("cuda")
            ptr = lambda t: t.data_ptr()
            n_E, mem = int(E.shape[0]), RGF_MEM_DEVICE
            # Wait for the producer of the arrays (torch's current stream)
            # only: a device-wide synchronize is refused while an engine
            # thread is capturing its step into a CUDA graph.
            torch.cuda.current_stream(dev.H_diag.device).synchronize()
        else:
            c = lambda a: np.ascontiguousarray(a, dtype=np.complex128)
            arrs = {"H_diag": c(dev.H_diag), "S_diag": c(dev.S_diag)}
            if N > 1:
                arrs["H_lower"], arrs["S_lower"] = c(dev.H_lower), c(dev.S_lower)
            leads = [[c(getattr(ld, k)) for k in ("H00", "S00", "H10", "S10", "Hc", "Sc")]
                     for ld in (dev.lead_L, dev.lead_R)]
            E = np.ascontiguousarray(E, dtype=np.float64)
            ptr = lambda a: a.ctypes.data
            n_E, mem = int(E.shape[0]), RGF_MEM_HOST
        req = rgf_request()
        req.n_layers, req.b, req.eta, req.n_E, req.mem = N, b, float(eta), n_E, mem
        for k, a in arrs.items():
            setattr(req, k, ptr(a))
        for side in range(2):
            for k in range(6):
                req.lead[side][k] = ptr(leads[side][k])
        req.E = ptr(E)
        t = rgf_server_submit(self.handle, req)
        self._keep[t] = (arrs, leads, E, n_E)
        return t

    def poll(self, ticket, timeout_us=-1):
        n = self._keep[ticket][3]
        T = np.empty(n)
        err = np.empty(n)
        flags = np.empty(n, dtype=np.int32)
        st, lat = rgf_server_poll(self.handle, ticket, T, err, flags, timeout_us)
        if st != RGF_OK:
            return None
        del self._keep[ticket]
        return T, err, flags, lat

    def stats(self) -> dict:
        return rgf_server_stats_get(self.handle)

    def close(self):
        if self.handle:
            rgf_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ----------------------------------------------------------------- k points (include/rgf_kpoints.h)
def rgf_bloch_sum(R, k, X_R, X_k, cuda_stream=0):
    """X_k = sum_r exp(2 pi i k.R_r) X_R[r] for CUDA complex128 tensors
    X_R (n_R, n_blocks, b, b) and X_k (n_blocks, b, b); R (n_R, 2) ints, k (2,)."""
    R = np.ascontiguousarray(R, dtype=np.int32)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(-1)[:2])
    pr, mr = _ptr(X_R, np.complex128)
    pk, mk = _ptr(X_k, np.complex128)
    if mr != RGF_MEM_DEVICE or mk != RGF_MEM_DEVICE:
        raise TypeError("rgf_bloch_sum takes device tensors")
    n_R, n_blocks, b = int(X_R.shape[0]), int(X_R.shape[1]), int(X_R.shape[2])
    if R.shape != (n_R, 2) or tuple(X_k.shape) != (n_blocks, b, b):
        raise ValueError("shape mismatch")
    _check(lib().rgf_bloch_sum(n_R, R.ctypes.data, k.ctypes.data, n_blocks, b, pr, pk,
                               _P(cuda_stream) if cuda_stream else None), "rgf_bloch_sum")


def rgf_kmesh_mean(T_k, w, T, cuda_stream=0):
    """T = sum_k w[k] T_k[k] for CUDA float64 tensors T_k (n_k, n_E), w (n_k), T (n_E)."""
    p1, _ = _ptr(T_k, np.float64)
    p2, _ = _ptr(w, np.float64)
    p3, _ = _ptr(T, np.float64)
    _check(lib().rgf_kmesh_mean(int(T_k.shape[0]), int(T_k.shape[1]), p1, p2, p3,
                                _P(cuda_stream) if cuda_stream else None), "rgf_kmesh_mean")


class rgf_kdevice(ctypes.Structure):
    _fields_ = [("n_R", ctypes.c_int), ("R", ctypes.POINTER(ctypes.c_int)), ("n_layers", ctypes.c_int),
                ("b", ctypes.c_int), ("H_diag", _P), ("S_diag", _P), ("H_lower", _P), ("S_lower", _P),
                ("lead", _P * 2)]


def kpoint_transmission(server, kdev, kpts, weights, E, eta, group=8):
    """T(E) of a transverse-periodic device averaged over a k mesh, through
    ``server`` (a ``Server``) by ``rgf_kmesh_transmission``: the Bloch sums,
    the per-k requests and the mesh average all run in the library.
    ``kdev`` has R (n_R, 2) and R-resolved block arrays (as
    synth.devices.KDevice); ``group`` k-points are in flight at once.
    Returns (T (n_E,), T_k (n_k, n_E)) as host arrays."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    up = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.complex128)).cuda()
    XR = {n: up(getattr(kdev, n)) for n in ("H_diag", "S_diag", "H_lower", "S_lower")}
    fields = ("H00", "S00", "H10", "S10", "Hc", "Sc")
    LR = [up(np.stack([getattr(L, f) for f in fields], axis=1)) for L in (kdev.lead_L, kdev.lead_R)]
    R = np.ascontiguousarray(np.asarray(kdev.R), dtype=np.int32)
    N, b = int(XR["H_diag"].shape[1]), int(XR["H_diag"].shape[2])
    d = rgf_kdevice()
    d.n_R, d.R = int(R.shape[0]), R.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.n_layers, d.b = N, b
    d.H_diag, d.S_diag = XR["H_diag"].data_ptr(), XR["S_diag"].data_ptr()
    if N > 1:
        d.H_lower, d.S_lower = XR["H_lower"].data_ptr(), XR["S_lower"].data_ptr()
    d.lead[0], d.lead[1] = LR[0].data_ptr(), LR[1].data_ptr()
    kf = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 2)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    n_k, n_E = kf.shape[0], E.shape[0]
    T = torch.empty(n_E, dtype=torch.float64, device="cuda")
    Tk = torch.empty((n_k, n_E), dtype=torch.float64, device="cuda")
    _check(lib().rgf_kmesh_transmission(server.handle if hasattr(server, "handle") else server, ctypes.byref(d),
                                        n_k, kf.ctypes.data, w.ctypes.data, E.ctypes.data, n_E, float(eta),
                                        int(group), _P(T.data_ptr()), _P(Tk.data_ptr()), _P(stream)),
           "rgf_kmesh_transmission")
    return T.cpu().numpy(), Tk.cpu().numpy()


# ----------------------------------------------------------------- observables (include/rgf_observables.h)
def rgf_current(E, T, V, E_F, kT, I, cuda_stream=0):
    """Landauer current I[v] (ampere) for CUDA float64 tensors E, T (n_E),
    V, I (n_V); energies, biases, E_F and kT in eV."""
    pe, me = _ptr(E, np.float64)
    pt, mt = _ptr(T, np.float64)
    pv, mv = _ptr(V, np.float64)
    pi, mi = _ptr(I, np.float64)
    if {me, mt, mv, mi} != {RGF_MEM_DEVICE}:
        raise TypeError("rgf_current takes device tensors")
    _check(lib().rgf_current(int(E.shape[0]), pe, pt, int(V.shape[0]), pv, float(E_F), float(kT), pi,
                             _P(cuda_stream) if cuda_stream else None), "rgf_current")


def rgf_ldos(plan, E, D):
    """Layer DOS D (n_E, n_layers) of a mixed plan at energies E (host
    numpy arrays or CUDA tensors, both in the same memory space)."""
    pe, me = _ptr(E, np.float64)
    pd, md = _ptr(D, np.float64)
    _check(lib().rgf_ldos(plan, pe, int(E.shape[0]), pd, _mem_of((pe, me), (pd, md))), "rgf_ldos")


# ----------------------------------------------------------------- convenience
class Plan:
    """Owns one rgf_plan_t.  ``precision`` is RGF_FP64 or RGF_MIXED."""

    def __init__(self, n_layers, b, precision=RGF_FP64, eta=1e-6, energy_wave=0, ns_steps=6,
                 dec_tol=1e-14, dec_max_iter=100, cuda_stream=0):
        o = rgf_options_default()
        o.precision, o.eta, o.energy_wave, o.ns_steps = precision, eta, energy_wave, ns_steps
        o.dec_tol, o.dec_max_iter = dec_tol, dec_max_iter
        self.n_layers, self.b = n_layers, b
        self.handle = rgf_plan_create(n_layers, b, o, cuda_stream)

    def set_device(self, dev):
        """Copy a device description with H_diag/S_diag/H_lower/S_lower arrays
        and lead_L/lead_R (H00, S00, H10, S10, Hc, Sc)."""
        c = lambda a: np.ascontiguousarray(a, dtype=np.complex128)
        N = dev.H_diag.shape[0]
        low = (c(dev.H_lower), c(dev.S_lower)) if N > 1 else (None, None)
        rgf_set_device_blocks(self.handle, c(dev.H_diag), c(dev.S_diag), *low)
        for side, ld in ((RGF_LEAD_LEFT, dev.lead_L), (RGF_LEAD_RIGHT, dev.lead_R)):
            rgf_set_leads(self.handle, side, c(ld.H00), c(ld.S00), c(ld.H10), c(ld.S10), c(ld.Hc),
                          c(ld.Sc))

    def transmission(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        T = np.empty_like(E)
        err = np.empty_like(E)
        flags = np.empty(E.shape[0], dtype=np.int32)
        rgf_transmission(self.handle, E, T, err, flags)
        return T, err, flags

    def ldos(self, E):
        """Layer-resolved DOS (n_E, n_layers) of a RGF_MIXED plan."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        D = np.empty((E.shape[0], self.n_layers))
        rgf_ldos(self.handle, E, D)
        return D

    @property
    def stats(self):
        return rgf_plan_stats(self.handle)

    @property
    def energy_wave(self):
        return rgf_plan_energy_wave(self.handle)

    @property
    def device_bytes(self):
        return rgf_plan_device_bytes(self.handle)

    def close(self):
        if self.handle:
            rgf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ----------------------------------------------------------------- KPM Fermi level (include/rgf_kpm.h)
class KPM:
    """Owns one rgf_kpm_t: the device's H and S on the GPU with S factored.
    ``moments(R, n_mom, alpha, beta)`` takes the random vectors as a
    (n_rand, N b) complex array (host or CUDA tensor) and returns mu as a
    host array; ``fermi_level(mu, ...)`` runs the bisection kernel."""

    def __init__(self, dev, cuda_stream=0):
        import torch
        self.N, self.b = int(dev.H_diag.shape[0]), int(dev.H_diag.shape[1])
        self.stream = cuda_stream or torch.cuda.current_stream().cuda_stream
        c = lambda a: np.ascontiguousarray(a, dtype=np.complex128)
        arrs = [c(dev.H_diag), c(dev.S_diag)]
        lows = [c(dev.H_lower), c(dev.S_lower)] if self.N > 1 else [None, None]
        h = _P()
        _check(lib().rgf_kpm_create(ctypes.byref(h), self.N, self.b, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                    lows[0].ctypes.data if lows[0] is not None else None,
                                    lows[1].ctypes.data if lows[1] is not None else None, RGF_MEM_HOST,
                                    _P(self.stream)), "rgf_kpm_create")
        self.handle = h

    def scale(self, x0, iters=100, margin=0.05):
        """(alpha, beta) from a power iteration on S^-1 H started at x0."""
        import torch
        xd = torch.as_tensor(np.asarray(x0)).to(device="cuda", dtype=torch.complex128).contiguous()
        if xd.numel() != self.N * self.b:
            raise ValueError(f"x0 must have {self.N * self.b} entries")
        a, b_ = ctypes.c_double(), ctypes.c_double()
        _check(lib().rgf_kpm_scale(self.handle, _P(xd.data_ptr()), int(iters), float(margin), ctypes.byref(a),
                                   ctypes.byref(b_)), "rgf_kpm_scale")
        return a.value, b_.value

    def moments(self, R, n_mom, alpha, beta):
        import torch
        Rd = torch.as_tensor(R).to(device="cuda", dtype=torch.complex128).contiguous()
        if Rd.dim() != 2 or Rd.shape[1] != self.N * self.b:
            raise ValueError(f"random vectors must be (n_rand, {self.N * self.b})")
        mu = torch.empty(int(n_mom), dtype=torch.float64, device="cuda")
        _check(lib().rgf_kpm_moments(self.handle, float(alpha), float(beta), int(Rd.shape[0]), _P(Rd.data_ptr()),
                                     int(n_mom), _P(mu.data_ptr())), "rgf_kpm_moments")
        return mu.cpu().numpy()

    def fermi_level(self, mu, alpha, beta, n_electrons, spin=2.0):
        import torch
        mu_d = torch.as_tensor(np.ascontiguousarray(mu, dtype=np.float64)).cuda()
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(lib().rgf_kpm_fermi(int(mu_d.shape[0]), _P(mu_d.data_ptr()), float(alpha), float(beta),
                                   float(n_electrons), float(spin), _P(out.data_ptr()), _P(self.stream)),
               "rgf_kpm_fermi")
        torch.cuda.synchronize()
        return float(out.item())

    def close(self):
        if getattr(self, "handle", None):
            lib().rgf_kpm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
