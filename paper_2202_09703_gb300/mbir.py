"""Thin Python binding of ``libmbir.so`` (ctypes; argument marshalling only).

Every computation runs in the library's CUDA kernels.  torch supplies device
memory (``tensor.data_ptr()``) and streams (``stream.cuda_stream``).  If the
library has not been built the import of :func:`lib` fails loudly; there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_LAYERS = 8
MODES = {"auto": 0, "otf": 1, "tab": 2}
PRECISIONS = {"fp32": 0, "bf16": 1}
ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "non-finite",
          -5: "timeout", -6: "busy", -7: "unsupported", -8: "cancelled", -9: "not ready"}


class MbirError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, 'unknown')} ({code})")


class GeometryDesc(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int),
        ("thickness_m", C.c_double * MAX_LAYERS),
        ("speed_mps", C.c_double * MAX_LAYERS),
        ("atten_np_per_mhz_m", C.c_double * MAX_LAYERS),
        ("density_kgm3", C.c_double * MAX_LAYERS),
        ("img_w", C.c_int), ("img_h", C.c_int),
        ("pitch_m", C.c_double), ("img_x0_m", C.c_double), ("img_z0_m", C.c_double),
        ("n_tx", C.c_int), ("tx_x_m", C.POINTER(C.c_double)),
        ("n_rx", C.c_int), ("rx_offset_m", C.POINTER(C.c_double)),
        ("fs_hz", C.c_double), ("n_samples", C.c_int),
        ("fc_hz", C.c_double), ("n_cycles", C.c_double),
        ("beta", C.c_double), ("direct_arrival", C.c_int),
        ("gamma_max_s", C.c_double), ("gamma_bins", C.c_int), ("phases", C.c_int),
        ("precision", C.c_int), ("mode", C.c_int), ("flags", C.c_int),
        ("firing_angle_rad", C.c_double), ("apodization", C.c_int),
    ]


FLAG_NO_RECORDS = 1
FLAG_NO_TENSOR_CORES = 2


class Prior(C.Structure):
    _fields_ = [("p", C.c_double), ("q", C.c_double), ("T", C.c_double), ("sigma0", C.c_double),
                ("m", C.c_double), ("a", C.c_double), ("sigma_noise", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("cost", C.POINTER(C.c_double)), ("cost_len", C.c_int), ("iterations", C.c_int),
                ("grad_norm_first", C.c_double), ("grad_norm_last", C.c_double)]


class KernelTimes(C.Structure):
    _fields_ = [("forward_launches", C.c_int64), ("backproject_launches", C.c_int64),
                ("forward_ms", C.c_double), ("backproject_ms", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_pixels", C.c_int64), ("n_ascans", C.c_int64), ("n_samples", C.c_int64),
                ("pulse_support", C.c_int), ("gamma_bins", C.c_int), ("phases", C.c_int),
                ("gamma_max_s", C.c_double), ("mode", C.c_int), ("precision", C.c_int),
                ("device_bytes", C.c_int64), ("forward_window_spans", C.c_int),
                ("forward_window_ms", C.c_double * 3), ("adjoint_groups", C.c_int),
                ("adjoint_tensor_cores", C.c_int), ("forward_tensor_cores", C.c_int),
                ("n_records", C.c_int64), ("record_bytes", C.c_int64),
                ("tc_forward_variant", C.c_int), ("tc_adjoint_variant", C.c_int),
                ("tc_variant_ms", C.c_double * 4)]


_lib = None
_V = C.c_void_p


def lib(path: str | None = None):
    """Load libmbir.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(paper_2202_09703_gb300.build.build())")
    L = C.CDLL(path)
    D, Pp, S, I = C.POINTER(GeometryDesc), C.POINTER(Prior), C.POINTER(Stats), C.POINTER(Info)
    sig = {
        "mbir_create_geometry": [D, _V, C.POINTER(_V)],
        "mbir_destroy_geometry": [_V],
        "mbir_geometry_get_info": [_V, I],
        "mbir_set_forward_window": [_V, C.c_int],
        "mbir_set_tensor_core_variants": [_V, C.c_int, C.c_int],
        "mbir_forward": [_V, _V, _V, _V],
        "mbir_backproject": [_V, _V, _V, _V],
        "mbir_project": [_V, _V, _V, _V, _V],
        "mbir_prior_gradient": [_V, Pp, _V, _V, _V],
        "mbir_add_direct": [_V, _V, _V, _V],
        "mbir_reconstruct": [_V, _V, Pp, C.c_int, _V, C.c_int, _V, S, _V],
        "mbir_reconstruct_icd": [_V, _V, Pp, C.c_int, C.c_int, _V, C.c_int, _V, S, _V],
        "mbir_column_norms": [_V, _V, _V],
        "mbir_reconstruct_host": [_V, _V, Pp, C.c_int, _V, _V, S, _V],
        "mbir_pair_quantities": [_V, _V, _V, C.c_int, _V, _V, _V],
        "mbir_pulse_table": [_V, _V, C.c_size_t],
        "mbir_set_profiling": [_V, C.c_int],
        "mbir_get_kernel_times": [_V, C.POINTER(KernelTimes), C.c_int],
        "mbir_count_taps": [_V, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "mbir_engine_create": [C.c_size_t, C.c_int, C.POINTER(_V)],
        "mbir_engine_destroy": [_V],
        "mbir_engine_submit": [_V, _V, _V, Pp, C.c_int, _V, _V, C.POINTER(C.c_int64)],
        "mbir_engine_step": [_V, _V, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "mbir_engine_poll": [_V, C.c_int64, C.POINTER(C.c_int)],
        "mbir_engine_wait": [_V, C.c_int64, C.c_int, _V],
        "mbir_engine_cancel": [_V, C.c_int64, _V],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.mbir_geometry_bytes.argtypes = [_V]
    L.mbir_geometry_bytes.restype = C.c_size_t
    L.mbir_engine_bytes_in_use.argtypes = [_V]
    L.mbir_engine_bytes_in_use.restype = C.c_size_t
    L.mbir_error_string.argtypes = [C.c_int]
    L.mbir_error_string.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != 0:
        raise MbirError(rc, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def desc_from_scene(scene, mode: str = "auto", precision: str | None = None, flags: int = 0):
    d = GeometryDesc()
    n = len(scene.layers)
    d.n_layers = n
    for i, L in enumerate(scene.layers):
        d.thickness_m[i] = L.thickness
        d.speed_mps[i] = L.speed
        d.atten_np_per_mhz_m[i] = L.atten
        d.density_kgm3[i] = L.density
    d.img_w, d.img_h = scene.img_w, scene.img_h
    d.pitch_m, d.img_x0_m, d.img_z0_m = scene.pitch, scene.x0, scene.z0
    tx = np.ascontiguousarray(scene.tx_x, dtype=np.float64)
    rx = np.ascontiguousarray(scene.rx_offset, dtype=np.float64)
    d.n_tx, d.tx_x_m = len(tx), tx.ctypes.data_as(C.POINTER(C.c_double))
    d.n_rx, d.rx_offset_m = len(rx), rx.ctypes.data_as(C.POINTER(C.c_double))
    d.fs_hz, d.n_samples = scene.fs, scene.n_samples
    d.fc_hz, d.n_cycles = scene.fc, scene.n_cycles
    d.beta, d.direct_arrival = scene.beta, int(bool(scene.direct_arrival))
    d.gamma_max_s, d.gamma_bins, d.phases = scene.gamma_max, scene.G, scene.Q
    d.precision = PRECISIONS[precision or scene.precision]
    d.mode = MODES[mode]
    d.flags = flags
    d.firing_angle_rad = getattr(scene, "firing_angle", 0.0)
    d.apodization = 1 if getattr(scene, "apod_first_angle", False) else 0
    return d, (tx, rx)


def prior_struct(scene, sigma_noise: float) -> Prior:
    p = scene.prior
    return Prior(p.p, p.q, p.T, p.sigma0, p.m, p.a, sigma_noise)


class Geometry:
    """A geometry handle: device tables of one scan (see include/mbir.h)."""

    def __init__(self, scene, mode: str = "auto", precision: str | None = None, stream=None,
                 records: bool = True, tensor_cores: bool = True):
        self.scene = scene
        self._lib = lib()
        flags = (0 if records else FLAG_NO_RECORDS) | (0 if tensor_cores else FLAG_NO_TENSOR_CORES)
        desc, self._keep = desc_from_scene(scene, mode, precision, flags)
        h = C.c_void_p()
        _check(self._lib.mbir_create_geometry(C.byref(desc), _stream_ptr(stream), C.byref(h)),
               "mbir_create_geometry")
        self.h = h
        info = Info()
        _check(self._lib.mbir_geometry_get_info(self.h, C.byref(info)), "mbir_geometry_get_info")
        self.info = info
        self.mode = {1: "otf", 2: "tab"}[info.mode]
        self.precision = {0: "fp32", 1: "bf16"}[info.precision]

    def close(self):
        if getattr(self, "h", None):
            self._lib.mbir_destroy_geometry(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self) -> int:
        return int(self._lib.mbir_geometry_bytes(self.h))

    def forward(self, x, y, stream=None):
        _check(self._lib.mbir_forward(self.h, _ptr(x), _ptr(y), _stream_ptr(stream)), "mbir_forward")
        return y

    def backproject(self, r, x, stream=None):
        _check(self._lib.mbir_backproject(self.h, _ptr(r), _ptr(x), _stream_ptr(stream)), "mbir_backproject")
        return x

    def project(self, r, e, gk=None, stream=None):
        _check(self._lib.mbir_project(self.h, _ptr(r), _ptr(e), _ptr(gk), _stream_ptr(stream)), "mbir_project")
        return e

    def add_direct(self, gk, y, stream=None):
        _check(self._lib.mbir_add_direct(self.h, _ptr(gk), _ptr(y), _stream_ptr(stream)), "mbir_add_direct")
        return y

    def prior_gradient(self, x, out, sigma_noise: float = 1.0, stream=None):
        pr = prior_struct(self.scene, sigma_noise)
        _check(self._lib.mbir_prior_gradient(self.h, C.byref(pr), _ptr(x), _ptr(out), _stream_ptr(stream)),
               "mbir_prior_gradient")
        return out

    def reconstruct(self, y, sigma_noise: float, n_iter: int, x, x_given: bool = False, g=None,
                    want_cost: bool = False, stream=None):
        pr = prior_struct(self.scene, sigma_noise)
        st = Stats()
        cost = np.zeros(max(n_iter, 1))
        if want_cost:
            st.cost = cost.ctypes.data_as(C.POINTER(C.c_double))
            st.cost_len = n_iter
        _check(self._lib.mbir_reconstruct(self.h, _ptr(y), C.byref(pr), n_iter, _ptr(x), int(x_given), _ptr(g),
                                          C.byref(st), _stream_ptr(stream)), "mbir_reconstruct")
        return {"cost": cost[:n_iter] if want_cost else None, "iterations": st.iterations,
                "grad_norm_first": st.grad_norm_first, "grad_norm_last": st.grad_norm_last}

    def reconstruct_icd(self, y, sigma_noise: float, n_sweeps: int, spacing: int, x, x_given: bool = False,
                        g=None, want_cost: bool = False, stream=None):
        """Coloured ICD (``mbir_reconstruct_icd``); spacing >= the image sides is sequential ICD."""
        pr = prior_struct(self.scene, sigma_noise)
        st = Stats()
        cost = np.zeros(max(n_sweeps, 1))
        if want_cost:
            st.cost = cost.ctypes.data_as(C.POINTER(C.c_double))
            st.cost_len = n_sweeps
        _check(self._lib.mbir_reconstruct_icd(self.h, _ptr(y), C.byref(pr), n_sweeps, spacing, _ptr(x),
                                              int(x_given), _ptr(g), C.byref(st), _stream_ptr(stream)),
               "mbir_reconstruct_icd")
        return {"cost": cost[:n_sweeps] if want_cost else None, "iterations": st.iterations}

    def column_norms(self, out, stream=None):
        """|A_v|^2 per pixel into the N-float device tensor ``out``."""
        _check(self._lib.mbir_column_norms(self.h, _ptr(out), _stream_ptr(stream)), "mbir_column_norms")
        return out

    def reconstruct_host(self, y_host, sigma_noise: float, n_iter: int, x_host, g_host=None, stream=None):
        """y_host, x_host, g_host: host tensors (pinned for asynchronous copies)."""
        pr = prior_struct(self.scene, sigma_noise)
        st = Stats()
        _check(self._lib.mbir_reconstruct_host(self.h, _ptr(y_host), C.byref(pr), n_iter, _ptr(x_host),
                                               _ptr(g_host), C.byref(st), _stream_ptr(stream)),
               "mbir_reconstruct_host")
        return x_host

    def pair_quantities(self, pix, k):
        pix = np.ascontiguousarray(pix, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        n = len(pix)
        T = np.zeros(n, np.float64)
        g = np.zeros(n, np.float32)
        w = np.zeros(n, np.float32)
        _check(self._lib.mbir_pair_quantities(self.h, pix.ctypes.data, k.ctypes.data, n, T.ctypes.data,
                                              g.ctypes.data, w.ctypes.data), "mbir_pair_quantities")
        return T, g, w

    def set_profiling(self, on: bool = True):
        _check(self._lib.mbir_set_profiling(self.h, int(on)), "mbir_set_profiling")

    def kernel_times(self, reset: bool = False) -> dict:
        t = KernelTimes()
        _check(self._lib.mbir_get_kernel_times(self.h, C.byref(t), int(reset)), "mbir_get_kernel_times")
        return {"forward_launches": t.forward_launches, "backproject_launches": t.backproject_launches,
                "forward_ms": t.forward_ms, "backproject_ms": t.backproject_ms}

    def set_forward_window(self, spans: int):
        """Override the autotuned A x window (1, 2 or 4 spans per warp)."""
        _check(self._lib.mbir_set_forward_window(self.h, int(spans)), "mbir_set_forward_window")
        _check(self._lib.mbir_geometry_get_info(self.h, C.byref(self.info)), "mbir_geometry_get_info")

    def set_tensor_core_variants(self, forward: int = -1, adjoint: int = -1):
        """Override the timed choice of the tensor-core A x / A^T variants (0 or 1; -1 keeps)."""
        _check(self._lib.mbir_set_tensor_core_variants(self.h, int(forward), int(adjoint)),
               "mbir_set_tensor_core_variants")
        _check(self._lib.mbir_geometry_get_info(self.h, C.byref(self.info)), "mbir_geometry_get_info")

    def count_taps(self):
        a, b = C.c_int64(), C.c_int64()
        _check(self._lib.mbir_count_taps(self.h, C.byref(a), C.byref(b)), "mbir_count_taps")
        return a.value, b.value

    def pulse_table(self) -> np.ndarray:
        G, Q, Tw = self.info.gamma_bins, self.info.phases, self.info.pulse_support
        out = np.zeros(G * (Q * Tw + 1))
        _check(self._lib.mbir_pulse_table(self.h, out.ctypes.data, out.size), "mbir_pulse_table")
        return out.reshape(G, Q * Tw + 1)


class Engine:
    """Batched / served reconstructions (continuous batching, see include/mbir.h)."""

    QUEUED, RUNNING, DONE = 0, 1, 3

    def __init__(self, budget_bytes: int, max_active: int = 256):
        self._lib = lib()
        h = C.c_void_p()
        _check(self._lib.mbir_engine_create(budget_bytes, max_active, C.byref(h)), "mbir_engine_create")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self._lib.mbir_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, geo: "Geometry", y, sigma_noise: float, n_iter: int, x, g=None) -> int:
        pr = prior_struct(geo.scene, sigma_noise)
        t = C.c_int64()
        _check(self._lib.mbir_engine_submit(self.h, geo.h, _ptr(y), C.byref(pr), n_iter, _ptr(x), _ptr(g),
                                            C.byref(t)), "mbir_engine_submit")
        self._keep[t.value] = (geo, y, x, g)
        return t.value

    def step(self, stream=None):
        na, nq = C.c_int(), C.c_int()
        _check(self._lib.mbir_engine_step(self.h, _stream_ptr(stream), C.byref(na), C.byref(nq)), "mbir_engine_step")
        return na.value, nq.value

    def poll(self, ticket: int) -> int:
        st = C.c_int()
        rc = self._lib.mbir_engine_poll(self.h, ticket, C.byref(st))
        if rc not in (0,) and st.value >= 0:
            _check(rc, "mbir_engine_poll")
        return st.value

    def wait(self, ticket: int, timeout_ms: int = 600000, stream=None):
        _check(self._lib.mbir_engine_wait(self.h, ticket, timeout_ms, _stream_ptr(stream)), "mbir_engine_wait")

    def cancel(self, ticket: int, stream=None):
        _check(self._lib.mbir_engine_cancel(self.h, ticket, _stream_ptr(stream)), "mbir_engine_cancel")

    def run_until_idle(self, stream=None, max_steps: int = 1_000_000):
        for _ in range(max_steps):
            na, nq = self.step(stream)
            if na == 0 and nq == 0:
                return
        raise RuntimeError("engine did not drain")

    @property
    def bytes_in_use(self) -> int:
        return int(self._lib.mbir_engine_bytes_in_use(self.h))
