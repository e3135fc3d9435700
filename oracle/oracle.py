"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this module.  It builds ``mbir_oracle.c`` with gcc on
first use (or through :func:`build`) and exposes the oracle with numpy arrays.
Scenes are duck-typed: any object with the attributes of
``paper_2202_09703_gb300.synth.Scene`` works; this module imports nothing from
the CUDA library's package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mbir_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
MAX_LAYERS = 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP, IEEE math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mbir_oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Geom(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int),
        ("thickness", C.c_double * MAX_LAYERS),
        ("speed", C.c_double * MAX_LAYERS),
        ("atten", C.c_double * MAX_LAYERS),
        ("density", C.c_double * MAX_LAYERS),
        ("img_w", C.c_int), ("img_h", C.c_int),
        ("pitch", C.c_double), ("x0", C.c_double), ("z0", C.c_double),
        ("n_tx", C.c_int), ("tx_x", C.POINTER(C.c_double)),
        ("n_rx", C.c_int), ("rx_offset", C.POINTER(C.c_double)),
        ("fs", C.c_double), ("n_samples", C.c_int),
        ("fc", C.c_double), ("n_cycles", C.c_double),
        ("beta", C.c_double), ("direct_arrival", C.c_int),
        ("gamma_max", C.c_double), ("G", C.c_int), ("Q", C.c_int),
        ("tilt", C.c_double), ("apod_first", C.c_int),
    ]


class _Prior(C.Structure):
    _fields_ = [("p", C.c_double), ("q", C.c_double), ("T", C.c_double),
                ("sigma0", C.c_double), ("m", C.c_double), ("a", C.c_double),
                ("sigma_noise", C.c_double)]


_D = C.POINTER(C.c_double)
_L = C.POINTER(C.c_long)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            G, P = C.POINTER(_Geom), C.POINTER(_Prior)
            sig = {
                "orc_pulse_support": (C.c_int, [G]),
                "orc_pulse": (C.c_double, [G, C.c_double]),
                "orc_gamma_max": (C.c_double, [G]),
                "orc_effective_G": (C.c_int, [G]),
                "orc_pulse_table": (None, [G, _D, C.c_int]),
                "orc_leg": (None, [G, C.c_double, C.c_double, _D, _D, _D, _D]),
                "orc_transmission": (C.c_double, [G, C.c_double]),
                "orc_plan_create": (C.c_void_p, [G, _L, C.c_long, C.c_int]),
                "orc_plan_destroy": (None, [C.c_void_p]),
                "orc_plan_pair": (None, [C.c_void_p, C.c_long, C.c_int, _D, _D, _D]),
                "orc_plan_H": (C.c_double, [C.c_void_p, C.c_double, C.c_double]),
                "orc_forward": (None, [C.c_void_p, _D, _D, C.c_int, C.c_int, C.c_int]),
                "orc_backproject": (None, [C.c_void_p, _D, _D, C.c_int]),
                "orc_dense_A": (None, [C.c_void_p, _D]),
                "orc_direct_columns": (None, [C.c_void_p, _D]),
                "orc_project": (None, [C.c_void_p, _D, _D, _D]),
                "orc_prior_cost": (C.c_double, [G, P, _D]),
                "orc_prior_grad": (None, [G, P, _D, _D]),
                "orc_prior_curv": (C.c_double, [G, P, _D, _D]),
                "orc_rho": (C.c_double, [P, C.c_double, C.c_double]),
                "orc_drho": (C.c_double, [P, C.c_double, C.c_double]),
                "orc_kappa": (C.c_double, [P, C.c_double, C.c_double]),
                "orc_reconstruct": (C.c_int, [C.c_void_p, P, _D, C.c_int, _D, C.c_int,
                                              _D, _D, _D, C.c_int]),
                "orc_column_norms": (None, [C.c_void_p, _D, C.c_int]),
                "orc_icd": (C.c_int, [C.c_void_p, P, _D, C.c_int, C.c_int, _D, C.c_int, _D, _D, C.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D)


class Geometry:
    """Marshals a scene into the oracle's own C struct (arrays kept alive)."""

    def __init__(self, scene):
        self.scene = scene
        g = _Geom()
        layers = scene.layers
        if not 1 <= len(layers) <= MAX_LAYERS:
            raise ValueError("1..8 layers")
        g.n_layers = len(layers)
        for i, L in enumerate(layers):
            g.thickness[i] = L.thickness
            g.speed[i] = L.speed
            g.atten[i] = L.atten * 1e-6        # Np/(MHz m) -> s/m
            g.density[i] = L.density
        g.img_w, g.img_h = scene.img_w, scene.img_h
        g.pitch, g.x0, g.z0 = scene.pitch, scene.x0, scene.z0
        self._tx = np.ascontiguousarray(scene.tx_x, dtype=np.float64)
        self._rx = np.ascontiguousarray(scene.rx_offset, dtype=np.float64)
        g.n_tx, g.tx_x = len(self._tx), _ptr(self._tx)
        g.n_rx, g.rx_offset = len(self._rx), _ptr(self._rx)
        g.fs, g.n_samples = scene.fs, scene.n_samples
        g.fc, g.n_cycles = scene.fc, scene.n_cycles
        g.beta, g.direct_arrival = scene.beta, int(bool(scene.direct_arrival))
        g.gamma_max, g.G, g.Q = scene.gamma_max, scene.G, scene.Q
        g.tilt, g.apod_first = scene.firing_angle, int(bool(scene.apod_first_angle))
        self.g = g

    @property
    def ref(self):
        return C.byref(self.g)

    def pulse_support(self) -> int:
        return lib().orc_pulse_support(self.ref)

    def pulse(self, t: float) -> float:
        return lib().orc_pulse(self.ref, t)

    def gamma_max(self) -> float:
        return lib().orc_gamma_max(self.ref)

    def effective_G(self) -> int:
        return lib().orc_effective_G(self.ref)

    def pulse_table(self, panels_scale: int = 1) -> np.ndarray:
        G = self.effective_G()
        nq = self.scene.Q * self.pulse_support() + 1
        out = np.zeros(G * nq)
        lib().orc_pulse_table(self.ref, _ptr(out), panels_scale)
        return out.reshape(G, nq)

    def leg(self, h: float, z: float):
        T, gm, Th, t1 = (C.c_double(), C.c_double(), C.c_double(), C.c_double())
        lib().orc_leg(self.ref, h, z, C.byref(T), C.byref(gm), C.byref(Th), C.byref(t1))
        return T.value, gm.value, Th.value, t1.value

    def transmission(self, z: float) -> float:
        return lib().orc_transmission(self.ref, z)


def make_prior(scene, sigma_noise: float) -> _Prior:
    p = scene.prior
    return _Prior(p.p, p.q, p.T, p.sigma0, p.m, p.a, sigma_noise)


class Plan:
    """Leg cache + pulse table for a pixel subset (None = every pixel)."""

    def __init__(self, scene, pix=None, nthreads: int = 0):
        self.geom = Geometry(scene)
        self.scene = scene
        self.nthreads = nthreads or (os.cpu_count() or 1)
        if pix is None:
            self._pix = None
            self.npix = scene.img_w * scene.img_h
            self.h = lib().orc_plan_create(self.geom.ref, None, 0, self.nthreads)
        else:
            self._pix = np.ascontiguousarray(pix, dtype=np.int64)
            self.npix = len(self._pix)
            self.h = lib().orc_plan_create(self.geom.ref, self._pix.ctypes.data_as(_L),
                                           self.npix, self.nthreads)

    def close(self):
        if self.h:
            lib().orc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pair(self, slot: int, k: int):
        T, gm, w = C.c_double(), C.c_double(), C.c_double()
        lib().orc_plan_pair(self.h, slot, k, C.byref(T), C.byref(gm), C.byref(w))
        return T.value, gm.value, w.value

    def H(self, gamma: float, tau: float) -> float:
        return lib().orc_plan_H(self.h, gamma, tau)

    def forward(self, x, k_lo: int = 0, k_hi: int | None = None) -> np.ndarray:
        s = self.scene
        k_hi = s.K if k_hi is None else k_hi
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        y = np.zeros((k_hi - k_lo, s.M))
        lib().orc_forward(self.h, _ptr(x), _ptr(y), k_lo, k_hi, self.nthreads)
        return y

    def backproject(self, r) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        b = np.zeros(self.npix)
        lib().orc_backproject(self.h, _ptr(r), _ptr(b), self.nthreads)
        return b

    def dense_A(self) -> np.ndarray:
        s = self.scene
        A = np.zeros((s.K * s.M, self.npix))
        lib().orc_dense_A(self.h, _ptr(A))
        return A

    def direct_columns(self) -> np.ndarray:
        s = self.scene
        d = np.zeros((s.n_rx, s.M))
        lib().orc_direct_columns(self.h, _ptr(d))
        return d

    def project(self, r):
        s = self.scene
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        e = np.zeros(s.K * s.M)
        gk = np.zeros(s.K)
        lib().orc_project(self.h, _ptr(r), _ptr(e), _ptr(gk))
        return e.reshape(s.K, s.M), gk

    def reconstruct(self, y, sigma_noise: float, n_iter: int, x0=None):
        s = self.scene
        pr = make_prior(s, sigma_noise)
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        x = np.zeros(s.N) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
        gk = np.zeros(s.K)
        cost = np.zeros(max(n_iter, 1))
        gn = np.zeros(max(n_iter, 1))
        rc = lib().orc_reconstruct(self.h, C.byref(pr), _ptr(y), n_iter, _ptr(x),
                                   int(x0 is not None), _ptr(gk), _ptr(cost), _ptr(gn),
                                   self.nthreads)
        if rc != 0:
            raise RuntimeError("oracle reconstruct needs a plan over every pixel")
        return x.reshape(s.img_h, s.img_w), gk, cost[:n_iter], gn[:n_iter]


    def column_norms(self) -> np.ndarray:
        """|A_v|^2 for every plan pixel."""
        out = np.zeros(self.npix)
        lib().orc_column_norms(self.h, _ptr(out), self.nthreads)
        return out

    def icd(self, y, sigma_noise: float, n_sweeps: int, spacing: int, x0=None):
        """Coloured ICD (spacing >= image side: sequential ICD in raster order)."""
        s = self.scene
        pr = make_prior(s, sigma_noise)
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        x = np.zeros(s.N) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
        gk = np.zeros(s.K)
        cost = np.zeros(max(n_sweeps, 1))
        rc = lib().orc_icd(self.h, C.byref(pr), _ptr(y), n_sweeps, spacing, _ptr(x),
                           int(x0 is not None), _ptr(gk), _ptr(cost), self.nthreads)
        if rc != 0:
            raise RuntimeError("oracle ICD needs a plan over every pixel and spacing >= 2")
        return x.reshape(s.img_h, s.img_w), gk, cost[:n_sweeps]


# prior helpers ------------------------------------------------------------
def prior_cost(scene, x, sigma_noise: float = 1.0) -> float:
    g = Geometry(scene)
    pr = make_prior(scene, sigma_noise)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    return lib().orc_prior_cost(g.ref, C.byref(pr), _ptr(x))


def prior_grad(scene, x, sigma_noise: float = 1.0) -> np.ndarray:
    g = Geometry(scene)
    pr = make_prior(scene, sigma_noise)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.zeros_like(x)
    lib().orc_prior_grad(g.ref, C.byref(pr), _ptr(x), _ptr(out))
    return out


def prior_curv(scene, x, d, sigma_noise: float = 1.0) -> float:
    g = Geometry(scene)
    pr = make_prior(scene, sigma_noise)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
    return lib().orc_prior_curv(g.ref, C.byref(pr), _ptr(x), _ptr(d))


def rho(scene, delta, sigma):
    pr = make_prior(scene, 1.0)
    return lib().orc_rho(C.byref(pr), delta, sigma)


def drho(scene, delta, sigma):
    pr = make_prior(scene, 1.0)
    return lib().orc_drho(C.byref(pr), delta, sigma)


def kappa(scene, delta, sigma):
    pr = make_prior(scene, 1.0)
    return lib().orc_kappa(C.byref(pr), delta, sigma)
