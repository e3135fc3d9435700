"""Host-side checks of the C ABI library (no GPU needed).

The library must build for sm_103a, load, export every entry point that
include/mbir.h declares, and reject bad geometry descriptions before touching
the device.
"""
import ctypes as C
import os
import re

import pytest

from paper_2202_09703_gb300 import build as B
from paper_2202_09703_gb300 import mbir as M
from paper_2202_09703_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return M.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "mbir.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mbir_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "mbir_forward" in names and "mbir_backproject" in names and "mbir_reconstruct" in names
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(L):
    assert L.mbir_error_string(0) == b"ok"
    assert L.mbir_error_string(-1) == b"invalid argument"
    assert L.mbir_error_string(-5) == b"bounded wait timed out"


def _create(L, desc):
    h = C.c_void_p()
    return L.mbir_create_geometry(C.byref(desc), None, C.byref(h))


@pytest.mark.parametrize("field,value", [
    ("n_layers", 0), ("n_layers", 9), ("img_w", 0), ("img_h", -3), ("pitch_m", 0.0),
    ("img_z0_m", -1e-3), ("n_tx", 0), ("n_rx", 0), ("fs_hz", 0.0), ("n_samples", 0),
    ("fc_hz", -1.0), ("n_cycles", 0.0), ("beta", -1.0), ("gamma_bins", 1), ("precision", 7), ("mode", 5),
])
def test_invalid_geometry_rejected_before_device(L, field, value):
    desc, keep = M.desc_from_scene(S.cfg0())
    setattr(desc, field, value)
    assert _create(L, desc) == -1


@pytest.mark.parametrize("what", ["thickness_m", "speed_mps", "density_kgm3"])
def test_nonpositive_layer_rejected(L, what):
    desc, keep = M.desc_from_scene(S.cfg0())
    getattr(desc, what)[1] = 0.0
    assert _create(L, desc) == -1


def test_negative_attenuation_and_nan_positions_rejected(L):
    desc, keep = M.desc_from_scene(S.cfg0())
    desc.atten_np_per_mhz_m[0] = -0.1
    assert _create(L, desc) == -1
    desc, keep = M.desc_from_scene(S.cfg0())
    keep[0][3] = float("nan")
    assert _create(L, desc) == -1


def test_null_arguments_rejected(L):
    assert L.mbir_create_geometry(None, None, None) == -1
    assert L.mbir_forward(None, None, None, None) == -1
    assert L.mbir_backproject(None, None, None, None) == -1
    assert L.mbir_destroy_geometry(None) == 0
    assert L.mbir_geometry_bytes(None) == 0
