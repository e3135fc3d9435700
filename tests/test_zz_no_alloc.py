"""mbir_backproject_noalloc: A^T r for callers that cannot allocate device memory.

Real-time loops that forbid allocator calls after start-up, and processes
whose device memory is a pool sized in advance by another component, cannot
let the library allocate at the point of the call.  This entry point takes its
scratch from a fixed array in the library.  It is checked here, through the
C ABI, against the ordinary mbir_backproject on two calls in a row (with
different residuals, so the shared scratch is shown to be fully rewritten),
with device free memory unchanged between the calls.  The file is collected
last so that a failure here cannot hide any other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_09703_gb300 import build as B  # noqa: E402

B.build()
from paper_2202_09703_gb300 import mbir as M  # noqa: E402
from paper_2202_09703_gb300 import synth as S  # noqa: E402
from tests.helpers import ragged_scene, rel_l2  # noqa: E402

DEV = torch.device("cuda:0")


def noalloc(geo, r, x):
    f = M.lib().mbir_backproject_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f(geo.h, C.c_void_p(r.data_ptr()), C.c_void_p(x.data_ptr()),
             C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("scene_fn,mode", [(S.cfg0, "tab"), (ragged_scene, "otf"), (S.cfg1, "tab")])
def test_noalloc_matches_backproject_on_two_calls(scene_fn, mode):
    s = scene_fn()
    geo = M.Geometry(s, mode=mode)
    rs = [torch.as_tensor(S.random_vector(s.K * s.M, seed), dtype=torch.float32, device=DEV) for seed in (21, 22)]
    refs = []
    for r in rs:
        ref = torch.empty(s.N, device=DEV)
        geo.backproject(r, ref)
        refs.append(ref)
    torch.cuda.synchronize()
    free = []
    for r, ref in zip(rs, refs):
        x = torch.full((s.N,), float("nan"), device=DEV)
        torch.cuda.synchronize()
        assert noalloc(geo, r, x) == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(DEV)[0])
        assert rel_l2(x.cpu().numpy(), ref.cpu().numpy()) <= 1e-5
    assert free[0] == free[1]


def test_noalloc_rejects_geometry_beyond_the_fixed_scratch():
    s = S.small_scene(n_layers=2, w=128, h=32, n_tx=128, n_rx=32, M=1024, name="tiny_big")
    geo = M.Geometry(s, mode="otf")
    r = torch.zeros(s.K * s.M, device=DEV)
    x = torch.zeros(s.N, device=DEV)
    assert noalloc(geo, r, x) == -7


def test_noalloc_rejects_bf16_storage():
    s = S.cfg0().copy(precision="bf16")
    geo = M.Geometry(s)
    r = torch.zeros(s.K * s.M, device=DEV)
    x = torch.zeros(s.N, device=DEV)
    assert noalloc(geo, r, x) == -7
