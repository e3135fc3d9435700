"""mbir_backproject_noalloc: A^T r for callers that cannot allocate device memory.

Real-time loops that forbid allocator calls after start-up, and processes
whose device memory is a pool sized in advance by another component, cannot
let the library allocate at the point of the call.  This entry point takes its
scratch from a fixed array in the library, set up when the geometry is
created.  It is checked here, through the C ABI, on two calls in a row (with
different residuals, so the shared scratch is shown to be fully rewritten)
against the ordinary mbir_backproject and against the FP64 oracle's A^T r,
with device free memory the same before the first call and after each call.
The file is collected last so that a failure here cannot hide any other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
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


def _sample_pixels(s, n, seed):
    """Every pixel of small images; for larger ones the corners, the centre and random pixels."""
    if s.N <= 8192:
        return np.arange(s.N)
    rnd = S.SplitMix64(seed).integers(0, s.N - 1, n)
    fixed = np.array([0, s.img_w - 1, s.N - s.img_w, s.N - 1, (s.img_h // 2) * s.img_w + s.img_w // 2])
    return np.unique(np.concatenate([fixed, rnd]))


@pytest.mark.parametrize("scene_fn,mode", [(S.cfg0, "tab"), (ragged_scene, "otf"), (S.cfg1, "tab")])
def test_noalloc_matches_backproject_and_oracle_on_two_calls(scene_fn, mode):
    s = scene_fn()
    geo = M.Geometry(s, mode=mode)
    r_np = [S.random_vector(s.K * s.M, seed) for seed in (21, 22)]
    rs = [torch.as_tensor(r, dtype=torch.float32, device=DEV) for r in r_np]
    refs = []
    for r in rs:
        ref = torch.empty(s.N, device=DEV)
        geo.backproject(r, ref)
        refs.append(ref)
    xs = [torch.full((s.N,), float("nan"), device=DEV) for _ in rs]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info(DEV)[0]]            # before the first call
    for r, x in zip(rs, xs):
        assert noalloc(geo, r, x) == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(DEV)[0])
    assert free[1] == free[0] and free[2] == free[0]
    pix = _sample_pixels(s, 48, 5)
    plan = O.Plan(s, pix=pix)
    for r, x, ref in zip(r_np, xs, refs):
        got = x.cpu().numpy()
        assert rel_l2(got, ref.cpu().numpy()) <= 1e-5
        # the oracle's A^T r of the residual as the kernel sees it (FP32 storage)
        b = plan.backproject(r.astype(np.float32).astype(np.float64))
        assert rel_l2(got[pix], b) <= 1e-5


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
