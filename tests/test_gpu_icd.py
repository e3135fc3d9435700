"""Coloured iterative coordinate descent on the GPU against the FP64 oracle (needs a GB300).

Gates: column norms within relative L2 1e-5 of the oracle's; after the sweeps the
image and the direct-arrival gains within relative L2 1e-4 and the cost per
sweep within 1e-4 relative (FP32); BF16 storage within 1e-2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_09703_gb300 import synth as S
from tests.helpers import oracle_data, ragged_scene, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_09703_gb300 import build as B  # noqa: E402

B.build()
from paper_2202_09703_gb300 import mbir as M  # noqa: E402

DEV = torch.device("cuda:0")


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV)


@pytest.mark.parametrize("mode", ["otf", "tab"])
@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_column_norms_match_oracle(mode, scene_fn):
    s = scene_fn()
    geo = M.Geometry(s, mode=mode)
    out = torch.empty(s.N, device=DEV)
    geo.column_norms(out)
    torch.cuda.synchronize()
    ref = O.Plan(s).column_norms()
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("scene_fn,spacing", [(S.cfg0, 2), (S.cfg0, 3), (ragged_scene, 2), (ragged_scene, 40)])
def test_icd_matches_oracle(scene_fn, spacing):
    """spacing 40 on the 40 x 23 scene is sequential ICD: one pixel per colour."""
    s = scene_fn()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=3)
    n_sweeps = 2
    x_ref, g_ref, cost_ref = plan.icd(y, sig, n_sweeps, spacing)
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    g = torch.empty(s.K, device=DEV)
    out = geo.reconstruct_icd(to_dev(y), sig, n_sweeps, spacing, x, g=g, want_cost=True)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_ref) <= 1e-4
    assert np.allclose(out["cost"], cost_ref, rtol=1e-4)
    assert np.all(np.diff(out["cost"]) <= 1e-6 * abs(out["cost"][0]))
    if s.direct_arrival:
        assert rel_l2(g.cpu().numpy(), g_ref) <= 1e-4


@pytest.mark.parametrize("mode", ["otf", "tab-norec"])
def test_icd_without_colour_records(mode):
    """OTF mode and TAB mode without records: the colour's A^T on its pixel lattice, the full A x."""
    s = ragged_scene()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=5)
    x_ref, _, cost_ref = plan.icd(y, sig, 2, 3)
    geo = M.Geometry(s, mode="tab", records=False) if mode == "tab-norec" else M.Geometry(s, mode=mode)
    x = torch.empty(s.N, device=DEV)
    out = geo.reconstruct_icd(to_dev(y), sig, 2, 3, x, want_cost=True)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_ref) <= 1e-4
    assert np.allclose(out["cost"], cost_ref, rtol=1e-4)


def test_icd_work_lists_rebuilt_per_spacing():
    """Switching the spacing rebuilds the colour lists; the same spacing gives the same bits again."""
    s = S.cfg0()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=6)
    geo = M.Geometry(s)
    yd = to_dev(y)
    xs = []
    for sp in (4, 3, 4):
        x = torch.empty(s.N, device=DEV)
        geo.reconstruct_icd(yd, sig, 1, sp, x)
        torch.cuda.synchronize()
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[2])
    assert rel_l2(xs[1], plan.icd(y, sig, 1, 3)[0]) <= 1e-4


def test_icd_from_a_start_image():
    s = ragged_scene()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=4)
    x0 = 0.5 * x_true.reshape(-1)
    x_ref, _, cost_ref = plan.icd(y, sig, 2, 3, x0=x0)
    geo = M.Geometry(s)
    x = to_dev(x0)
    out = geo.reconstruct_icd(to_dev(y), sig, 2, 3, x, x_given=True, want_cost=True)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_ref) <= 1e-4
    assert np.allclose(out["cost"], cost_ref, rtol=1e-4)


def test_icd_bf16_storage():
    s = S.cfg0().copy(precision="bf16")
    plan, x_true, g_true, y, sig = oracle_data(s, seed=3)
    x_ref, _, _ = plan.icd(y, sig, 2, 2)
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    geo.reconstruct_icd(to_dev(y, torch.bfloat16), sig, 2, 2, x)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_ref) <= 1e-2


@pytest.mark.parametrize("spacing", [0, 1])
def test_icd_rejects_spacing_below_two(spacing):
    s = S.cfg0()
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    with pytest.raises(M.MbirError) as ei:
        geo.reconstruct_icd(torch.zeros(s.K * s.M, device=DEV), 0.1, 1, spacing, x)
    assert ei.value.code == -1
