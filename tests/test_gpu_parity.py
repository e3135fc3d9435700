"""CUDA path against the FP64 oracle, element by element (needs a GB300).

Gates: pair delays within 1e-3 sample (RMS <= 2e-5 sample), FP32 A x and
A^T r within relative L2 1e-5, BF16 storage within 1e-2, projection and
prior gradient within 1e-5, and the MAP image after the fixed iteration count
within relative L2 1e-4 of the oracle's.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_09703_gb300 import synth as S
from tests.helpers import many_layer_scene, oracle_data, ragged_scene, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_09703_gb300 import build as B  # noqa: E402

B.build()
from paper_2202_09703_gb300 import mbir as M  # noqa: E402

DEV = torch.device("cuda:0")
MODES = ["otf", "tab", "tab-norec"]


def make_geo(s, mode="auto", **kw):
    """'tab-norec' is TAB mode without the sorted record list (on-the-fly A x records)."""
    if mode == "tab-norec":
        return M.Geometry(s, mode="tab", records=False, **kw)
    return M.Geometry(s, mode=mode, **kw)


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV)


def gpu_forward(geo, x):
    s = geo.scene
    dt = torch.bfloat16 if geo.precision == "bf16" else torch.float32
    y = torch.empty(s.K * s.M, dtype=dt, device=DEV)
    geo.forward(to_dev(x), y)
    torch.cuda.synchronize()
    return y.float().cpu().numpy().reshape(s.K, s.M)


def gpu_backproject(geo, r):
    s = geo.scene
    dt = torch.bfloat16 if geo.precision == "bf16" else torch.float32
    b = torch.empty(s.N, dtype=torch.float32, device=DEV)
    geo.backproject(to_dev(r, dt), b)
    torch.cuda.synchronize()
    return b.cpu().numpy()


# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", ["cfg0", "cfg1"])
def test_pulse_table_matches_oracle(cfg):
    s = S.CONFIGS[cfg]()
    geo = M.Geometry(s)
    assert geo.info.pulse_support == O.Geometry(s).pulse_support()
    assert geo.info.gamma_max_s == pytest.approx(O.Geometry(s).gamma_max(), rel=1e-14)
    t_gpu = geo.pulse_table()
    t_orc = O.Geometry(s).pulse_table()
    assert np.max(np.abs(t_gpu - t_orc)) < 1e-10


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_pair_delays_weights_attenuation(mode, scene_fn):
    s = scene_fn()
    geo = make_geo(s, mode)
    plan = O.Plan(s)
    pix = np.repeat(np.arange(s.N), s.K)
    ks = np.tile(np.arange(s.K), s.N)
    T, g, w = geo.pair_quantities(pix, ks)
    ref = np.array([plan.pair(int(v), int(k)) for v, k in zip(pix, ks)])
    dT = (T - ref[:, 0] * s.fs)
    assert np.max(np.abs(dT)) <= 1e-3
    assert math.sqrt(np.mean(dT ** 2)) <= 2e-5
    # gamma enters H through exp(-gamma f): its effect on A scales with f_c * w.
    # (Grazing legs have a large relative gamma error but cos^beta ~ 0 there.)
    assert np.max(s.fc * np.abs(g - ref[:, 1]) * ref[:, 2]) <= 1e-6
    assert np.max(np.abs(w - ref[:, 2])) <= 2e-6


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene,
                                      lambda: S.small_scene(n_layers=1, w=32, h=16, n_tx=2, n_rx=3, M=200)])
def test_forward_parity(mode, scene_fn):
    s = scene_fn()
    geo = make_geo(s, mode)
    plan = O.Plan(s)
    for x in (S.phantom(s, 1), S.random_vector(s.N, 2).reshape(s.img_h, s.img_w)):
        y_ref = plan.forward(x)
        y = gpu_forward(geo, x)
        assert rel_l2(y, y_ref) <= 1e-5


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_backproject_parity(mode, scene_fn):
    s = scene_fn()
    geo = make_geo(s, mode)
    plan = O.Plan(s)
    r = S.random_vector(s.K * s.M, 3)
    b_ref = plan.backproject(r)
    b = gpu_backproject(geo, r)
    assert rel_l2(b, b_ref) <= 1e-5


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n_layers", [5, 6])
def test_many_layer_scenes_match_oracle(mode, n_layers):
    """Five and six layers (eq. 4-6 with L > 4, served by the kernels' 8-layer
    instantiation): delays, weights and attenuation of every pair, A x and
    A^T r against the oracle."""
    s = many_layer_scene(n_layers)
    geo = make_geo(s, mode)
    plan = O.Plan(s)
    pix = np.repeat(np.arange(s.N), s.K)
    ks = np.tile(np.arange(s.K), s.N)
    T, g, w = geo.pair_quantities(pix, ks)
    ref = np.array([plan.pair(int(v), int(k)) for v, k in zip(pix, ks)])
    dT = T - ref[:, 0] * s.fs
    assert np.max(np.abs(dT)) <= 1e-3
    assert math.sqrt(np.mean(dT ** 2)) <= 2e-5
    assert np.max(np.abs(w - ref[:, 2])) <= 2e-6
    assert np.max(s.fc * np.abs(g - ref[:, 1]) * ref[:, 2]) <= 1e-6
    rows = np.arange(s.img_h)
    z = (rows + 0.5) * s.pitch
    assert z[-1] > sum(L.thickness for L in s.layers[:-1])      # pixels in the last layer too
    for x in (S.phantom(s, 4), S.random_vector(s.N, 43).reshape(s.img_h, s.img_w)):
        assert rel_l2(gpu_forward(geo, x), plan.forward(x)) <= 1e-5
    r = S.random_vector(s.K * s.M, 44)
    assert rel_l2(gpu_backproject(geo, r), plan.backproject(r)) <= 1e-5


@pytest.mark.parametrize("mode", MODES)
def test_adjoint_identity_on_gpu(mode):
    s = S.cfg0()
    geo = make_geo(s, mode)
    x = S.random_vector(s.N, 4)
    r = S.random_vector(s.K * s.M, 5)
    Ax = gpu_forward(geo, x).reshape(-1)
    ATr = gpu_backproject(geo, r)
    lhs, rhs = float(Ax.astype(np.float64) @ r), float(x @ ATr.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("mode", MODES)
def test_outputs_are_bitwise_reproducible(mode):
    s = S.cfg0()
    geo = make_geo(s, mode)
    x = S.phantom(s, 0)
    r = S.random_vector(s.K * s.M, 6)
    assert np.array_equal(gpu_forward(geo, x), gpu_forward(geo, x))
    assert np.array_equal(gpu_backproject(geo, r), gpu_backproject(geo, r))
    # a second handle of the same geometry gives the same bits
    geo2 = make_geo(s, mode)
    assert np.array_equal(gpu_forward(geo, x), gpu_forward(geo2, x))


def test_forward_window_does_not_change_output_bits():
    """CUDA-core A x windows of 1, 2 and 4 spans per warp give identical
    outputs, and the creation-time autotuner reports the three timings it chose
    from (it runs when that kernel is the geometry's A x; with the tensor-core
    A x the timings are not taken)."""
    s = S.cfg0()
    assert list(make_geo(s, "tab").info.forward_window_ms) == [0.0, 0.0, 0.0]
    geo = make_geo(s, "tab", tensor_cores=False)
    info = geo.info
    assert info.forward_window_spans in (1, 2, 4)
    ms = list(info.forward_window_ms)
    assert all(t > 0 for t in ms)
    assert ms[(1, 2, 4).index(info.forward_window_spans)] == min(ms)
    x = S.random_vector(s.N, 21).reshape(s.img_h, s.img_w)
    outs = []
    for spans in (1, 2, 4):
        geo.set_forward_window(spans)
        assert geo.info.forward_window_spans == spans
        outs.append(gpu_forward(geo, x))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    plan = O.Plan(s)
    assert rel_l2(outs[0], plan.forward(x)) <= 1e-5
    with pytest.raises(M.MbirError):
        geo.set_forward_window(3)


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_bf16_tensor_core_adjoint_matches_cuda_core_adjoint_and_oracle(scene_fn):
    """BF16 form: A^T on the tensor cores (per-tile correlation GEMM + four
    corners per pair) against the CUDA-core adjoint on the same stored BF16
    residual and table, and against the FP64 oracle.  The tensor-core form
    reads its pair weights from the 12 B packed records (w rounded to FP16,
    2^-12 relative), the CUDA-core adjoint from the legs in FP32: their
    difference is at that level, far inside the BF16 form's oracle bound."""
    s = scene_fn().copy(precision="bf16")
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.adjoint_tensor_cores == 1 and cc.info.adjoint_tensor_cores == 0
    plan = O.Plan(s)
    for seed in (31, 32):
        r = S.random_vector(s.K * s.M, seed)
        b_tc, b_cc = gpu_backproject(tc, r), gpu_backproject(cc, r)
        assert rel_l2(b_tc, b_cc) <= 1e-3
        assert rel_l2(b_tc, plan.backproject(r)) <= 1e-2
    # reproducible: the per-pixel fixed-point sums do not depend on the order of the additions
    assert np.array_equal(gpu_backproject(tc, r), b_tc)


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene,
                                      lambda: S.small_scene(n_layers=1, w=32, h=16, n_tx=2, n_rx=3, M=200)])
def test_fp32_tensor_core_adjoint_matches_cuda_core_adjoint_and_oracle(scene_fn):
    """FP32 form: A^T on the tensor cores with the residual window and the
    table each scaled by a power of two and split into two FP16 parts (three
    products kept, error below FP32 rounding), against the CUDA-core adjoint
    and the FP64 oracle."""
    s = scene_fn()
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.adjoint_tensor_cores == 1 and cc.info.adjoint_tensor_cores == 0
    plan = O.Plan(s)
    for seed in (51, 52):
        r = S.random_vector(s.K * s.M, seed)
        b_tc, b_cc = gpu_backproject(tc, r), gpu_backproject(cc, r)
        assert rel_l2(b_tc, b_cc) <= 1e-6
        assert rel_l2(b_tc, plan.backproject(r)) <= 1e-5
    assert np.array_equal(gpu_backproject(tc, r), b_tc)


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene,
                                      lambda: S.small_scene(n_layers=1, w=32, h=16, n_tx=2, n_rx=3, M=200),
                                      lambda: S.small_scene(n_layers=2, w=24, h=20, n_tx=3, n_rx=2, M=180,
                                                            atten=False)])
def test_fp32_tensor_core_forward_matches_cuda_core_forward_and_oracle(scene_fn):
    """FP32 form: A x on the tensor cores (per-(sample, table row) sums of
    weight x x in FP32 and the table, each scaled by a power of two and split
    into two FP16 parts, three products kept, two phase-aligned halves of the
    table rows) against the CUDA-core A x and the FP64 oracle; the last scene
    has one gamma plane."""
    s = scene_fn()
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.forward_tensor_cores == 1 and cc.info.forward_tensor_cores == 0
    plan = O.Plan(s)
    for x in (S.phantom(s, 2), S.random_vector(s.N, 34).reshape(s.img_h, s.img_w)):
        y_tc, y_cc = gpu_forward(tc, x), gpu_forward(cc, x)
        assert rel_l2(y_tc, y_cc) <= 1e-6
        assert rel_l2(y_tc, plan.forward(x)) <= 1e-5
    assert np.array_equal(gpu_forward(tc, x), y_tc)


@pytest.mark.parametrize("case", ["zero", "one_pixel", "tiny", "huge"])
def test_fp32_tensor_core_forward_scaling_edge_cases(case):
    """The FP32 tensor-core A x scales each (tile, row half) of per-sample sums by a power of two before
    the FP16 split: an all-zero image gives exact zeros, and a single pixel or images at 1e-30 / 1e30
    (far outside FP16's range) match the CUDA-core A x to FP32 accuracy."""
    s = ragged_scene()
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    x = S.phantom(s, 3).astype(np.float64)
    if case == "zero":
        x = np.zeros_like(x)
    elif case == "one_pixel":
        x = np.zeros_like(x)
        x[s.img_h // 2, s.img_w // 3] = 0.7
    elif case == "tiny":
        x = x * 1e-30
    else:
        x = x * 1e30
    y_tc, y_cc = gpu_forward(tc, x), gpu_forward(cc, x)
    assert np.all(np.isfinite(y_tc))
    if case == "zero":
        assert not np.any(y_tc)
    else:
        assert rel_l2(y_tc, y_cc) <= 1e-6


@pytest.mark.parametrize("precision,bound", [("fp32", 1e-6), ("bf16", 4e-3)])
@pytest.mark.parametrize("case", ["first_layer", "deepest_layer", "zero"])
def test_tensor_core_forward_single_pixels_per_ascan(precision, bound, case):
    """One pixel in the first layer, one in the deepest, and an all-zero image:
    every A-scan of the tensor-core A x against the CUDA-core A x of the same
    form on its own (an A-scan whose only record falls in a dropped plane or
    column range would be far off), and against the oracle.  The BF16 form
    rounds each per-(sample, table row) sum once to BF16 (2^-9 relative)."""
    s = ragged_scene().copy(precision=precision)
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.forward_tensor_cores == 1 and cc.info.forward_tensor_cores == 0
    x = np.zeros((s.img_h, s.img_w))
    if case == "first_layer":
        x[1, s.img_w // 2 + 3] = 0.8
    elif case == "deepest_layer":
        x[s.img_h - 1, s.img_w // 3] = -0.6
    y_tc, y_cc = gpu_forward(tc, x), gpu_forward(cc, x)
    if case == "zero":
        assert not np.any(y_tc) and not np.any(y_cc)
        return
    y_ref = O.Plan(s).forward(x)
    live = 0
    for k in range(s.K):
        nc = np.linalg.norm(y_cc[k])
        if nc == 0.0:
            assert not np.any(y_tc[k])
            continue
        live += 1
        assert np.linalg.norm(y_tc[k] - y_cc[k]) <= bound * nc, k
        assert rel_l2(y_tc[k], y_ref[k]) <= (1e-5 if precision == "fp32" else 1e-2), k
    assert live >= s.K // 2


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_bf16_tensor_core_forward_matches_cuda_core_forward_and_oracle(scene_fn):
    """BF16 form: A x on the tensor cores (per-(sample, table row) sums of
    weight x x rounded once to BF16, a table GEMM and anti-diagonal sums)
    against the CUDA-core A x and the FP64 oracle.  The one extra BF16
    rounding of the sums bounds their difference at the BF16 level."""
    s = scene_fn().copy(precision="bf16")
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.forward_tensor_cores == 1 and cc.info.forward_tensor_cores == 0
    plan = O.Plan(s)
    for x in (S.phantom(s, 2), S.random_vector(s.N, 33).reshape(s.img_h, s.img_w)):
        y_tc, y_cc = gpu_forward(tc, x), gpu_forward(cc, x)
        assert rel_l2(y_tc, y_cc) <= 5e-3
        assert rel_l2(y_tc, plan.forward(x)) <= 1e-2
    assert np.array_equal(gpu_forward(tc, x), y_tc)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tensor_core_variants_are_timed_and_give_the_same_bits(precision):
    """At creation each tensor-core pool's two variants are timed once and
    the faster one kept; every combination gives the same output bits."""
    s = ragged_scene().copy(precision=precision)
    geo = make_geo(s, "tab")
    info = geo.info
    ms = list(info.tc_variant_ms)
    assert all(t > 0 for t in ms)
    assert ms[info.tc_forward_variant] == min(ms[0], ms[1])
    assert ms[2 + info.tc_adjoint_variant] == min(ms[2], ms[3])
    x = S.phantom(s, 4)
    r = S.random_vector(s.K * s.M, 44)
    outs = []
    for fv in (0, 1):
        for bv in (0, 1):
            geo.set_tensor_core_variants(fv, bv)
            assert geo.info.tc_forward_variant == fv and geo.info.tc_adjoint_variant == bv
            outs.append((gpu_forward(geo, x), gpu_backproject(geo, r)))
    for y, b in outs[1:]:
        assert np.array_equal(y, outs[0][0]) and np.array_equal(b, outs[0][1])
    with pytest.raises(M.MbirError):
        geo.set_tensor_core_variants(2, 0)
    cc = make_geo(s, "tab", tensor_cores=False)
    with pytest.raises(M.MbirError):
        cc.set_tensor_core_variants(1, -1)


def _gapped_scene():
    """Two columns of pixels 20 mm apart in water: consecutive rows' echoes
    are some 250 samples apart, so every A-scan's 128-sample tiles with records
    alternate with tiles without any (the first and the last ones empty too)."""
    s = S.small_scene(n_layers=1, w=2, h=5, n_tx=2, n_rx=2, M=1500, name="tiny_gapped")
    return s.copy(pitch=20e-3, tx_x=S.centred_positions(2, 2e-3, 20e-3))


@pytest.mark.parametrize("precision,bound", [("fp32", 1e-6), ("bf16", 5e-3)])
def test_tensor_core_applies_with_empty_tiles_between_records(precision, bound):
    """The tensor-core A x holds its output in a ring of samples that it
    flushes as tiles complete; tiles without records between tiles with
    records take a separate path.  Both applies against the CUDA-core ones
    and the oracle on a scene made of such gaps."""
    s = _gapped_scene().copy(precision=precision)
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.forward_tensor_cores == 1 and tc.info.adjoint_tensor_cores == 1
    plan = O.Plan(s)
    n0 = np.array([[np.floor(plan.pair(v, k)[0] * s.fs) for v in range(s.N)] for k in range(s.K)])
    for k in range(s.K):
        live = set((n0[k] // 128).astype(int))
        assert any(t not in live for t in range(min(live), max(live)))   # a gap between tiles with records
    for seed in (2, 3):
        x = S.random_vector(s.N, seed).reshape(s.img_h, s.img_w)
        y_tc, y_cc = gpu_forward(tc, x), gpu_forward(cc, x)
        assert rel_l2(y_tc, y_cc) <= bound
        assert rel_l2(y_tc, plan.forward(x)) <= (1e-5 if precision == "fp32" else 1e-2)
        r = S.random_vector(s.K * s.M, seed + 10)
        b_tc = gpu_backproject(tc, r)
        assert rel_l2(b_tc, gpu_backproject(cc, r)) <= (1e-6 if precision == "fp32" else 1e-3)
        assert rel_l2(b_tc, plan.backproject(r)) <= (1e-5 if precision == "fp32" else 1e-2)


@pytest.mark.parametrize("precision,per_pair", [("fp32", 16), ("bf16", 12)])
def test_tensor_core_records_are_packed(precision, per_pair):
    """The tensor-core forms keep only the packed records: 16 B per active
    pair in the FP32 form and 12 B in the BF16 form, against 24 B per pair
    for the sorted records of the CUDA-core A x; one record per active pair."""
    s = S.cfg0().copy(precision=precision)
    tc = make_geo(s, "tab")
    cc = make_geo(s, "tab", tensor_cores=False)
    assert tc.info.forward_tensor_cores == 1 and cc.info.forward_tensor_cores == 0
    pairs, _ = tc.count_taps()
    assert tc.info.n_records == cc.info.n_records == pairs > 0
    assert tc.info.record_bytes == per_pair * pairs
    assert cc.info.record_bytes == 24 * pairs


def test_otf_and_tab_modes_agree():
    s = S.cfg0()
    x = S.phantom(s, 3)
    a = gpu_forward(make_geo(s, "otf"), x)
    b = gpu_forward(make_geo(s, "tab"), x)
    c = gpu_forward(make_geo(s, "tab-norec"), x)
    assert rel_l2(a, b) <= 2e-6 and rel_l2(c, b) <= 2e-6


def test_bf16_storage_within_stated_error():
    s = S.cfg0().copy(precision="bf16")
    geo = M.Geometry(s)
    plan = O.Plan(s)
    x = S.phantom(s, 1)
    assert rel_l2(gpu_forward(geo, x), plan.forward(x)) <= 1e-2
    r = S.random_vector(s.K * s.M, 7)
    assert rel_l2(gpu_backproject(geo, r), plan.backproject(r)) <= 1e-2


# --------------------------------------------------------------------------
# full-size 256x512 workload on sampled outputs
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg1_plan():
    s = S.cfg1()
    return s, O.Plan(s)


@pytest.mark.parametrize("mode", MODES)
def test_cfg1_forward_sampled_ascans(cfg1_plan, mode):
    s, plan = cfg1_plan
    geo = make_geo(s, mode)
    for x in (S.phantom(s, 0), S.random_vector(s.N, 12).reshape(s.img_h, s.img_w)):
        y = gpu_forward(geo, x)
        for k in (0, 517, s.K - 1):
            y_ref = plan.forward(x, k, k + 1)[0]
            assert rel_l2(y[k], y_ref) <= 1e-5


@pytest.mark.parametrize("mode", MODES)
def test_cfg1_backproject_sampled_pixels(mode):
    s = S.cfg1()
    geo = make_geo(s, mode)
    r = S.random_vector(s.K * s.M, 8)
    b = gpu_backproject(geo, r)
    rng = S.SplitMix64(99)
    pix = np.unique(rng.integers(0, 300 * s.img_w, 160))     # rows inside the record
    plan = O.Plan(s, pix=pix)
    b_ref = plan.backproject(r)
    assert rel_l2(b[pix], b_ref) <= 1e-5


@pytest.mark.parametrize("cfg", ["cfg1", "cfg2"])
def test_full_size_delays_on_sampled_pairs(cfg):
    """Delays at the full workloads' magnitudes (up to ~4000 samples in the
    256x512 scan and ~8000 in the 512x1024 one, where eq. 4's rounding bites
    hardest): 4096 random (pixel, A-scan) pairs with a non-zero weight against
    the oracle, max 1e-3 sample and RMS 2e-5 sample; weights and attenuation
    as for the small scenes."""
    s = S.CONFIGS[cfg]().copy(precision="fp32")
    geo = make_geo(s, "tab")
    rng = S.SplitMix64(31 if cfg == "cfg1" else 32)
    pix = rng.integers(0, s.N - 1, 4096)
    ks = rng.integers(0, s.K - 1, 4096)
    upix, slot = np.unique(pix, return_inverse=True)
    plan = O.Plan(s, pix=upix)
    T, g, w = geo.pair_quantities(pix, ks)
    ref = np.array([plan.pair(int(sl), int(k)) for sl, k in zip(slot, ks)])
    act = ref[:, 2] > 0
    assert act.sum() > 1000
    dT = (T - ref[:, 0] * s.fs)[act]
    assert np.max(ref[act, 0] * s.fs) > 0.8 * s.M          # delays near the end of the record are included
    assert np.max(np.abs(dT)) <= 1e-3
    assert math.sqrt(np.mean(dT ** 2)) <= 2e-5
    assert np.max(np.abs(w - ref[:, 2])) <= 2e-6
    assert np.max(s.fc * np.abs(g - ref[:, 1]) * ref[:, 2]) <= 1e-6


def test_cfg2_fp32_sampled_ascans_and_pixels():
    """The 512x1024 workload (128 Tx x 32 Rx, 4096 samples) in the FP32 form,
    the benchmark's configuration: A x on the first, middle and last A-scans
    and A^T r on 64 pixels (corners, centre and random) against the oracle at
    relative L2 1e-5."""
    s = S.cfg2().copy(precision="fp32")
    geo = make_geo(s, "tab")
    assert geo.info.forward_tensor_cores == 1 and geo.info.adjoint_tensor_cores == 1
    plan = O.Plan(s)
    x = S.phantom(s, 0)
    y = gpu_forward(geo, x)
    for k in (0, s.K // 2, s.K - 1):
        assert rel_l2(y[k], plan.forward(x, k, k + 1)[0]) <= 1e-5, k
    r = S.random_vector(s.K * s.M, 18)
    b = gpu_backproject(geo, r)
    rng = S.SplitMix64(6)
    pix = np.unique(np.concatenate([[0, s.img_w - 1, s.N // 2 + s.img_w // 2, s.N - s.img_w, s.N - 1],
                                    rng.integers(0, s.N - 1, 59)]))
    bp = O.Plan(s, pix=pix)
    assert rel_l2(b[pix], bp.backproject(r)) <= 1e-5


# --------------------------------------------------------------------------
# direct arrivals, prior, MAP iteration
# --------------------------------------------------------------------------
def test_projection_parity():
    s = ragged_scene()
    geo = M.Geometry(s)
    plan = O.Plan(s)
    r = S.random_vector(s.K * s.M, 9)
    e_ref, g_ref = plan.project(r)
    e = torch.empty(s.K * s.M, device=DEV)
    gk = torch.empty(s.K, device=DEV)
    geo.project(to_dev(r), e, gk)
    torch.cuda.synchronize()
    assert rel_l2(e.cpu().numpy(), e_ref) <= 1e-6
    assert rel_l2(gk.cpu().numpy(), g_ref) <= 1e-5


def test_prior_gradient_parity():
    s = S.cfg1().copy(img_w=48, img_h=40)
    geo = M.Geometry(s)
    x = S.random_vector(s.N, 10, -0.5, 0.5)
    x[::7] = 0.0
    out = torch.empty(s.N, device=DEV)
    geo.prior_gradient(to_dev(x), out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.prior_grad(s, x)) <= 1e-5


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_reconstruct_matches_oracle(scene_fn):
    s = scene_fn()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=1)
    n_iter = s.n_iter
    x_ref, g_ref, cost_ref, gn_ref = plan.reconstruct(y, sig, n_iter)
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    g = torch.empty(s.K, device=DEV)
    out = geo.reconstruct(to_dev(y), sig, n_iter, x, g=g, want_cost=True)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    assert rel_l2(xg, x_ref) <= 1e-4
    assert np.allclose(out["cost"], cost_ref, rtol=1e-4)
    assert np.all(np.diff(out["cost"]) <= 1e-6 * abs(out["cost"][0]))
    if s.direct_arrival:
        assert rel_l2(g.cpu().numpy(), g_ref) <= 1e-4


def test_reconstruct_host_buffers_match_device_call():
    s = S.cfg0()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=2)
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    geo.reconstruct(to_dev(y), sig, 5, x)
    torch.cuda.synchronize()
    yh = torch.as_tensor(y.astype(np.float32)).reshape(-1).pin_memory()
    xh = torch.empty(s.N, dtype=torch.float32).pin_memory()
    geo.reconstruct_host(yh, sig, 5, xh)
    assert np.array_equal(xh.numpy(), x.cpu().numpy())


def test_nonfinite_data_is_reported():
    s = S.cfg0()
    geo = M.Geometry(s)
    y = np.zeros((s.K, s.M), np.float32)
    y[3, 7] = np.nan
    x = torch.empty(s.N, device=DEV)
    with pytest.raises(M.MbirError) as ei:
        geo.reconstruct(to_dev(y), 0.1, 3, x)
    assert ei.value.code == -4


def test_invalid_prior_is_rejected():
    s = S.cfg0().copy(prior=S.Prior(p=2.0, q=2.0))
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    with pytest.raises(M.MbirError) as ei:
        geo.reconstruct(torch.zeros(s.K * s.M, device=DEV), 0.1, 3, x)
    assert ei.value.code == -1


# --------------------------------------------------------------------------
# precision form at full size: 512 x 1024 image, 128 Tx x 32 Rx, 4096 samples
# --------------------------------------------------------------------------
def test_cfg2_bf16_sampled_ascans_and_pixels():
    s = S.cfg2()
    assert s.precision == "bf16"
    geo = M.Geometry(s)
    plan = O.Plan(s)
    x = S.random_vector(s.N, 14).reshape(s.img_h, s.img_w)
    y = gpu_forward(geo, x)
    for k in (0, s.K // 2 + 7):
        assert rel_l2(y[k], plan.forward(x, k, k + 1)[0]) <= 1e-2
    r = S.random_vector(s.K * s.M, 15)
    b = gpu_backproject(geo, r)
    rng = S.SplitMix64(5)
    pix = np.unique(rng.integers(0, s.N - 1, 48))
    bp = O.Plan(s, pix=pix)
    assert rel_l2(b[pix], bp.backproject(r)) <= 1e-2


@pytest.mark.parametrize("M_len", [4096, 9000])
def test_long_records_use_smaller_adjoint_configurations(M_len):
    """Long A-scans shrink the adjoint's residual ring (two workers x two
    stages, then one worker) to fit shared memory; results are unchanged."""
    s = S.small_scene(n_layers=2, w=40, h=24, n_tx=2, n_rx=3, M=M_len, direct=True, name="tiny_long")
    geo = make_geo(s, "tab")
    plan = O.Plan(s)
    r = S.random_vector(s.K * s.M, 16)
    assert rel_l2(gpu_backproject(geo, r), plan.backproject(r)) <= 1e-5
    x = S.random_vector(s.N, 17)
    assert rel_l2(gpu_forward(geo, x), plan.forward(x)) <= 1e-5


def test_records_too_long_for_shared_memory_are_refused():
    s = S.small_scene(n_layers=2, w=16, h=8, n_tx=1, n_rx=1, M=16000, name="tiny_toolong")
    with pytest.raises(M.MbirError) as ei:
        M.Geometry(s, mode="tab")
    assert ei.value.code == -7


# --------------------------------------------------------------------------
# image error against the oracle, per configuration and precision
# --------------------------------------------------------------------------
def _gpu_reconstruct(s, y, sig, n_iter):
    geo = M.Geometry(s)
    yt = to_dev(np.asarray(y, np.float32).reshape(-1))
    if geo.precision == "bf16":
        yt = yt.to(torch.bfloat16)
    x = torch.empty(s.N, device=DEV)
    geo.reconstruct(yt, sig, n_iter, x)
    torch.cuda.synchronize()
    geo.close()
    return x.cpu().numpy()


@pytest.mark.parametrize("precision,tensor_cores", [("fp32", True), ("bf16", True), ("fp32", False)])
def test_fused_update_stencil_gives_the_same_bits(precision, tensor_cores):
    """mbir_reconstruct applies each step's MAP update where the next
    iteration reads it (x in the prior stencil, e in the adjoint's max |e|
    pass or a pass of its own); with the per-iteration cost recorded it
    applies them at the end of the iteration.  Same arithmetic: the images
    must agree bit for bit, from x = 0 and from a given start image, and the
    fused run must match the oracle's reconstruction."""
    s = ragged_scene().copy(precision=precision)
    plan = O.Plan(s)
    y = plan.forward(S.phantom(s, 5)) + 0.02 * S.unit_noise(s, 5)
    geo = M.Geometry(s, mode="tab", tensor_cores=tensor_cores)
    assert geo.info.adjoint_tensor_cores == (1 if tensor_cores else 0)
    yt = to_dev(np.asarray(y, np.float32).reshape(-1))
    if precision == "bf16":
        yt = yt.to(torch.bfloat16)
    x0 = to_dev(S.random_vector(s.N, 6) * 0.1)
    for given in (False, True):
        xa = x0.clone() if given else torch.empty(s.N, device=DEV)
        xb = x0.clone() if given else torch.empty(s.N, device=DEV)
        geo.reconstruct(yt, 0.02, 7, xa, x_given=given)
        out = geo.reconstruct(yt, 0.02, 7, xb, x_given=given, want_cost=True)
        torch.cuda.synchronize()
        assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy()), given
        assert np.all(np.diff(out["cost"]) <= 1e-6 * abs(out["cost"][0]))
    x_ref = plan.reconstruct(y, 0.02, 7)[0].reshape(-1)
    xg = torch.empty(s.N, device=DEV)
    geo.reconstruct(yt, 0.02, 7, xg)
    torch.cuda.synchronize()
    assert rel_l2(xg.cpu().numpy(), x_ref) <= (1e-4 if precision == "fp32" else 1e-2)


def test_cfg1_reconstruction_matches_oracle():
    """The 4-layer 256x512 workload in FP32: three MAP iterations against the
    FP64 oracle's (measured 9.5e-8 relative)."""
    s = S.cfg1()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=1)
    x_ref = np.asarray(plan.reconstruct(y, sig, 3)[0]).reshape(-1)
    assert rel_l2(_gpu_reconstruct(s, y, sig, 3), x_ref) <= 1e-4


@pytest.mark.slow
def test_cfg1_full_reconstruction_matches_oracle():
    """The 4-layer 256x512 workload in FP32 with its full 50 MAP iterations
    against the FP64 oracle's image (relative L2 1e-4), and the costs per
    iteration."""
    s = S.cfg1()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=1)
    x_ref, g_ref, cost_ref, _ = plan.reconstruct(y, sig, s.n_iter)
    geo = M.Geometry(s)
    x = torch.empty(s.N, device=DEV)
    out = geo.reconstruct(to_dev(np.asarray(y, np.float32).reshape(-1)), sig, s.n_iter, x, want_cost=True)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), np.asarray(x_ref).reshape(-1)) <= 1e-4
    assert np.allclose(out["cost"], cost_ref, rtol=1e-4)


def test_bf16_reconstruction_image_error_against_oracle():
    """BF16 storage form of the 2-layer 64x64 workload, 20 iterations, against
    the FP64 oracle (measured 1.4e-3 relative)."""
    s = S.cfg0().copy(precision="bf16")
    plan, x_true, g_true, y, sig = oracle_data(s, seed=1)
    x_ref = np.asarray(plan.reconstruct(y, sig, s.n_iter)[0]).reshape(-1)
    assert rel_l2(_gpu_reconstruct(s, y, sig, s.n_iter), x_ref) <= 1e-2


def test_cfg2_bf16_image_against_fp32_form():
    """The 512x1024 precision workload, 50 iterations: the BF16 storage form
    (tensor cores) against the FP32 form on the same data (measured 1.8e-3),
    both equally far from the phantom."""
    s16 = S.cfg2()
    s32 = s16.copy(precision="fp32")
    g32 = M.Geometry(s32)
    xt = np.asarray(S.phantom(s32, 0), np.float64).reshape(-1)
    y = torch.empty(s32.K * s32.M, device=DEV)
    g32.forward(to_dev(xt), y)      # data from the FP32 operator (pinned to the oracle elsewhere)
    sig = float(np.sqrt(float((y.double() ** 2).sum()) / (100 * s32.K * s32.M)))
    y += sig * to_dev(S.unit_noise(s32, 0).reshape(-1))
    y_np = y.cpu().numpy()
    g32.close()
    x32 = _gpu_reconstruct(s32, y_np, sig, s32.n_iter)
    x16 = _gpu_reconstruct(s16, y_np, sig, s16.n_iter)
    assert rel_l2(x16, x32) <= 1e-2
    e32, e16 = rel_l2(x32, xt), rel_l2(x16, xt)
    assert abs(e16 - e32) <= 1e-2 * e32


@pytest.mark.parametrize("scene_fn", [S.cfg0, ragged_scene])
def test_saft_image_matches_oracle(scene_fn):
    """SAFT (delay-and-sum) is A^T y with the beam profile phi = 1: the GPU
    adjoint of a beta = 0 geometry against the oracle's, on data made with
    the beam model."""
    s = scene_fn()
    plan, x_true, g_true, y, sig = oracle_data(s, seed=3)
    s0 = s.copy(beta=0.0)
    geo = make_geo(s0, "tab")
    assert rel_l2(gpu_backproject(geo, y), O.Plan(s0).backproject(y)) <= 1e-5


# --------------------------------------------------------------------------
# beam-model variants: transmitter firing angle, first-layer apodization angle
# --------------------------------------------------------------------------
BEAM_VARIANTS = [
    ("tilt+5deg", lambda: S.cfg0().copy(firing_angle=math.radians(5.0)), "tab"),
    ("tilt-3deg ragged", lambda: ragged_scene().copy(firing_angle=math.radians(-3.0)), "tab"),
    ("first angle", lambda: ragged_scene().copy(apod_first_angle=True), "tab"),
    ("first angle otf", lambda: ragged_scene().copy(apod_first_angle=True), "otf"),
    ("first angle + tilt", lambda: S.cfg0().copy(apod_first_angle=True, firing_angle=math.radians(5.0)), "tab"),
]


@pytest.mark.parametrize("name,scene_fn,mode", BEAM_VARIANTS, ids=[v[0] for v in BEAM_VARIANTS])
def test_beam_variants_match_oracle(name, scene_fn, mode):
    s = scene_fn()
    geo = make_geo(s, mode)
    plan = O.Plan(s)
    pix = np.repeat(np.arange(s.N), s.K)
    ks = np.tile(np.arange(s.K), s.N)
    T, g, w = geo.pair_quantities(pix, ks)
    ref = np.array([plan.pair(int(v), int(k)) for v, k in zip(pix, ks)])
    assert np.max(np.abs(w - ref[:, 2])) <= 2e-6
    assert np.max(np.abs(T - ref[:, 0] * s.fs)) <= 1e-3
    x = S.random_vector(s.N, 41).reshape(s.img_h, s.img_w)
    assert rel_l2(gpu_forward(geo, x), plan.forward(x)) <= 1e-5
    r = S.random_vector(s.K * s.M, 42)
    assert rel_l2(gpu_backproject(geo, r), plan.backproject(r)) <= 1e-5


def test_tilted_transmitter_needs_tab_mode():
    s = S.cfg0().copy(firing_angle=math.radians(5.0))
    with pytest.raises(M.MbirError) as ei:
        make_geo(s, "otf")
    assert ei.value.code == -7
