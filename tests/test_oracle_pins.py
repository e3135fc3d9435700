"""Pins of the FP64 oracle against mathematics the paper fixes (no GPU).

Each test checks the oracle against something other than itself: closed forms,
brute force, an independent Fermat minimisation, the Faddeeva closed form of
the attenuated pulse, invariants (adjointness, projection, majorization) and a
dense linear solve.  A plausible slip anywhere in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import wofz

from oracle import oracle as O
from paper_2202_09703_gb300 import synth as S


def _scene_layers(speeds, thicknesses, atten=None, w=8, h=8, pitch=0.5e-3):
    s = S.small_scene(n_layers=1, w=w, h=h)
    atten = atten if atten is not None else [0.0] * len(speeds)
    s.layers = [S.Layer(t, c, a, 1000.0 + 500 * i)
                for i, (t, c, a) in enumerate(zip(thicknesses, speeds, atten))]
    s.pitch = pitch
    return s


# --------------------------------------------------------------------------
# travel time of one leg (Section 2, eq. 4-6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("h,z", [(0.0, 1e-3), (2e-3, 1.7e-3), (1e-2, 3e-3), (3e-2, 0.4e-3)])
def test_leg_one_layer_closed_form(h, z):
    s = _scene_layers([1480.0], [50e-3], atten=[0.7])
    T, gm, Th, t1 = O.Geometry(s).leg(h, z)
    dist = math.hypot(h, z)
    assert T == pytest.approx(dist / 1480.0, rel=1e-13)
    assert gm == pytest.approx(0.7e-6 * dist, rel=1e-13)      # gamma = alpha * path
    assert Th == pytest.approx(math.atan2(h, z), abs=1e-12)


def test_leg_equal_speed_split_is_invariant():
    a = _scene_layers([2000.0], [40e-3])
    b = _scene_layers([2000.0, 2000.0, 2000.0], [3e-3, 4e-3, 33e-3])
    for h, z in [(1e-3, 2e-3), (5e-3, 9e-3), (2e-2, 30e-3)]:
        Ta = O.Geometry(a).leg(h, z)[0]
        Tb = O.Geometry(b).leg(h, z)[0]
        assert Tb == pytest.approx(Ta, rel=1e-12)


def test_leg_zero_offset_is_vertical():
    s = _scene_layers([1480.0, 5900.0, 3000.0], [2e-3, 1.5e-3, 20e-3])
    z = 6e-3
    T, gm, Th, t1 = O.Geometry(s).leg(0.0, z)
    assert T == pytest.approx(2e-3 / 1480 + 1.5e-3 / 5900 + 2.5e-3 / 3000, rel=1e-14)
    assert t1 == 0.0 and Th == 0.0


def _fermat_path(speeds, eta, h):
    """Crossing points 0 = x_0 < x_1 < ... < x_L = h of the path that minimises
    sum sqrt((x_l - x_{l-1})^2 + eta_l^2) / c_l (Fermat's principle, Newton
    with backtracking on the convex total time), and that minimum."""
    c = np.asarray(speeds, float)
    e = np.asarray(eta, float)
    if len(e) == 1:
        return np.array([0.0, h]), math.hypot(h, e[0]) / c[0]
    x = h * np.cumsum(e)[:-1] / e.sum()              # straight-line start

    def total(xi):
        pts = np.concatenate([[0.0], xi, [h]])
        return float(np.sum(np.sqrt(np.diff(pts) ** 2 + e ** 2) / c))

    for _ in range(200):
        pts = np.concatenate([[0.0], x, [h]])
        u = np.diff(pts)
        d = np.sqrt(u * u + e * e)
        g1 = u / (c * d)                              # d/du of each segment
        g2 = e * e / (c * d ** 3)                     # d2/du2
        grad = g1[:-1] - g1[1:]
        Hm = np.diag(g2[:-1] + g2[1:]) - np.diag(g2[1:-1], 1) - np.diag(g2[1:-1], -1)
        step = np.linalg.solve(Hm, grad)
        t0 = total(x)
        lam = 1.0
        while total(x - lam * step) > t0 and lam > 1e-12:
            lam *= 0.5
        x = x - lam * step
        if np.max(np.abs(lam * step)) < 1e-18:
            break
    return np.concatenate([[0.0], x, [h]]), total(x)


def _fermat_time(speeds, eta, h):
    """Minimum of sum sqrt((x_l - x_{l-1})^2 + eta_l^2) / c_l over crossings."""
    return _fermat_path(speeds, eta, h)[1]


def _crossed(thick, z):
    """Layer thicknesses above depth z (the voxel's own layer cut at z)."""
    eta, top = [], 0.0
    for t in thick:
        if z <= top + t or len(eta) == len(thick) - 1:
            eta.append(z - top)
            break
        eta.append(t)
        top += t
    return eta


@pytest.mark.parametrize("speeds,thick", [
    ([1480.0, 5900.0], [2e-3, 10e-3]),
    ([1480.0, 5900.0, 3000.0], [2e-3, 1.5e-3, 20e-3]),
    ([3000.0, 1500.0, 4500.0], [1e-3, 2e-3, 20e-3]),
])
@pytest.mark.parametrize("h,z", [(1e-3, 4.5e-3), (6e-3, 8e-3), (2.5e-2, 12e-3)])
def test_leg_matches_fermat_minimum(speeds, thick, h, z):
    s = _scene_layers(speeds, thick)
    T = O.Geometry(s).leg(h, z)[0]
    eta = _crossed(thick, z)
    used = speeds[:len(eta)]
    assert T == pytest.approx(_fermat_time(used, eta, h), rel=1e-12)


@pytest.mark.parametrize("speeds,thick,atten", [
    ([1480.0, 5900.0], [2e-3, 10e-3], [0.7, 2.5]),
    ([1480.0, 5900.0, 3000.0], [2e-3, 1.5e-3, 20e-3], [0.4, 1.3, 6.0]),
    ([3000.0, 1500.0, 4500.0], [1e-3, 2e-3, 20e-3], [5.0, 0.3, 2.0]),
])
@pytest.mark.parametrize("h,z", [(1e-3, 4.5e-3), (6e-3, 8e-3), (2.5e-2, 12e-3)])
def test_leg_gamma_and_angles_follow_the_fermat_path(speeds, thick, atten, h, z):
    """Eq. 3, 6 and 12 along the ray in two and three layers: the attenuation
    gamma is the sum over crossed layers of alpha_l times the length of the
    path's segment in that layer, the first angle is atan(dx_1 / eta_1) and the
    beam-profile angle Theta is the sum of atan(dx_l / eta_l), all taken from
    the crossing points of the independent Fermat minimisation."""
    s = _scene_layers(speeds, thick, atten=atten)
    T, gm, Th, t1 = O.Geometry(s).leg(h, z)
    eta = np.asarray(_crossed(thick, z))
    assert len(eta) >= 2
    pts, Tf = _fermat_path(speeds[:len(eta)], eta, h)
    dx = np.diff(pts)
    seg = np.sqrt(dx * dx + eta * eta)
    alpha = np.asarray(atten[:len(eta)]) * 1e-6       # Np/(MHz m) -> s/m
    assert T == pytest.approx(Tf, rel=1e-12)
    assert gm == pytest.approx(float(np.sum(alpha * seg)), rel=1e-9)
    assert t1 == pytest.approx(math.atan2(dx[0], eta[0]), rel=1e-9)
    assert Th == pytest.approx(float(np.sum(np.arctan2(dx, eta))), rel=1e-9)


def test_leg_binary_search_bracket_brute_force():
    speeds, thick = [1480.0, 5900.0, 3000.0], [2e-3, 1.5e-3, 20e-3]
    s = _scene_layers(speeds, thick)
    h, z = 7e-3, 9e-3
    eta = np.array([2e-3, 1.5e-3, 9e-3 - 3.5e-3])
    c = np.array(speeds)
    crit = math.asin(c[0] / c.max())
    th1 = np.linspace(0.0, crit, 1_000_001)[:-1]
    sl = np.sin(th1)[:, None] * c[None, :] / c[0]     # Snell in closed form
    height = np.sum(eta[None, :] * sl / np.sqrt(1.0 - sl * sl), axis=1)
    i = np.searchsorted(height, h)                    # height is increasing
    _, _, _, t1 = O.Geometry(s).leg(h, z)
    assert th1[i - 1] <= t1 <= th1[i]
    assert np.all(np.diff(height) > 0)


def test_leg_calculus_and_monotonicity():
    speeds, thick = [1480.0, 5900.0, 3000.0, 4500.0], [2e-3, 1.2e-3, 4e-3, 10e-3]
    g = O.Geometry(_scene_layers(speeds, thick))
    h, z = 6e-3, 6e-3                                  # voxel in the cement layer
    T, _, _, t1 = g.leg(h, z)
    p = math.sin(t1) / speeds[0]                      # ray parameter
    dh = 1e-7
    dT_dh = (g.leg(h + dh, z)[0] - g.leg(h - dh, z)[0]) / (2 * dh)
    dT_dz = (g.leg(h, z + dh)[0] - g.leg(h, z - dh)[0]) / (2 * dh)
    assert dT_dh == pytest.approx(p, rel=1e-6)
    assert dT_dz == pytest.approx(math.sqrt(speeds[2] ** -2 - p * p), rel=1e-6)
    hs = np.linspace(0, 3e-2, 40)
    Ts = [g.leg(x, z)[0] for x in hs]
    assert np.all(np.diff(Ts) > 0)
    # depth: increasing inside each layer (dT/dz = sqrt(c^-2 - p^2) > 0); at a
    # boundary into a faster layer the Snell path may run along the fast layer
    # and the time drops, so monotonicity holds per layer only
    tops = np.cumsum([0.0] + thick)
    for lo, hi in zip(tops[:-1], tops[1:]):
        zs = np.linspace(lo + 1e-6, hi - 1e-6, 25)
        Tz = [g.leg(h, x)[0] for x in zs]
        assert np.all(np.diff(Tz) > 0)
    assert g.leg(h, 2e-3 + 1e-6)[0] < g.leg(h, 2e-3 - 1e-6)[0]


def test_transmission_two_way_normal_incidence():
    s = _scene_layers([1480.0, 5900.0, 3000.0], [2e-3, 1.5e-3, 20e-3])
    g = O.Geometry(s)
    Z = [L.density * L.speed for L in s.layers]
    t12 = 4 * Z[0] * Z[1] / (Z[0] + Z[1]) ** 2
    t23 = 4 * Z[1] * Z[2] / (Z[1] + Z[2]) ** 2
    assert g.transmission(1e-3) == 1.0
    assert g.transmission(3e-3) == pytest.approx(t12, rel=1e-15)
    assert g.transmission(10e-3) == pytest.approx(t12 * t23, rel=1e-15)


def test_transmission_conserves_energy_and_is_reciprocal():
    """The two-way normal-incidence transmission through an interface is the
    energy that is not reflected, 1 - R^2 with R = (Z2 - Z1) / (Z2 + Z1); it is
    the same with the two media swapped, 1 between matched impedances, and
    below 1 otherwise."""
    def tau_below(layers, z):
        s = _scene_layers([L[0] for L in layers], [L[1] for L in layers])
        s.layers = [S.Layer(t, c, 0.0, rho) for (c, t, rho) in layers]
        return O.Geometry(s).transmission(z)
    a, b = (1480.0, 2e-3, 1000.0), (5900.0, 2e-3, 7850.0)
    Za, Zb = a[0] * a[2], b[0] * b[2]
    R = (Zb - Za) / (Zb + Za)
    assert tau_below([a, b], 3e-3) == pytest.approx(1.0 - R * R, rel=1e-14)
    assert tau_below([b, a], 3e-3) == pytest.approx(tau_below([a, b], 3e-3), rel=1e-14)
    matched = (2960.0, 2e-3, 500.0)                       # same impedance as water (1480 x 1000)
    assert tau_below([a, matched], 3e-3) == pytest.approx(1.0, rel=1e-14)
    three = tau_below([a, b, (3000.0, 5e-3, 1900.0)], 5e-3)
    R2 = (3000.0 * 1900.0 - Zb) / (3000.0 * 1900.0 + Zb)
    assert three == pytest.approx((1.0 - R * R) * (1.0 - R2 * R2), rel=1e-14) and three < 1.0


# --------------------------------------------------------------------------
# pulse family (eq. 9-10)
# --------------------------------------------------------------------------
def _h_closed_form(scene, gamma, tau):
    """h(gamma, tau) through the Faddeeva function (scipy.special.wofz)."""
    sg = scene.n_cycles / (2 * math.sqrt(2 * math.log(2)) * scene.fc)
    Tw = math.ceil(8 * sg * scene.fs)
    tc = 0.5 * Tw / scene.fs
    A = 2 * math.pi ** 2 * sg ** 2
    beta = -gamma + 1j * 2 * math.pi * (tau - tc)
    tot = 0.0
    for a in (scene.fc, -scene.fc):
        b = a + beta / (2 * A)
        I = 0.5 * math.sqrt(math.pi / A) * math.exp(-A * a * a) * wofz(-1j * math.sqrt(A) * b)
        tot += I
    return (sg * math.sqrt(2 * math.pi) * tot).real


def test_pulse_table_no_attenuation_is_the_pulse():
    s = S.cfg0().copy(layers=[S.Layer(10e-3, 1480, 0.0, 1000), S.Layer(10e-3, 5900, 0.0, 7850)])
    g = O.Geometry(s)
    assert g.effective_G() == 1
    tab = g.pulse_table()
    Tw = g.pulse_support()
    assert Tw == 68
    taus = np.arange(s.Q * Tw + 1) / (s.fs * s.Q)
    ref = np.array([g.pulse(t) for t in taus])
    assert np.max(np.abs(tab[0] - ref)) < 1e-12


@pytest.mark.parametrize("cfg", ["cfg0", "cfg1"])
def test_pulse_is_a_two_cycle_gaussian_burst(cfg):
    """Eq. 9-10 reading: a Gaussian-modulated sinusoid whose envelope's full
    width at half maximum is n_c = 2 carrier periods, centred in its window
    of t0 = ceil(8 sigma fs) samples.  At the centre and one period either
    side the carrier is 1, so the pulse is 1 and 1/2 there; half a period
    out the carrier is -1 and the envelope exp(-(1/(2 f_c))^2 / (2 sigma^2))."""
    s = S.CONFIGS[cfg]()
    g = O.Geometry(s)
    sigma = 2.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)) * s.fc)
    Tw = g.pulse_support()
    assert Tw == math.ceil(8.0 * sigma * s.fs) == 68
    tc = 0.5 * Tw / s.fs
    assert abs(g.pulse(tc) - 1.0) < 1e-12
    for sgn in (-1.0, 1.0):
        assert abs(g.pulse(tc + sgn / s.fc) - 0.5) < 1e-12
        half = tc + sgn / (2.0 * s.fc)
        assert abs(g.pulse(half) + math.exp(-(0.5 / s.fc) ** 2 / (2.0 * sigma ** 2))) < 1e-12


def test_gamma_max_is_twice_the_two_way_vertical_loss():
    """The table's attenuation range (reading R10): twice the two-way loss of
    the vertical path to the deepest pixel centre, i.e. four times the
    one-way leg's gamma at zero offset (the leg's gamma is pinned against the
    Fermat path above); zero, and a single plane, without attenuation."""
    for s in (S.cfg0(), S.cfg1(), _scene_layers([1480.0, 3000.0, 4500.0], [2e-3, 1.5e-3, 3e-3],
                                                  atten=[2.0, 30.0, 20.0], h=12)):
        g = O.Geometry(s)
        zb = s.z0 + (s.img_h - 0.5) * s.pitch
        assert abs(g.gamma_max() - 4.0 * g.leg(0.0, zb)[1]) <= 1e-12 * g.gamma_max()
        assert g.effective_G() == s.G > 1
    s0 = S.cfg0().copy(layers=[S.Layer(10e-3, 1480, 0.0, 1000), S.Layer(10e-3, 5900, 0.0, 7850)])
    g0 = O.Geometry(s0)
    assert g0.gamma_max() == 0.0 and g0.effective_G() == 1


def test_pulse_table_matches_faddeeva_closed_form():
    s = S.cfg1()
    g = O.Geometry(s)
    tab = g.pulse_table()
    G = g.effective_G()
    gmax = g.gamma_max()
    nq = tab.shape[1]
    for gi in (0, 3, G - 1):
        gam = gi * gmax / (G - 1)
        for q in range(0, nq, 37):
            ref = _h_closed_form(s, gam, q / (s.fs * s.Q))
            assert abs(tab[gi, q] - ref) < 1e-11


def test_pulse_table_quadrature_converged_and_energy_decreases():
    s = S.cfg1()
    g = O.Geometry(s)
    t1 = g.pulse_table(1)
    t2 = g.pulse_table(2)
    assert np.max(np.abs(t1 - t2)) < 1e-12
    energy = np.sum(t1 * t1, axis=1)
    assert np.all(np.diff(energy) < 0)


def _cell_curvature_bound(s, gam_lo, dgam, tau_lo, dtau):
    """Largest |d2h/dtau2| and |d2h/dgamma2| of the closed form over one table
    cell, sampled on a 9 x 9 grid with central differences of step 1/40 cell."""
    ht, hg = dtau / 40, dgam / 40 if dgam > 0 else 0.0
    mt = mg = 0.0
    for a in np.linspace(0.0, 1.0, 9):
        for b in np.linspace(0.0, 1.0, 9):
            g0, t0 = gam_lo + a * dgam, tau_lo + b * dtau
            c = _h_closed_form(s, g0, t0)
            mt = max(mt, abs(_h_closed_form(s, g0, t0 + ht) - 2 * c + _h_closed_form(s, g0, t0 - ht)) / ht ** 2)
            if hg > 0:
                gp, gm_ = g0 + hg, max(g0 - hg, 0.0)
                mg = max(mg, abs(_h_closed_form(s, gp, t0) - 2 * c + _h_closed_form(s, gm_, t0))
                         / (hg * (gp - gm_) / 2))
    return mt, mg


def test_table_read_between_nodes_matches_the_closed_form():
    """The operator's h~(gamma, tau) between table nodes (eq. 9-10 read by the
    bilinear rule of the discrete operator): at off-node phases and between
    attenuation planes it equals the Faddeeva closed form within the
    interpolation bound dtau^2/8 max|h_tautau| + dgamma^2/8 max|h_gammagamma|.
    An interpolation weight taken on the wrong node (phi for 1 - phi, psi for
    1 - psi) or a neighbouring cell is off by a first-order term, tens of times
    that bound."""
    s = S.cfg1()
    p = O.Plan(s, pix=np.array([0]), nthreads=1)
    g = O.Geometry(s)
    G, gmax = g.effective_G(), g.gamma_max()
    Tw = g.pulse_support()
    dtau, dgam = 1.0 / (s.fs * s.Q), gmax / (G - 1)
    checked = 0
    for gi in (0, 4, G - 2):
        for q in (5 * s.Q + 3, 30 * s.Q + 11, 41 * s.Q + 7, (Tw - 3) * s.Q + 14):
            mt, mg = _cell_curvature_bound(s, gi * dgam, dgam, q * dtau, dtau)
            bound = 1.05 * (dtau ** 2 / 8 * mt + dgam ** 2 / 8 * mg) + 5e-11
            for phi in (0.27, 0.81):
                for psi in (0.0, 0.33, 0.9):
                    gam, tau = (gi + psi) * dgam, (q + phi) * dtau
                    ref = _h_closed_form(s, gam, tau)
                    assert abs(p.H(gam, tau) - ref) <= bound, (gi, q, phi, psi)
                    checked += 1
            # the read is affine along each axis inside the cell
            h1, h2, h3 = (p.H((gi + 0.4) * dgam, (q + f) * dtau) for f in (0.1, 0.45, 0.8))
            assert abs((h2 - h1) - (h3 - h2)) <= 1e-11 * (abs(h1) + abs(h3) + 1e-300)
            h1, h2, h3 = (p.H((gi + f) * dgam, (q + 0.6) * dtau) for f in (0.1, 0.45, 0.8))
            assert abs((h2 - h1) - (h3 - h2)) <= 1e-11 * (abs(h1) + abs(h3) + 1e-300)
    assert checked == 72


def test_table_read_clamps_gamma_and_honours_the_open_window():
    """Attenuation beyond the table's top reads the last plane and negative
    attenuation the first (both on a node: the closed form there); the open
    window of eq. 10 gives 0 at tau <= 0 and tau >= t0."""
    s = S.cfg1()
    p = O.Plan(s, pix=np.array([0]), nthreads=1)
    g = O.Geometry(s)
    gmax, Tw = g.gamma_max(), g.pulse_support()
    dtau = 1.0 / (s.fs * s.Q)
    for q in (3 * s.Q, 20 * s.Q + 5, 47 * s.Q + 9):
        tau = q * dtau
        assert p.H(3.0 * gmax, tau) == p.H(gmax, tau)
        assert abs(p.H(gmax, tau) - _h_closed_form(s, gmax, tau)) < 5e-11
        assert p.H(-1e-6, tau) == p.H(0.0, tau)
        assert abs(p.H(0.0, tau) - g.pulse(tau)) < 5e-11
    t0 = Tw / s.fs
    for gam in (0.0, 0.5 * gmax):
        assert p.H(gam, 0.0) == 0.0 and p.H(gam, -dtau) == 0.0
        assert p.H(gam, t0) == 0.0 and p.H(gam, t0 + 1e-12) == 0.0
        assert p.H(gam, 0.5 * dtau) != 0.0 and p.H(gam, t0 - 0.5 * dtau) != 0.0


# --------------------------------------------------------------------------
# operator (eq. 11, 13): dense matrix, adjointness, impulse response
# --------------------------------------------------------------------------
def _tiny(direct=False, layers=2, atten=True):
    return S.small_scene(n_layers=layers, w=8, h=10, n_tx=2, n_rx=2, M=160,
                         direct=direct, atten=atten)


def test_dense_matrix_matches_operators_and_adjoint():
    s = _tiny(layers=3)
    p = O.Plan(s, nthreads=2)
    A = p.dense_A()
    x = S.random_vector(s.N, 1)
    y = S.random_vector(s.K * s.M, 2)
    Ax = p.forward(x).reshape(-1)
    ATy = p.backproject(y)
    assert np.linalg.norm(A @ x - Ax) <= 1e-13 * np.linalg.norm(Ax)
    assert np.linalg.norm(A.T @ y - ATy) <= 1e-13 * np.linalg.norm(ATy)
    lhs, rhs = float(Ax @ y), float(x @ ATy)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.count_nonzero(A) > 0.05 * A.size


def test_impulse_response_single_layer_on_node():
    c, fs = 1500.0, 10e6
    s = S.small_scene(n_layers=1, w=4, h=4, n_tx=1, n_rx=1, M=128, atten=False)
    s.layers = [S.Layer(20e-3, c, 0.0, 1000.0)]
    s.rx_offset = np.array([0.0])
    col = 1
    s.tx_x = np.array([(col + 0.5) * s.pitch])
    p = O.Plan(s, nthreads=1)
    x = np.zeros((s.img_h, s.img_w))
    x[1, col] = 1.0                                 # depth 0.75 mm: 2d/c = 1 us = 10 samples
    y = p.forward(x)[0]
    g = O.Geometry(s)
    ref = np.array([g.pulse((n - 10) / fs) if 0 < n - 10 < 68 else 0.0 for n in range(s.M)])
    assert np.max(np.abs(y - ref)) < 1e-12


def test_pair_weight_is_transmission_times_apodization():
    s = _tiny(layers=2)
    p = O.Plan(s, nthreads=1)
    g = O.Geometry(s)
    v = 7 * s.img_w + 3
    r, cc = divmod(v, s.img_w)
    xc, zr = (cc + 0.5) * s.pitch, (r + 0.5) * s.pitch
    k = 3
    i, j = divmod(k, s.n_rx)
    T, gm, w = p.pair(v, k)
    lt = g.leg(xc - s.tx_x[i], zr)
    lr = g.leg(xc - s.tx_x[i] - s.rx_offset[j], zr)
    assert T == pytest.approx(lt[0] + lr[0], rel=1e-15)
    assert gm == pytest.approx(lt[1] + lr[1], rel=1e-15)
    ref_w = g.transmission(zr) * max(math.cos(lt[2]), 0) ** s.beta * max(math.cos(lr[2]), 0) ** s.beta
    assert w == pytest.approx(ref_w, rel=1e-14)


def test_saft_weights_are_the_transmission_alone():
    """SAFT (delay-and-sum, Section 1) is A^T with the beam profile phi = 1:
    with beta = 0 every pair inside the 90-degree limit weighs the
    interface transmission only, wherever the pixel lies."""
    s = _tiny(layers=2)
    s.beta = 0.0
    p = O.Plan(s, nthreads=1)
    g = O.Geometry(s)
    for v in (3, 7 * s.img_w + 3, s.N - 1):
        zr = (v // s.img_w + 0.5) * s.pitch
        for k in range(s.K):
            assert p.pair(v, k)[2] == g.transmission(zr)


def test_saft_image_of_a_point_reflector_peaks_at_the_reflector():
    """Delay-and-sum focuses: the SAFT image (A^T y, beta = 0) of the data of
    one point reflector (y = A e_v with the beam model) is largest at v among
    the pixels of v's layer (the transmission factor differs between layers:
    about 0.12 from water into steel, so water pixels are not comparable)."""
    for n_layers, pixels in ((1, (9 * 24 + 11, 15 * 24 + 6)), (2, (9 * 24 + 11, 15 * 24 + 6))):
        s = S.small_scene(n_layers=n_layers, w=24, h=20, n_tx=6, n_rx=4, M=400, atten=False)
        p = O.Plan(s, nthreads=2)
        p0 = O.Plan(s.copy(beta=0.0), nthreads=2)
        top = s.layers[0].thickness if n_layers == 2 else 0.0
        z = (np.arange(s.img_h) + 0.5) * s.pitch
        same_layer = np.repeat(z >= top, s.img_w)
        for v in pixels:
            x = np.zeros(s.N)
            x[v] = 1.0
            img = p0.backproject(p.forward(x).reshape(-1))
            assert same_layer[v]
            assert int(np.argmax(np.where(same_layer, img, -np.inf))) == v


def _pair_factors(s, v, k):
    p = O.Plan(s, nthreads=1)
    g = O.Geometry(s)
    r, c = divmod(v, s.img_w)
    xc, zr = (c + 0.5) * s.pitch, (r + 0.5) * s.pitch
    i, j = divmod(k, s.n_rx)
    return p.pair(v, k)[2], g, xc, zr, s.tx_x[i], s.tx_x[i] + s.rx_offset[j]


def test_first_angle_apodization():
    """Beam-profile variant (eq. 12 with theta_1 instead of the angle sum):
    identical to eq. 12 in one layer, and cos^beta(theta_1) of each leg with
    the transmission in two layers."""
    s1 = _tiny(layers=1)
    for v, k in ((7 * s1.img_w + 3, 3), (2, 0)):
        assert _pair_factors(s1.copy(apod_first_angle=True), v, k)[0] == pytest.approx(
            _pair_factors(s1, v, k)[0], rel=1e-14)
    s2 = _tiny(layers=2).copy(apod_first_angle=True)
    v, k = 7 * s2.img_w + 3, 3
    w, g, xc, zr, ut, ur = _pair_factors(s2, v, k)
    a_t, a_r = g.leg(xc - ut, zr)[3], g.leg(xc - ur, zr)[3]
    assert g.leg(xc - ut, zr)[2] > a_t                       # the sum differs from theta_1 here
    ref = g.transmission(zr) * math.cos(a_t) ** s2.beta * math.cos(a_r) ** s2.beta
    assert w == pytest.approx(ref, rel=1e-14)


def test_firing_angle_closed_form_in_one_layer():
    """A transmitter tilted by psi toward +x (Section 3's 5-degree firing
    angle): in one layer its factor is max(cos(atan((x - u)/z) - psi), 0)^beta,
    larger on the +x side than at the mirrored pixel; receivers are unchanged."""
    psi = math.radians(5.0)
    s = _tiny(layers=1).copy(firing_angle=psi)
    for v, k in ((7 * s.img_w + 6, 2), (7 * s.img_w + 1, 2), (3, 0), (9 * s.img_w + 7, 1)):
        w, g, xc, zr, ut, ur = _pair_factors(s, v, k)
        phi_t = max(math.cos(math.atan((xc - ut) / zr) - psi), 0.0) ** s.beta
        phi_r = max(math.cos(math.atan(abs(xc - ur) / zr)), 0.0) ** s.beta
        assert w == pytest.approx(phi_t * phi_r, rel=1e-12)
    # mirror: tilt -psi on the mirrored scan gives the same weight
    sm = s.copy(firing_angle=-psi, tx_x=s.img_w * s.pitch - np.asarray(s.tx_x),
                rx_offset=-np.asarray(s.rx_offset))
    for v, k in ((7 * s.img_w + 6, 2), (4 * s.img_w + 1, 3)):
        r, c = divmod(v, s.img_w)
        vm = r * s.img_w + (s.img_w - 1 - c)
        assert _pair_factors(sm, vm, k)[0] == pytest.approx(_pair_factors(s, v, k)[0], rel=1e-12)


def test_direct_columns_are_the_pulse_delayed_along_the_array():
    """Eq. 1's direct-arrival basis (reading: one column per receiver, the
    unattenuated pulse after the path |o_j| / c_1 through the first layer):
    with offsets whose delays fall on whole samples the columns equal
    s(n dt - |o_j| / c_1) inside the open window and 0 outside; an offset that
    falls between table nodes agrees within the bilinear bound."""
    fs, c1 = 10e6, 1500.0
    offs = np.array([-1.5e-3, 0.75e-3, 3e-3, 1.0e-3])       # 10, 5, 20 and 6.67 samples
    for atten in (False, True):
        s = S.small_scene(n_layers=2, w=4, h=4, n_tx=1, n_rx=1, M=140, direct=True, atten=atten)
        s.layers[0].speed = c1                        # the second layer (steel) is much faster
        s.rx_offset = offs
        p = O.Plan(s, pix=np.array([0]), nthreads=1)
        g = O.Geometry(s)
        Tw = g.pulse_support()
        d = p.direct_columns()
        assert d.shape == (len(offs), s.M)
        n = np.arange(s.M)
        for j, o in enumerate(offs[:3]):
            D = round(abs(o) / c1 * fs)
            ref = np.array([g.pulse((m - D) / fs) if 0 < m - D < Tw else 0.0 for m in n])
            assert np.max(np.abs(d[j] - ref)) < (1e-12 if not atten else 5e-11), (atten, j)
        Dt = abs(offs[3]) / c1
        dtau = 1.0 / (fs * s.Q)
        ts = np.linspace(0.0, Tw / fs, 4001)
        s2 = np.array([g.pulse(t) for t in ts])
        curv = np.max(np.abs(np.diff(s2, 2))) / (ts[1] - ts[0]) ** 2
        ref = np.array([g.pulse(m / fs - Dt) if 0 < m / fs - Dt < Tw / fs else 0.0 for m in n])
        assert np.max(np.abs(d[3] - ref)) <= 1.05 * dtau ** 2 / 8 * curv + 5e-11


def test_projection_removes_direct_arrivals():
    s = _tiny(direct=True)
    p = O.Plan(s, nthreads=1)
    d = p.direct_columns()
    r = S.random_vector(s.K * s.M, 5).reshape(s.K, s.M)
    e, gk = p.project(r)
    for k in range(s.K):
        dj = d[k % s.n_rx]
        assert abs(dj @ e[k]) < 1e-12 * np.linalg.norm(dj) * np.linalg.norm(r[k])
        assert np.allclose(r[k] - gk[k] * dj, e[k], atol=1e-15)


def test_direct_only_data_reconstructs_zero_image_and_gains():
    s = _tiny(direct=True)
    p = O.Plan(s, nthreads=1)
    d = p.direct_columns()
    g_true = S.direct_gains(s, 3)
    y = np.stack([g_true[k] * d[k % s.n_rx] for k in range(s.K)])
    x, gk, cost, gn = p.reconstruct(y, sigma_noise=0.05, n_iter=5)
    assert np.max(np.abs(x)) < 1e-12
    assert np.allclose(gk, g_true, rtol=1e-12, atol=0)


# --------------------------------------------------------------------------
# prior (eq. 14-17)
# --------------------------------------------------------------------------
def test_potential_derivative_and_curvature():
    s = S.cfg1()
    for sigma in (0.3, 0.05):
        for delta in (-0.7, -1e-3, 2e-4, 0.05, 1.3):
            h = 1e-7 * max(abs(delta), 1e-3)
            fd = (O.rho(s, delta + h, sigma) - O.rho(s, delta - h, sigma)) / (2 * h)
            assert O.drho(s, delta, sigma) == pytest.approx(fd, rel=1e-6)
            assert O.kappa(s, delta, sigma) == pytest.approx(O.drho(s, delta, sigma) / delta, rel=1e-14)
        # the curvature is continuous at 0 and non-increasing in |delta|
        k0 = O.kappa(s, 0.0, sigma)
        assert O.kappa(s, 1e-14, sigma) == pytest.approx(k0, rel=1e-9)
        ks = [O.kappa(s, d, sigma) for d in np.linspace(1e-6, 2.0, 50)]
        assert np.all(np.diff(ks) <= 0)


def test_prior_gradient_matches_finite_differences():
    s = S.small_scene(w=6, h=5).copy(prior=S.Prior(m=0.2, a=1.5))
    x = S.random_vector(s.N, 9, -0.5, 0.5)
    gr = O.prior_grad(s, x)
    h = 1e-6
    for v in range(s.N):
        xp, xm = x.copy(), x.copy()
        xp[v] += h
        xm[v] -= h
        fd = (O.prior_cost(s, xp) - O.prior_cost(s, xm)) / (2 * h)
        assert gr[v] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_prior_weights_follow_depth_rule():
    # with p = q = 2 the potential is delta^2 / (4 sigma^2): a two-pixel image
    # isolates sigma_g = sigma0 sqrt(m_s m_r) with m_s = 1 + (m-1)(z/zmax)^a
    s = S.small_scene(w=1, h=2).copy(prior=S.Prior(p=2.0, q=2.0, sigma0=0.4, m=0.25, a=2.0))
    x = np.array([0.3, -0.1])
    z = (np.arange(2) + 0.5) * s.pitch
    m = 1 + (0.25 - 1) * (z / z[-1]) ** 2.0
    sg = 0.4 * math.sqrt(m[0] * m[1])
    b_edge = 1.0 / (4 + 4 / math.sqrt(2))
    assert O.prior_cost(s, x) == pytest.approx(b_edge * 0.4 ** 2 / (4 * sg * sg), rel=1e-14)


def test_symmetric_bound_majorizes_prior():
    s = S.small_scene(w=7, h=6).copy(prior=S.Prior(m=0.3))
    x = S.random_vector(s.N, 11, -0.3, 0.3)
    d = S.random_vector(s.N, 12, -0.2, 0.2)
    r0 = O.prior_cost(s, x)
    g = O.prior_grad(s, x)
    cv = O.prior_curv(s, x, d)
    for t in (-3.0, -0.5, 0.01, 0.3, 1.0, 4.0):
        bound = r0 + t * float(g @ d) + 0.5 * t * t * cv
        assert O.prior_cost(s, x + t * d) <= bound + 1e-12


# --------------------------------------------------------------------------
# MAP iteration (eq. 18)
# --------------------------------------------------------------------------
def _noisy_data(s, seed=0, snr_db=20.0):
    p = O.Plan(s, nthreads=2)
    x_true = S.phantom(s, seed)
    y0 = p.forward(x_true)
    if s.direct_arrival:
        d = p.direct_columns()
        g = S.direct_gains(s, seed) * np.max(np.abs(y0))
        y0 = y0 + np.stack([g[k] * d[k % s.n_rx] for k in range(s.K)])
    sig = math.sqrt(np.sum(y0 ** 2) / (10 ** (snr_db / 10) * s.K * s.M))
    return p, x_true, y0 + sig * S.unit_noise(s, seed), sig


def test_map_cost_is_non_increasing():
    s = _tiny(direct=True, layers=3).copy(prior=S.Prior(m=0.2))
    p, _, y, sig = _noisy_data(s)
    x, gk, cost, gn = p.reconstruct(y, sig, 30)
    assert np.all(np.diff(cost) <= 1e-12 * abs(cost[0]))
    assert cost[-1] < cost[0]


def test_quadratic_prior_map_matches_dense_solve():
    s = S.small_scene(n_layers=2, w=6, h=6, n_tx=2, n_rx=2, M=96, direct=True)
    s = s.copy(prior=S.Prior(p=2.0, q=2.0, sigma0=0.5, m=0.5))
    p, _, y, sig = _noisy_data(s, seed=4)
    A = p.dense_A()
    d = p.direct_columns()
    K, M, N = s.K, s.M, s.N
    P = np.eye(K * M)
    for k in range(K):
        dj = d[k % s.n_rx]
        sl = slice(k * M, (k + 1) * M)
        P[sl, sl] -= np.outer(dj, dj) / (dj @ dj)
    # Hessian of sum b (x_s - x_r)^2 / (4 sigma_sr^2) assembled by brute force
    Hr = np.zeros((N, N))
    for v in range(N):
        e = np.zeros(N)
        e[v] = 1.0
        Hr[:, v] = O.prior_grad(s, e)
    lhs = A.T @ P @ A / sig ** 2 + Hr
    rhs = A.T @ P @ y.reshape(-1) / sig ** 2
    x_ref = np.linalg.solve(lhs, rhs)
    x, gk, cost, gn = p.reconstruct(y, sig, 3000)
    assert np.linalg.norm(x.reshape(-1) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_gradient_vanishes_at_convergence():
    s = S.small_scene(n_layers=2, w=6, h=6, n_tx=2, n_rx=2, M=96, direct=False)
    s = s.copy(prior=S.Prior(sigma0=0.5, m=0.5, T=0.5))
    p, _, y, sig = _noisy_data(s, seed=2)
    x, gk, cost, gn = p.reconstruct(y, sig, 4000)
    assert gn[-1] / gn[0] < 1e-9


# --------------------------------------------------------------------------
# iterative coordinate descent (Section 2 "Optimization": the paper's ICD)
# --------------------------------------------------------------------------
def test_icd_column_norms_match_dense_columns():
    s = S.small_scene(n_layers=2, w=5, h=4, n_tx=3, n_rx=2, M=128, direct=False)
    p = O.Plan(s, nthreads=2)
    A = p.dense_A()                     # every sample of every column, no tap window
    np.testing.assert_allclose(p.column_norms(), (A ** 2).sum(axis=0), rtol=1e-12, atol=0)


def test_icd_single_pixel_lands_on_the_least_squares_gain():
    # one pixel, no clique: one ICD update (with its step along the update) is the least-squares
    # fit of the projected column to the projected data, whatever curvature scaled the update
    s = S.small_scene(n_layers=2, w=1, h=1, n_tx=3, n_rx=2, M=128, direct=True).copy(z0=1.5e-3)
    p = O.Plan(s, nthreads=2)
    a = p.dense_A()[:, 0]
    y = 0.7 * a + 0.05 * np.max(np.abs(a)) * S.unit_noise(s, 3).reshape(-1)
    Pa = p.project(a)[0].reshape(-1)
    Py = p.project(y)[0].reshape(-1)
    x_ls = (Pa @ Py) / (Pa @ Pa)
    x, _, cost = p.icd(y, 0.1, 1, 2)
    assert x[0, 0] == pytest.approx(x_ls, rel=1e-12)
    assert cost[0] == pytest.approx(np.sum((Py - x_ls * Pa) ** 2) / (2 * 0.01), rel=1e-12)


def test_icd_update_minimises_the_surrogate_by_brute_force():
    # sequential ICD (one pixel per colour) from a non-flat start: each update is the minimiser of
    # the exact data term along that pixel plus, for every clique, the symmetric quadratic bound
    # of the potential taken at the start of the update; found here by a bounded 1-D search
    from scipy.optimize import minimize_scalar
    s = S.small_scene(n_layers=2, w=2, h=1, n_tx=3, n_rx=2, M=128, direct=True).copy(
        z0=1.5e-3, prior=S.Prior(m=0.5))
    p, _, y, sig = _noisy_data(s, seed=5)
    x0 = np.array([0.3, -0.2])
    be = 1.0 / (4.0 + 4.0 / math.sqrt(2.0))           # edge clique weight (8-neighbourhood, sum 1)
    zc = s.z0 + 0.5 * s.pitch
    sg = s.prior.sigma0 * (1.0 + (s.prior.m - 1.0) * (zc / zc) ** s.prior.a)   # sigma0 sqrt(m_s m_r), one row
    x = x0.copy()
    for v in (0, 1):
        r = 1 - v
        d0 = x[v] - x[r]
        kap = O.kappa(s, d0, sg)

        def f(u):
            xv = x.copy()
            xv[v] += u
            e, _ = p.project(y - p.forward(xv))
            return np.sum(e ** 2) / (2 * sig ** 2) + be * kap / 2 * (d0 + u) ** 2

        res = minimize_scalar(f, bounds=(-5.0, 5.0), method="bounded", options={"xatol": 1e-12})
        x[v] += res.x
    xi, _, _ = p.icd(y, sig, 1, 2, x0=x0)
    np.testing.assert_allclose(xi.reshape(-1), x, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("spacing", [2, 3])
def test_icd_reaches_the_map_minimiser(spacing):
    # pixels 3 mm apart (longer than the pulse) have nearly orthogonal columns: ICD converges in a
    # few dozen sweeps to the unique minimiser of eq. 18 that the conjugate-gradient iteration finds
    s = S.small_scene(n_layers=2, w=3, h=3, n_tx=4, n_rx=3, M=256, direct=True)
    s = s.copy(pitch=3e-3, tx_x=S.centred_positions(4, 2e-3, 4.5e-3))
    p, _, y, sig = _noisy_data(s, seed=1)
    xc, _, cc, gn = p.reconstruct(y, sig, 400)
    assert gn[-1] < 1e-10 * gn[0]
    xi, _, ci = p.icd(y, sig, 200, spacing)
    assert np.linalg.norm(xi - xc) <= 1e-9 * np.linalg.norm(xc)
    assert ci[-1] == pytest.approx(cc[-1], rel=1e-12)


@pytest.mark.parametrize("spacing", [2, 4, 16])
def test_icd_cost_is_non_increasing(spacing):
    s = _tiny(direct=True, layers=3).copy(prior=S.Prior(m=0.2))
    p, _, y, sig = _noisy_data(s)
    x, gk, cost = p.icd(y, sig, 8, spacing)
    assert np.all(np.diff(cost) <= 1e-12 * abs(cost[0]))
    assert cost[-1] < cost[0]
