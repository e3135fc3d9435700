"""Shared test helpers: seeded data through the oracle, error metrics."""
import math

import numpy as np

from oracle import oracle as O
from paper_2202_09703_gb300 import synth as S


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_data(scene, seed: int = 0, snr_db: float = 20.0, plan=None):
    """y = A x_true + D g_true + w with the oracle's operator (SNR in dB)."""
    p = plan or O.Plan(scene)
    x_true = S.phantom(scene, seed)
    y0 = p.forward(x_true)
    g_true = np.zeros(scene.K)
    if scene.direct_arrival:
        d = p.direct_columns()
        g_true = S.direct_gains(scene, seed) * np.max(np.abs(y0))
        y0 = y0 + np.stack([g_true[k] * d[k % scene.n_rx] for k in range(scene.K)])
    sig = math.sqrt(np.sum(y0 ** 2) / (10 ** (snr_db / 10) * scene.K * scene.M))
    y = y0 + sig * S.unit_noise(scene, seed)
    return p, x_true, g_true, y, sig


def ragged_scene():
    s = S.small_scene(n_layers=3, w=40, h=23, n_tx=3, n_rx=5, M=300, direct=True, name="tiny_ragged")
    s.layers[2].thickness = 50e-3
    return s


def many_layer_scene(n_layers: int):
    """A 5-8 layer medium (the kernels' 8-layer instantiation serves any scene
    with more than 4 layers): 2 mm layers of alternating slow and fast
    materials under a semi-infinite last layer, every layer holding pixels."""
    assert 5 <= n_layers <= 8
    s = S.small_scene(n_layers=1, w=36, h=30, n_tx=3, n_rx=4, M=420, direct=True,
                      name=f"tiny_layers{n_layers}")
    speeds = [1480.0, 5900.0, 3000.0, 4500.0, 2200.0, 3800.0, 2600.0, 5200.0]
    atten = [2.0, 5.0, 30.0, 20.0, 12.0, 8.0, 15.0, 4.0]
    dens = [1000.0, 7850.0, 1900.0, 2650.0, 1500.0, 2400.0, 1800.0, 7000.0]
    s.layers = [S.Layer(1.5e-3 if i < n_layers - 1 else 20e-3, speeds[i],
                        atten[i] * 0.058, dens[i]) for i in range(n_layers)]
    return s
