"""Seeded synthetic inputs: scene descriptions, phantoms and random draws.

This module holds the workloads' shapes and the random numbers that feed both
the CUDA path and the FP64 oracle.  It contains none of the reconstruction
method's arithmetic (no travel times, pulses, operators or priors): a scene is
a plain description of the layered medium and the acquisition of Section 2 of
the paper, and the draws are SplitMix64 + Box-Muller numbers.

Scenes (sizes follow the paper's layered, collimated-beam acquisitions; the
paper's own concrete-cylinder and K-Wave data are not available, these stand
in for them):

* ``cfg0``: 2 layers (water 10 mm at 1480 m/s over steel at 5900 m/s), 64x64
  image at 0.5 mm, 16 Tx positions at 2 mm, 8 receivers at 5 mm, 1 MHz
  2-cycle pulse sampled at 10 MHz, 512 samples, 3 rectangular reflectors.
* ``cfg1``: 4 layers (water 20 mm/1480, steel 12 mm/5900, cement 40 mm/3000,
  rock 100 mm/4500), 256x512 image at 0.5 mm, 64 Tx x 16 Rx, 2 MHz pulse at
  20 MHz, 2048 samples, interfaces plus 10-40 disc voids, direct arrivals on.
* ``cfg2``: cfg1's layers, 512x1024 image at 0.25 mm, 128 Tx x 32 Rx,
  4096 samples, BF16 storage.
* ``cfg3_scenes``: uneven random scenes for the batched form.
"""
from __future__ import annotations

import copy
import math
from dataclasses import dataclass, field, asdict

import numpy as np

_MASK = (1 << 64) - 1


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014) and Box-Muller normals
# --------------------------------------------------------------------------
class SplitMix64:
    """Counter-based SplitMix64 stream; ``uniform`` gives doubles in [0, 1)."""

    GOLDEN = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(self.GOLDEN)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * self.GOLDEN) & _MASK
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float, n: int) -> np.ndarray:
        return lo + (hi - lo) * self.uniform(n)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers in [lo, hi] inclusive."""
        return lo + np.minimum((self.uniform(n) * (hi - lo + 1)).astype(np.int64), hi - lo)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


# --------------------------------------------------------------------------
# Scene description
# --------------------------------------------------------------------------
@dataclass
class Layer:
    thickness: float          # m (the last layer extends below its thickness)
    speed: float              # m/s
    atten: float              # Np / (MHz m)
    density: float            # kg / m^3


@dataclass
class Prior:
    p: float = 1.1
    q: float = 2.0
    T: float = 0.01
    sigma0: float = 0.3
    m: float = 1.0
    a: float = 1.0


@dataclass
class Scene:
    name: str
    layers: list
    img_w: int
    img_h: int
    pitch: float
    x0: float
    z0: float
    tx_x: np.ndarray
    rx_offset: np.ndarray
    fs: float
    n_samples: int
    fc: float
    n_cycles: float = 2.0
    beta: float = 8.0
    direct_arrival: bool = False
    gamma_max: float = 0.0    # s; 0 selects the default rule
    G: int = 16
    Q: int = 16
    prior: Prior = field(default_factory=Prior)
    n_iter: int = 20
    precision: str = "fp32"
    firing_angle: float = 0.0       # rad: transmitter beam axis turned toward +x (Section 3 uses 5 degrees)
    apod_first_angle: bool = False  # eq. 12 with the first-layer angle instead of the sum of the angles

    @property
    def n_tx(self) -> int:
        return len(self.tx_x)

    @property
    def n_rx(self) -> int:
        return len(self.rx_offset)

    @property
    def K(self) -> int:
        return self.n_tx * self.n_rx

    @property
    def N(self) -> int:
        return self.img_w * self.img_h

    @property
    def M(self) -> int:
        return self.n_samples

    def copy(self, **kw) -> "Scene":
        s = copy.deepcopy(self)
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def describe(self) -> dict:
        d = asdict(self)
        d["tx_x"] = list(map(float, self.tx_x))
        d["rx_offset"] = list(map(float, self.rx_offset))
        return d


# Paper-equivalent attenuation (Np / (MHz m)) quoted for a 58 kHz pulse; the
# scenes scale it by 0.058 MHz / f_c so the loss per period matches the
# paper's experiment at the scene's own centre frequency.
_PAPER_FC_MHZ = 0.058
MATERIALS = {
    #          speed   alpha@58kHz  density
    "water":  (1480.0, 2.0, 1000.0),
    "steel":  (5900.0, 5.0, 7850.0),
    "cement": (3000.0, 30.0, 1900.0),
    "rock":   (4500.0, 20.0, 2650.0),
}


def material_layer(name: str, thickness: float, fc: float) -> Layer:
    c, a58, rho = MATERIALS[name]
    return Layer(thickness, c, a58 * _PAPER_FC_MHZ / (fc * 1e-6), rho)


def centred_positions(n: int, step: float, centre: float = 0.0) -> np.ndarray:
    return centre + (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * step


def cfg0() -> Scene:
    fc = 1e6
    w = h = 64
    pitch = 0.5e-3
    centre = w * pitch / 2
    return Scene(
        name="cfg0",
        layers=[material_layer("water", 10e-3, fc), material_layer("steel", 10e-3, fc)],
        img_w=w, img_h=h, pitch=pitch, x0=0.0, z0=0.0,
        tx_x=centred_positions(16, 2e-3, centre),
        rx_offset=centred_positions(8, 5e-3),
        fs=10e6, n_samples=512, fc=fc,
        direct_arrival=False,
        prior=Prior(m=1.0),
        n_iter=20,
    )


def cfg1() -> Scene:
    fc = 2e6
    w, h = 256, 512
    pitch = 0.5e-3
    centre = w * pitch / 2
    return Scene(
        name="cfg1",
        layers=[material_layer("water", 20e-3, fc), material_layer("steel", 12e-3, fc),
                material_layer("cement", 40e-3, fc), material_layer("rock", 100e-3, fc)],
        img_w=w, img_h=h, pitch=pitch, x0=0.0, z0=0.0,
        tx_x=centred_positions(64, 2e-3, centre),
        rx_offset=centred_positions(16, 5e-3),
        fs=20e6, n_samples=2048, fc=fc,
        direct_arrival=True,
        prior=Prior(m=0.1, a=1.0),
        n_iter=50,
    )


def cfg2() -> Scene:
    s = cfg1()
    w, h = 512, 1024
    pitch = 0.25e-3
    centre = w * pitch / 2
    return s.copy(name="cfg2", img_w=w, img_h=h, pitch=pitch,
                  tx_x=centred_positions(128, 1e-3, centre),
                  rx_offset=centred_positions(32, 5e-3),
                  n_samples=4096, precision="bf16")


def small_scene(n_layers: int = 2, w: int = 16, h: int = 16, n_tx: int = 2, n_rx: int = 2,
                M: int = 128, direct: bool = False, atten: bool = True, name: str = "tiny") -> Scene:
    """Tiny grids for brute-force and dense-matrix checks (1-3 layers)."""
    fc, fs = 1e6, 10e6
    names = ["water", "steel", "cement", "rock"]
    th = [3e-3, 2e-3, 2e-3, 2e-3]
    layers = [material_layer(names[i], th[i], fc) for i in range(n_layers)]
    if not atten:
        for L in layers:
            L.atten = 0.0
    pitch = 0.5e-3
    return Scene(
        name=name, layers=layers, img_w=w, img_h=h, pitch=pitch, x0=0.0, z0=0.0,
        tx_x=centred_positions(n_tx, 2e-3, w * pitch / 2),
        rx_offset=centred_positions(n_rx, 2.5e-3),
        fs=fs, n_samples=M, fc=fc, direct_arrival=direct, n_iter=10,
    )


def random_scene(rng: SplitMix64, idx: int) -> Scene:
    """One uneven scene of the batched workload (image sides from {64..512})."""
    sides = np.array([64, 128, 256, 512])
    w = int(sides[rng.integers(0, 3, 1)[0]])
    h = int(sides[rng.integers(0, 3, 1)[0]])
    L = int(rng.integers(2, 5, 1)[0])
    fc, fs = 2e6, 20e6
    layers = []
    for li in range(L):
        layers.append(Layer(float(rng.uniform_range(5e-3, 100e-3, 1)[0]),
                            float(rng.uniform_range(1400.0, 6000.0, 1)[0]),
                            float(rng.uniform_range(0.05, 1.0, 1)[0]),
                            float(rng.uniform_range(1000.0, 8000.0, 1)[0])))
    pitch = 0.5e-3
    n_tx = max(w // 4, 1)
    n_rx = int(rng.integers(8, 32, 1)[0])
    M = int(np.array([512, 1024, 2048, 4096])[rng.integers(0, 3, 1)[0]])
    return Scene(
        name=f"cfg3_{idx}", layers=layers, img_w=w, img_h=h, pitch=pitch, x0=0.0, z0=0.0,
        tx_x=centred_positions(n_tx, 2e-3, w * pitch / 2),
        rx_offset=centred_positions(n_rx, 5e-3),
        fs=fs, n_samples=M, fc=fc, direct_arrival=True,
        prior=Prior(m=0.1), n_iter=50,
    )


def cfg3_scenes(n: int = 96, seed: int = 0) -> list:
    rng = SplitMix64(seed * 7919 + 3)
    return [random_scene(rng, i) for i in range(n)]


CONFIGS = {"cfg0": cfg0, "cfg1": cfg1, "cfg2": cfg2}


# --------------------------------------------------------------------------
# Phantoms and draws
# --------------------------------------------------------------------------
def phantom_rects(scene: Scene, seed: int, n_rect: int = 3) -> np.ndarray:
    """Axis-aligned rectangles, 4-12 px per side, values U[0.2, 1]."""
    rng = SplitMix64(seed * 1000003 + 11)
    x = np.zeros((scene.img_h, scene.img_w))
    for _ in range(n_rect):
        hh = int(rng.integers(4, min(12, scene.img_h), 1)[0])
        ww = int(rng.integers(4, min(12, scene.img_w), 1)[0])
        r0 = int(rng.integers(0, scene.img_h - hh, 1)[0])
        c0 = int(rng.integers(0, scene.img_w - ww, 1)[0])
        x[r0:r0 + hh, c0:c0 + ww] = rng.uniform_range(0.2, 1.0, 1)[0]
    return x


def phantom_layered(scene: Scene, seed: int) -> np.ndarray:
    """Interface rows (impedance contrast at each layer top) plus 10-40 disc voids."""
    rng = SplitMix64(seed * 1000003 + 17)
    H, W = scene.img_h, scene.img_w
    x = np.zeros((H, W))
    top = 0.0
    for li in range(1, len(scene.layers)):
        top += scene.layers[li - 1].thickness
        r = int(math.floor((top - scene.z0) / scene.pitch))
        if 0 <= r < H:
            z1 = scene.layers[li - 1].density * scene.layers[li - 1].speed
            z2 = scene.layers[li].density * scene.layers[li].speed
            x[r, :] = (z2 - z1) / (z2 + z1)
    nv = int(rng.integers(10, 40, 1)[0])
    zz = scene.z0 + (np.arange(H) + 0.5) * scene.pitch
    xx = scene.x0 + (np.arange(W) + 0.5) * scene.pitch
    for _ in range(nv):
        rad = rng.uniform_range(1e-3, 4e-3, 1)[0]
        cx = rng.uniform_range(xx[0], xx[-1], 1)[0]
        cz = rng.uniform_range(zz[0], zz[-1], 1)[0]
        val = rng.uniform_range(-1.0, 1.0, 1)[0]
        mask = (xx[None, :] - cx) ** 2 + (zz[:, None] - cz) ** 2 <= rad * rad
        x[mask] = val
    return x


def phantom(scene: Scene, seed: int) -> np.ndarray:
    if scene.name == "cfg0" or scene.name.startswith("tiny"):
        return phantom_rects(scene, seed)
    return phantom_layered(scene, seed)


def direct_gains(scene: Scene, seed: int) -> np.ndarray:
    """Unscaled direct-arrival gains U[0.5, 1] per A-scan (the user scales them)."""
    return SplitMix64(seed * 1000003 + 23).uniform_range(0.5, 1.0, scene.K)


def unit_noise(scene: Scene, seed: int) -> np.ndarray:
    """Standard-normal noise of shape (K, M)."""
    return SplitMix64(seed * 1000003 + 29).normal(scene.K * scene.M).reshape(scene.K, scene.M)


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return SplitMix64(seed * 1000003 + 31).uniform_range(lo, hi, n)
