"""Seeded velocity models and acquisition geometry for the 2D Helmholtz workloads.

The paper's own models (its 1D well model and 2D surface model) exist only as
figures, so every workload here is synthetic and seeded. The shapes follow the
paper's examples: surface sources and receivers, a few low frequencies, layered
media with a smooth starting model (Section "Examples").

Conventions
-----------
* Arrays are row-major ``[z][x]`` (x fastest); ``c[iz, ix]`` is the velocity in
  m/s at physical node ``(x = ix*h, z = iz*h)`` measured from the top-left node.
* Source and receiver positions are physical node indices ``(ix, iz)``.
* Frequencies are in Hz; angular frequency is ``2*pi*f``.
* Slowness is ``m = 1/c`` (the paper's model parameter, Eq. 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Model:
    name: str
    velocity: np.ndarray            # [Pz][Px] float64, m/s
    h: float                        # grid spacing, m
    sources: np.ndarray             # [ns, 2] int (ix, iz), physical node indices
    freqs: np.ndarray               # [nf] Hz
    receivers: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int64))
    npml: int = 20                  # damping-layer width in nodes on each side
    alpha_max: float = 0.5          # damping at the outermost layer node
    seed: int | None = None

    @property
    def Px(self) -> int:
        return int(self.velocity.shape[1])

    @property
    def Pz(self) -> int:
        return int(self.velocity.shape[0])

    @property
    def slowness(self) -> np.ndarray:
        return 1.0 / self.velocity

    @property
    def omegas(self) -> np.ndarray:
        return 2.0 * np.pi * np.asarray(self.freqs, dtype=np.float64)


def _node(x_m: float, h: float) -> int:
    """Nearest node index to a coordinate in metres."""
    return int(np.rint(x_m / h))


def _grid(Px: int, Pz: int, h: float):
    x = np.arange(Px) * h
    z = np.arange(Pz) * h
    return np.meshgrid(x, z)  # X, Z each [Pz][Px]


def homogeneous_model(Px: int, Pz: int, h: float, c: float, freqs=(5.0,),
                      sources=None, npml: int = 20, alpha_max: float = 0.5) -> Model:
    if sources is None:
        sources = [(Px // 2, Pz // 2)]
    return Model("homogeneous", np.full((Pz, Px), float(c)), float(h),
                 np.asarray(sources, np.int64).reshape(-1, 2), np.asarray(freqs, float),
                 npml=npml, alpha_max=alpha_max)


def c1_model() -> Model:
    """Small plain case: 101 x 101 physical nodes, h = 10 m, 5 Hz, one surface source.

    Velocity rises linearly from 1500 m/s at the top to 3000 m/s at the bottom,
    plus a +300 m/s Gaussian anomaly (sigma 100 m) centred at (500 m, 500 m).
    """
    Px = Pz = 101
    h = 10.0
    X, Z = _grid(Px, Pz, h)
    c = 1500.0 + 1500.0 * Z / 1000.0
    c += 300.0 * np.exp(-((X - 500.0) ** 2 + (Z - 500.0) ** 2) / (2.0 * 100.0 ** 2))
    src = np.array([[_node(500.0, h), _node(20.0, h)]], np.int64)
    return Model("c1_101x101_5Hz", c, h, src, np.array([5.0]))


def c2_model(seed: int = 2) -> Model:
    """Single large solve: 1001 x 1001 physical nodes, h = 5 m, 15 Hz.

    12 random horizontal layers (velocities uniform in [1500, 4500] m/s) plus three
    Gaussian anomalies (amplitude in [-300, 300] m/s, sigma in [50, 200] m), clipped
    to [1500, 4500] m/s. One source at the surface centre (2500 m, 20 m).
    """
    rng = np.random.default_rng(seed)
    Px = Pz = 1001
    h = 5.0
    L = (Px - 1) * h
    X, Z = _grid(Px, Pz, h)
    depths = np.sort(rng.uniform(0.0, L, 11))
    vel = rng.uniform(1500.0, 4500.0, 12)
    c = vel[np.searchsorted(depths, Z)]
    for _ in range(3):
        amp = rng.uniform(-300.0, 300.0)
        sig = rng.uniform(50.0, 200.0)
        cx, cz = rng.uniform(0.1 * L, 0.9 * L, 2)
        c = c + amp * np.exp(-((X - cx) ** 2 + (Z - cz) ** 2) / (2.0 * sig ** 2))
    c = np.clip(c, 1500.0, 4500.0)
    src = np.array([[_node(2500.0, h), _node(20.0, h)]], np.int64)
    return Model("c2_1001x1001_15Hz", c, h, src, np.array([15.0]), seed=seed)


def _c3_velocity(rng, Px: int, Pz: int, h: float) -> np.ndarray:
    X, Z = _grid(Px, Pz, h)
    depth_max = (Pz - 1) * h
    depths = np.sort(rng.uniform(0.0, depth_max, 7))
    vel = np.sort(rng.uniform(1500.0, 4000.0, 8))
    c = vel[np.searchsorted(depths, Z)]
    z0 = rng.uniform(600.0, 1200.0)
    theta = np.deg2rad(rng.uniform(5.0, 20.0))
    below = Z > z0 + X * np.tan(theta)
    c = np.where(below, np.maximum(c, 3500.0), c)
    return c


def c3_model(seed: int = 3) -> Model:
    """Batched multi-RHS case: 401 x 201 physical nodes, h = 10 m.

    8 flat layers with increasing velocity in [1500, 4000] m/s and a dipping
    interface below which c >= 3500 m/s. 64 surface sources (x = 110 + 60 s m,
    z = 20 m) times 5 frequencies (3..7 Hz) = 320 right-hand sides.
    """
    rng = np.random.default_rng(seed)
    Px, Pz, h = 401, 201, 10.0
    c = _c3_velocity(rng, Px, Pz, h)
    src = np.array([[_node(110.0 + 60.0 * s, h), _node(20.0, h)] for s in range(64)], np.int64)
    return Model("c3_401x201_64src_5f", c, h, src, np.array([3.0, 4.0, 5.0, 6.0, 7.0]), seed=seed)


def c4_models(seed: int = 4):
    """FWI gradient case: true model and a smoothed starting model, 401 x 201, h = 10 m.

    The true velocity is drawn like the batched case; the starting model is its
    Gaussian-smoothed velocity (sigma = 200 m, 'nearest' edges). 32 surface sources
    (x = 110 + 120 s m), 201 surface receivers (x = 20 r m), 3..6 Hz.
    Returns ``(true_model, start_model)`` sharing geometry.
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    Px, Pz, h = 401, 201, 10.0
    c_true = _c3_velocity(rng, Px, Pz, h)
    c0 = gaussian_filter(c_true, sigma=200.0 / h, mode="nearest")
    src = np.array([[_node(110.0 + 120.0 * s, h), _node(20.0, h)] for s in range(32)], np.int64)
    rec = np.array([[_node(20.0 * r, h), _node(20.0, h)] for r in range(201)], np.int64)
    freqs = np.array([3.0, 4.0, 5.0, 6.0])
    true = Model("c4_true_401x201", c_true, h, src, freqs, rec, seed=seed)
    start = Model("c4_start_401x201", c0, h, src.copy(), freqs.copy(), rec.copy(), seed=seed)
    return true, start


def layered_model(rng, Px: int, Pz: int, h: float, nlayers: int,
                  vmin: float = 1500.0, vmax: float = 4500.0) -> np.ndarray:
    """Random horizontal layers: sorted uniform interface depths, uniform velocities."""
    _, Z = _grid(Px, Pz, h)
    depths = np.sort(rng.uniform(0.0, (Pz - 1) * h, nlayers - 1))
    vel = rng.uniform(vmin, vmax, nlayers)
    return vel[np.searchsorted(depths, Z)]


def c5_request(i: int, sizes=(128, 256, 512, 1024)) -> Model:
    """One serving request: seed 5 + i.

    Square physical grid drawn from ``sizes``, frequency uniform in [2, 25] Hz with
    h = 1500 / (10 f) (ten points per wavelength at 1500 m/s), 4..12 random layers
    in [1500, 4500] m/s, one source at the surface centre.
    """
    rng = np.random.default_rng(5 + i)
    n = int(rng.choice(np.asarray(sizes)))
    f = float(rng.uniform(2.0, 25.0))
    h = 1500.0 / (10.0 * f)
    nl = int(rng.integers(4, 13))
    c = layered_model(rng, n, n, h, nl)
    src = np.array([[n // 2, 2]], np.int64)
    return Model(f"c5_req{i}_{n}", c, h, src, np.array([f]), seed=5 + i)


def gardner_density(velocity: np.ndarray) -> np.ndarray:
    """Density (g/cm^3) from velocity (m/s) by Gardner's empirical relation
    0.31 c^0.25: a layered density that follows the velocity model, as input for
    the variable-density operator."""
    return 0.31 * np.asarray(velocity, np.float64) ** 0.25


def random_complex(rng, shape, dtype=np.complex128) -> np.ndarray:
    """Standard complex normal samples (real and imaginary parts N(0, 1/2))."""
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return (a / np.sqrt(2.0)).astype(dtype)
