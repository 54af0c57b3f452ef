"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the FP64 oracle's callers.
It draws random numbers and lays out trajectories, lever arms, pixel grids,
scatterer lists and band-limited noise.  It holds none of the backprojection
arithmetic: no rotations, no ranges, no delays, no interpolation.

The paper's own data (a stripmap wreck survey and a near-field sub-bottom
volume, Sec. III-A/B) and its timing dataset (Sec. III-C) are not available;
these generators stand in for them with the sizes of the five workloads:

  small_2d      128 pings x 4 RX x 2048 samples, 256^2 pixels at 2 cm (straight track)
  stripmap_2d   2048 pings x 32 RX x 16384 samples, 4096^2 pixels at 1.5 cm, motion
  volume_3d     1024 pings (32x32 lattice) x 64 RX (8x8) x 8192 samples, 1024^2 x 128 voxels at 2 cm
  learned_2d    small_2d geometry with 16-bit echoes and the learned interpolator
  autofocus_2d  1024 pings x 16 RX x 8192 samples, 2048^2 pixels at 1.5 cm, nav error 2 cm

Frame: north-east-down (x along-track, y cross-track, z down); the origin is
on the seafloor below the first ping, so the platform sits at negative z.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

FC = 100e3          # carrier [Hz]
BANDWIDTH = 20e3    # LFM bandwidth [Hz]
FS = 40e3           # complex baseband sample rate [Hz]
C_SOUND = 1500.0    # sound speed [m/s]
PULSE_T = 5e-3      # LFM length [s]
NU_BAND = BANDWIDTH / (2.0 * FS)   # one-sided band edge in cycles/sample (0.25)


@dataclass(frozen=True)
class Grid:
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int = 1

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass(frozen=True)
class Workload:
    name: str
    n_pings: int
    n_rx: int
    n_samples: int
    t0: float
    grid: Grid
    array: str = "line"            # "line": RX along-track; "planar": 8x8 in body x-y
    ping_spacing: float = 0.1
    altitude: float = 10.0
    rx_pitch: float = 0.025
    lattice: int = 0               # >0: pings on a lattice x lattice grid (3D collection)
    lattice_pitch: float = 0.64
    motion: bool = False
    speed: float = 1.95            # along-track speed [m/s] (sets the ping interval and the velocity)
    nav_error: float = 0.0         # std of per-axis position error added to nav [m]
    n_points: int = 10
    point_patch: tuple = ()        # (x_lo, x_hi, y_lo, y_hi, z)
    echo_dtype: str = "c64"
    taps: int = 8
    seed: int = 1234
    extra: dict = field(default_factory=dict)

    @property
    def updates(self) -> int:
        return self.grid.n * self.n_pings * self.n_rx


def _stripmap_grid(P, spacing, nx, ny, d, y0):
    track = P * spacing
    x0 = 0.5 * (track - nx * d)
    return Grid(x0, y0, 0.0, d, d, 0.0, nx, ny, 1)


WORKLOADS = {
    "small_2d": Workload(
        "small_2d", 128, 4, 2048, 0.025, _stripmap_grid(128, 0.1, 256, 256, 0.02, 20.0),
        n_points=10, point_patch=(0.0, 0.0, 20.0, 25.0, 0.0), seed=1235),
    "stripmap_2d": Workload(
        "stripmap_2d", 2048, 32, 16384, 0.05, _stripmap_grid(2048, 0.1, 4096, 4096, 0.015, 40.0),
        motion=True, n_points=200, seed=1236),
    "volume_3d": Workload(
        "volume_3d", 1024, 64, 8192, 0.0,
        Grid(0.5 * (32 * 0.64 - 1024 * 0.02), 0.5 * (32 * 0.64 - 1024 * 0.02), 0.0,
             0.02, 0.02, 0.02, 1024, 1024, 128),
        array="planar", rx_pitch=0.02, altitude=2.0, lattice=32, lattice_pitch=0.64,
        motion=True, n_points=64, echo_dtype="f16", seed=1237),
    "learned_2d": Workload(
        "learned_2d", 128, 4, 2048, 0.025, _stripmap_grid(128, 0.1, 256, 256, 0.02, 20.0),
        n_points=10, point_patch=(0.0, 0.0, 20.0, 25.0, 0.0), echo_dtype="bf16", seed=1238),
    "autofocus_2d": Workload(
        "autofocus_2d", 1024, 16, 8192, 0.04, _stripmap_grid(1024, 0.1, 2048, 2048, 0.015, 30.0),
        nav_error=0.02, n_points=100, seed=1239),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return replace(w, **overrides) if overrides else w


def scaled(w: Workload, n_pings: int | None = None, n_rx: int | None = None,
           nx: int | None = None, ny: int | None = None, nz: int | None = None,
           n_samples: int | None = None) -> Workload:
    """Same geometry family with fewer pings / channels / pixels (parity cases)."""
    g = w.grid
    g2 = replace(g, nx=nx or g.nx, ny=ny or g.ny, nz=nz or g.nz)
    return replace(w, n_pings=n_pings or w.n_pings, n_rx=n_rx or w.n_rx,
                   n_samples=n_samples or w.n_samples, grid=g2)


# --------------------------------------------------------------------------
# Navigation: vehicle positions and attitude per ping, lever arms.

def nav(w: Workload, seed_offset: int = 0):
    """Returns dict(pos [P,3], att [P,3] (roll, pitch, yaw rad), tx_lever [3],
    rx_lever [C,3], true_pos [P,3], vel [P,3]).  ``pos`` includes the
    navigation error (if any); ``true_pos`` is what the echoes are simulated
    from; ``vel`` is the platform velocity at each ping [m/s] (along-track
    speed plus the rates of the sway and heave sinusoids; zero on a lattice),
    the receiver velocity during reception when continuous motion is
    modelled."""
    rng = np.random.default_rng(w.seed + 17 * seed_offset)
    P, C = w.n_pings, w.n_rx
    if w.lattice:
        L = w.lattice
        i = np.arange(P)
        ix, iy = i % L, i // L
        pos = np.stack([ix * w.lattice_pitch, iy * w.lattice_pitch, np.full(P, -w.altitude)], 1)
    else:
        pos = np.stack([np.arange(P) * w.ping_spacing, np.zeros(P), np.full(P, -w.altitude)], 1)
    att = np.zeros((P, 3))
    vel = np.zeros((P, 3))
    if not w.lattice:
        vel[:, 0] = w.speed
    if w.motion:
        i = np.arange(P)
        t_sway, t_heave = rng.uniform(20.0, 60.0, size=2)
        p_sway, p_heave = rng.uniform(0.0, 2.0 * np.pi, size=2)
        pos[:, 1] += 0.05 * np.sin(2.0 * np.pi * i / t_sway + p_sway)
        pos[:, 2] += 0.05 * np.sin(2.0 * np.pi * i / t_heave + p_heave)
        att[:, 2] = np.cumsum(rng.normal(0.0, np.deg2rad(0.01), size=P))
        if not w.lattice:
            pings_per_s = w.speed / w.ping_spacing
            vel[:, 1] = 0.05 * 2.0 * np.pi / t_sway * pings_per_s * np.cos(2.0 * np.pi * i / t_sway + p_sway)
            vel[:, 2] = 0.05 * 2.0 * np.pi / t_heave * pings_per_s * np.cos(2.0 * np.pi * i / t_heave + p_heave)
    if w.array == "planar":
        n = int(round(np.sqrt(C)))
        assert n * n == C
        a = (np.arange(n) - 0.5 * (n - 1)) * w.rx_pitch
        gx, gy = np.meshgrid(a, a, indexing="xy")
        rx = np.stack([gx.reshape(-1), gy.reshape(-1), np.zeros(C)], 1)
    else:
        rx = np.stack([(np.arange(C) - 0.5 * (C - 1)) * w.rx_pitch, np.zeros(C), np.zeros(C)], 1)
    tx = np.zeros(3)
    true_pos = pos.copy()
    if w.nav_error > 0:
        pos = pos + rng.normal(0.0, w.nav_error, size=pos.shape)
    return dict(pos=pos, att=att, tx_lever=tx, rx_lever=rx, true_pos=true_pos, vel=vel)


def scatterers(w: Workload, seed_offset: int = 0) -> np.ndarray:
    """Point scatterers [n,5] = (x, y, z, Re A, Im A), |A| ~ U[0.5, 1], uniform phase.
    Placed on pixel centres inside the patch (or the whole grid)."""
    rng = np.random.default_rng(w.seed + 1000 + seed_offset)
    g = w.grid
    n = w.n_points
    if w.point_patch:
        _, _, ylo, yhi, z = w.point_patch
        iy_lo = int(np.ceil((ylo - g.y0) / g.dy))
        iy_hi = int(np.floor((yhi - g.y0) / g.dy))
        iy_lo, iy_hi = max(iy_lo, 0), min(iy_hi, g.ny - 1)
    else:
        iy_lo, iy_hi = 0, g.ny - 1
    ix = rng.integers(8, g.nx - 8, size=n)
    iy = rng.integers(iy_lo + 8 if iy_hi - iy_lo > 16 else iy_lo, max(iy_hi - 8, iy_lo + 1), size=n)
    iz = rng.integers(0, g.nz, size=n)
    amp = rng.uniform(0.5, 1.0, size=n)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n)
    pts = np.stack([g.x0 + ix * g.dx, g.y0 + iy * g.dy, g.z0 + iz * g.dz,
                    amp * np.cos(ph), amp * np.sin(ph)], 1)
    return pts


def scatterer_indices(w: Workload, scat: np.ndarray) -> np.ndarray:
    """Integer pixel indices (ix, iy, iz) of scatterers placed by ``scatterers``."""
    g = w.grid
    ix = np.rint((scat[:, 0] - g.x0) / g.dx).astype(np.int64)
    iy = np.rint((scat[:, 1] - g.y0) / g.dy).astype(np.int64)
    iz = np.zeros_like(ix) if g.nz == 1 else np.rint((scat[:, 2] - g.z0) / g.dz).astype(np.int64)
    return np.stack([ix, iy, iz], 1)


# --------------------------------------------------------------------------
# Noise and random echoes

def bandlimited_noise(shape, nu_b: float, power: float, seed: int) -> np.ndarray:
    """Complex Gaussian noise, flat spectrum on |nu| <= nu_b cycles/sample
    along the last axis, mean power ``power`` per sample (complex128)."""
    rng = np.random.default_rng(seed)
    n = shape[-1]
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Z = np.fft.fft(z, axis=-1)
    nu = np.fft.fftfreq(n)
    Z[..., np.abs(nu) > nu_b] = 0.0
    x = np.fft.ifft(Z, axis=-1)
    x *= np.sqrt(power / np.mean(np.abs(x) ** 2))
    return x


def snr_noise_power(scat: np.ndarray, snr_db: float = 20.0) -> float:
    """Noise power per sample relative to the unit-peak compressed pulse:
    mean(|A|^2) / 10^(SNR/10)."""
    return float(np.mean(scat[:, 3] ** 2 + scat[:, 4] ** 2) / 10.0 ** (snr_db / 10.0))


def random_echo(P: int, C: int, Ns: int, seed: int, nu_b: float = NU_BAND, pool: int = 64,
                dtype=np.complex64, out: np.ndarray | None = None) -> np.ndarray:
    """Echo-shaped random input [P,C,Ns]: every row is a band-limited complex
    Gaussian realisation (the statistics of a range-compressed speckle echo),
    drawn from a pool of ``pool`` independent rows with a random circular shift
    and random phase per row.  Deterministic in ``seed``."""
    rng = np.random.default_rng(seed)
    base = bandlimited_noise((pool, Ns), nu_b, 1.0, seed + 1).astype(np.complex64)
    rows = P * C
    which = rng.integers(0, pool, size=rows)
    shift = rng.integers(0, Ns, size=rows)
    phase = np.exp(1j * rng.uniform(0, 2 * np.pi, size=rows)).astype(np.complex64)
    if out is None:
        out = np.empty((P, C, Ns), dtype=dtype)
    flat = out.reshape(rows, Ns)
    for r in range(rows):
        s = int(shift[r])
        src = base[which[r]]
        flat[r, : Ns - s] = src[s:] * phase[r]
        flat[r, Ns - s:] = src[:s] * phase[r]
    return out


def random_image(shape, seed: int) -> np.ndarray:
    """Complex Gaussian image (unit power), for adjoint / VJP inputs."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def random_pixel_indices(g: Grid, n: int, seed: int) -> np.ndarray:
    """n random (ix, iy, iz) inside the grid."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, g.nx, n), rng.integers(0, g.ny, n), rng.integers(0, g.nz, n)], 1)


def training_draws(n: int, rows: int, lo: int, hi: int, seed: int):
    """Learned-interpolator training draws: fractions U[0,1), echo row, sample index."""
    rng = np.random.default_rng(seed)
    return (rng.random(n), rng.integers(0, rows, n), rng.integers(lo, hi, n))
