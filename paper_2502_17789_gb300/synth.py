"""Seeded synthetic inputs for the IDG workloads.

This module only *makes inputs*: station layouts, earth-rotation uvw tracks,
frequencies, A-term samples, point-source skies and the visibilities those
skies produce.  It holds none of the gridding / degridding arithmetic, and it
is the only code shared by the GPU path's tests and the oracle's tests.

Recipes:
  * stations on a flat array at the MWA latitude (-26.703 deg), pointing at
    declination -27 deg, hour angle centred on transit; uvw from the textbook
    ENU -> equatorial -> (u,v,w) rotation (Thompson, Moran & Swenson, ch. 4);
  * point sources with log-normal fluxes (mu=0, sigma=1 Jy) uniform in a
    square field; visibilities are their sum through the measurement equation
    with the same A-term model, plus complex Gaussian noise;
  * A-terms: identity, random complex Jones (tests), or a Gaussian primary
    beam times the phase of a thin Kolmogorov screen at 100 km height.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPEED_OF_LIGHT = 299792458.0
EARTH_ROTATION = 7.2921e-5  # rad / s
MWA_LATITUDE = np.deg2rad(-26.703)
DECLINATION = np.deg2rad(-27.0)


@dataclass
class Observation:
    n_stations: int
    baselines: np.ndarray        # int32 [n_bl, 2], p < q
    uvw: np.ndarray              # float64 [n_bl, n_t, 3] metres
    freqs: np.ndarray            # float64 [n_ch] Hz, ascending
    aterm_offsets: np.ndarray    # int32 [n_int + 1] timestep boundaries
    times: np.ndarray            # float64 [n_t] seconds from transit
    enu: np.ndarray              # float64 [n_st, 3] station positions
    grid_size: int
    subgrid_size: int
    kernel_padding: int
    image_size: float
    aterm_nodes: int = 9
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_baselines(self) -> int:
        return int(self.baselines.shape[0])

    @property
    def n_timesteps(self) -> int:
        return int(self.uvw.shape[1])

    @property
    def n_channels(self) -> int:
        return int(self.freqs.shape[0])

    @property
    def n_intervals(self) -> int:
        return int(self.aterm_offsets.shape[0] - 1)

    @property
    def n_vis(self) -> int:
        return self.n_baselines * self.n_timesteps * self.n_channels


# ---------------------------------------------------------------------------
# array layouts and uvw tracks
# ---------------------------------------------------------------------------

def stations_uniform_disk(rng: np.random.Generator, n: int, diameter_m: float) -> np.ndarray:
    r = 0.5 * diameter_m * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n)], axis=1)


def stations_lognormal(rng: np.random.Generator, n: int, median_m: float, sigma: float,
                       clip_m: float) -> np.ndarray:
    r = np.minimum(np.exp(np.log(median_m) + sigma * rng.standard_normal(n)), clip_m)
    th = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n)], axis=1)


def all_pairs(n_st: int) -> np.ndarray:
    p, q = np.triu_indices(n_st, k=1)
    return np.stack([p, q], axis=1).astype(np.int32)


def uvw_tracks(enu: np.ndarray, pairs: np.ndarray, hour_angles: np.ndarray,
               lat: float = MWA_LATITUDE, dec: float = DECLINATION) -> np.ndarray:
    """Baseline vectors (q - p) rotated to (u,v,w) metres, [n_bl, n_t, 3]."""
    d = enu[pairs[:, 1]] - enu[pairs[:, 0]]
    E, N, U = d[:, 0], d[:, 1], d[:, 2]
    X = -np.sin(lat) * N + np.cos(lat) * U
    Y = E
    Z = np.cos(lat) * N + np.sin(lat) * U
    H = hour_angles[None, :]
    X, Y, Z = X[:, None], Y[:, None], Z[:, None]
    u = np.sin(H) * X + np.cos(H) * Y
    v = -np.sin(dec) * np.cos(H) * X + np.sin(dec) * np.sin(H) * Y + np.cos(dec) * Z
    w = np.cos(dec) * np.cos(H) * X - np.cos(dec) * np.sin(H) * Y + np.sin(dec) * Z
    return np.ascontiguousarray(np.stack([u, v, w], axis=2))


def make_observation(enu, n_t, dt, freqs, steps_per_interval, grid_size, subgrid_size,
                     kernel_padding, image_size, aterm_nodes=9, name="", pairs=None) -> Observation:
    pairs = all_pairs(enu.shape[0]) if pairs is None else np.asarray(pairs, np.int32)
    times = (np.arange(n_t) - 0.5 * (n_t - 1)) * dt
    uvw = uvw_tracks(enu, pairs, times * EARTH_ROTATION)
    offs = list(range(0, n_t, max(1, steps_per_interval))) + [n_t] if n_t > 0 else [0, 0]
    if n_t > 0 and offs[0] != 0:
        offs = [0] + offs
    return Observation(int(enu.shape[0]), pairs, uvw, np.asarray(freqs, np.float64),
                       np.asarray(offs, np.int32), times, enu, grid_size, subgrid_size,
                       kernel_padding, image_size, aterm_nodes, name)


# ---------------------------------------------------------------------------
# the five workloads (scale < 1 shrinks stations / timesteps for tests)
# ---------------------------------------------------------------------------

def config(idx: int, seed: int = 0, subgrid_size: int | None = None, n_stations: int | None = None,
           n_timesteps: int | None = None, n_channels: int | None = None) -> Observation:
    """Observation of workload `idx` (1..4); optional overrides shrink it."""
    rng = np.random.default_rng(seed)
    if idx == 1:
        n_st = n_stations or 32
        enu = stations_uniform_disk(rng, n_st, 1000.0)
        n_t = 16 if n_timesteps is None else n_timesteps
        n_ch = n_channels or 8
        freqs = 150e6 + 1e6 * np.arange(n_ch)
        return make_observation(enu, n_t, 8.0, freqs, max(n_t, 1), 512, subgrid_size or 32, 12, 0.35,
                                name="small-32-stations")
    if idx in (2, 3):
        n_st = n_stations or 128
        enu = stations_uniform_disk(rng, n_st, 3000.0)
        n_t = 56 if n_timesteps is None else n_timesteps
        n_ch = n_channels or 24
        freqs = np.linspace(140e6, 170e6, n_ch)
        return make_observation(enu, n_t, 2.0, freqs, 4, 4096, subgrid_size or 96, 18, 0.5,
                                name="mwa-like-128-stations" if idx == 2 else "mixed-precision-1000-sources")
    if idx == 4:
        n_st = n_stations or 256
        enu = stations_lognormal(rng, n_st, 300.0, 1.0, 3000.0)
        n_t = 360 if n_timesteps is None else n_timesteps
        n_ch = n_channels or 30
        freqs = np.linspace(140e6, 170e6, n_ch)
        return make_observation(enu, n_t, 0.5, freqs, 8, 8192, subgrid_size or 96, 18, 0.5,
                                name="uneven-256-stations")
    raise ValueError(f"unknown workload {idx}")


# ---------------------------------------------------------------------------
# A-terms: [n_int][n_st][nodes][nodes][4] complex64, node (a_m, a_l)
# ---------------------------------------------------------------------------

def node_coords(image_size: float, nodes: int) -> np.ndarray:
    return -0.5 * image_size + image_size * np.arange(nodes) / (nodes - 1)


def aterms_identity(n_int: int, n_st: int, nodes: int = 9) -> np.ndarray:
    a = np.zeros((n_int, n_st, nodes, nodes, 4), np.complex64)
    a[..., 0] = 1
    a[..., 3] = 1
    return a


def aterms_random(rng: np.random.Generator, n_int: int, n_st: int, nodes: int = 9,
                  leakage: float = 0.3) -> np.ndarray:
    """Smooth-ish random full Jones matrices (diagonal near 1, off-diagonal
    leakage), complex64."""
    shape = (n_int, n_st, nodes, nodes)
    a = np.zeros(shape + (4,), np.complex128)
    for e in range(4):
        z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        a[..., e] = (1.0 if e in (0, 3) else 0.0) + (0.3 if e in (0, 3) else leakage) * z
    return a.astype(np.complex64)


def aterms_with_leakage(rng: np.random.Generator, aterms: np.ndarray, leakage: float) -> np.ndarray:
    """Add polarisation leakage to A-terms: off-diagonal entries equal to
    `leakage` times a unit complex Gaussian times the mean diagonal, so that
    every Jones matrix is full (complex64)."""
    a = np.array(aterms, dtype=np.complex128, copy=True)
    scale = 0.5 * (a[..., 0] + a[..., 3])
    for e in (1, 2):
        z = (rng.standard_normal(a.shape[:-1]) + 1j * rng.standard_normal(a.shape[:-1])) / np.sqrt(2.0)
        a[..., e] += leakage * z * scale
    return a.astype(np.complex64)


def kolmogorov_screen(rng: np.random.Generator, n: int, rms_rad: float) -> np.ndarray:
    """Real random field with a k^(-11/3) power spectrum on an n x n grid,
    scaled to the requested rms phase."""
    k = np.fft.fftfreq(n)
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    kk[0, 0] = np.inf
    amp = kk ** (-11.0 / 6.0)
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    f = np.real(np.fft.ifft2(z * amp))
    f -= f.mean()
    return f * (rms_rad / f.std())


@dataclass
class BeamScreen:
    """Gaussian beam x ionospheric phase screen (the A-term model)."""
    screen: np.ndarray      # phase [n, n] radians
    pixel_m: float
    height_m: float
    wind_mps: float
    fwhm_rad: float

    def _phase(self, x_m, y_m):
        n = self.screen.shape[0]
        gx = x_m / self.pixel_m + 0.5 * n
        gy = y_m / self.pixel_m + 0.5 * n
        gx = np.clip(gx, 0, n - 1.001)
        gy = np.clip(gy, 0, n - 1.001)
        ix, iy = np.floor(gx).astype(int), np.floor(gy).astype(int)
        fx, fy = gx - ix, gy - iy
        s = self.screen
        return ((1 - fx) * (1 - fy) * s[iy, ix] + fx * (1 - fy) * s[iy, ix + 1]
                + (1 - fx) * fy * s[iy + 1, ix] + fx * fy * s[iy + 1, ix + 1])

    def gain(self, enu: np.ndarray, t_s: float, l: np.ndarray, m: np.ndarray) -> np.ndarray:
        """Scalar complex gain [n_st, *l.shape] for directions (l, m) at time t."""
        n = np.sqrt(np.maximum(1.0 - l * l - m * m, 1e-6))
        beam = np.exp(-4.0 * np.log(2.0) * (l * l + m * m) / self.fwhm_rad ** 2)
        px = enu[:, 0].reshape((-1,) + (1,) * l.ndim) + self.height_m * l / n + self.wind_mps * t_s
        py = enu[:, 1].reshape((-1,) + (1,) * l.ndim) + self.height_m * m / n
        return beam * np.exp(1j * self._phase(px, py))


def beam_screen_model(rng: np.random.Generator, rms_rad: float = 2.0) -> BeamScreen:
    return BeamScreen(kolmogorov_screen(rng, 600, rms_rad), 100.0, 100e3, 50.0, 0.35)


def aterms_beam_screen(obs: Observation, model: BeamScreen) -> np.ndarray:
    nodes = obs.aterm_nodes
    c = node_coords(obs.image_size, nodes)
    mm, ll = np.meshgrid(c, c, indexing="ij")  # [a_m, a_l]
    out = np.zeros((obs.n_intervals, obs.n_stations, nodes, nodes, 4), np.complex64)
    for a in range(obs.n_intervals):
        t0, t1 = obs.aterm_offsets[a], obs.aterm_offsets[a + 1]
        tm = float(np.mean(obs.times[t0:t1])) if t1 > t0 else 0.0
        g = model.gain(obs.enu, tm, ll, mm)
        out[a, :, :, :, 0] = g
        out[a, :, :, :, 3] = g
    return out


# ---------------------------------------------------------------------------
# skies and visibilities
# ---------------------------------------------------------------------------

@dataclass
class Sky:
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray


def point_sources(rng: np.random.Generator, n: int, half_width: float) -> Sky:
    return Sky(rng.uniform(-half_width, half_width, n), rng.uniform(-half_width, half_width, n),
               np.exp(rng.standard_normal(n)))


def random_visibilities(rng: np.random.Generator, obs: Observation, sigma: float = 1.0) -> np.ndarray:
    shape = (obs.n_baselines, obs.n_timesteps, obs.n_channels, 4)
    v = sigma * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return v.astype(np.complex64)


def simulate_visibilities(obs: Observation, sky: Sky, model: BeamScreen | None = None,
                          noise_sigma: float = 0.0, rng: np.random.Generator | None = None,
                          device: str = "cpu"):
    """Unpolarised point sources observed through scalar station gains
    (identity when `model` is None): V_pq = sum_s S g_p conj(g_q) I_2
    exp(-2 pi i (u l + v m + w (n - 1))), plus complex Gaussian noise.
    Returns complex64 [n_bl, n_t, n_ch, 4] as a numpy array (device='cpu')
    or a torch tensor on `device`."""
    import torch

    dev = torch.device(device)
    n_bl, n_t, n_ch = obs.n_baselines, obs.n_timesteps, obs.n_channels
    uvw = torch.as_tensor(obs.uvw, dtype=torch.float64, device=dev)
    fc = torch.as_tensor(obs.freqs / SPEED_OF_LIGHT, dtype=torch.float64, device=dev)
    t_int = np.zeros(n_t, np.int64)
    for a in range(obs.n_intervals):
        t_int[obs.aterm_offsets[a]:obs.aterm_offsets[a + 1]] = a
    t_int = torch.as_tensor(t_int, device=dev)
    p = torch.as_tensor(obs.baselines[:, 0].astype(np.int64), device=dev)
    q = torch.as_tensor(obs.baselines[:, 1].astype(np.int64), device=dev)
    acc = torch.zeros((n_bl, n_t, n_ch), dtype=torch.complex128, device=dev)
    for s in range(len(sky.flux)):
        l, m = float(sky.l[s]), float(sky.m[s])
        n1 = np.sqrt(1.0 - l * l - m * m) - 1.0
        D = uvw[..., 0] * l + uvw[..., 1] * m + uvw[..., 2] * n1          # metres [bl, t]
        ph = -2.0 * np.pi * D[..., None] * fc[None, None, :]             # radians [bl, t, ch]
        e = torch.polar(torch.ones_like(ph), ph)
        if model is None:
            coef = torch.full((n_bl, n_t), float(sky.flux[s]), dtype=torch.complex128, device=dev)
        else:
            g = np.stack([model.gain(obs.enu, float(np.mean(obs.times[obs.aterm_offsets[a]:obs.aterm_offsets[a + 1]])),
                                     np.array(l), np.array(m))
                          for a in range(obs.n_intervals)])  # [n_int, n_st]
            g = torch.as_tensor(g, dtype=torch.complex128, device=dev)
            gi = g[t_int]                                                # [t, st]
            coef = float(sky.flux[s]) * gi[:, p].T * torch.conj(gi[:, q].T)  # [bl, t]
        acc += coef[..., None] * e
    out = torch.zeros((n_bl, n_t, n_ch, 4), dtype=torch.complex64, device=dev)
    out[..., 0] = acc.to(torch.complex64)
    out[..., 3] = acc.to(torch.complex64)
    if noise_sigma > 0:
        g = torch.Generator(device="cpu")
        g.manual_seed(int(rng.integers(0, 2 ** 62)) if rng is not None else 0)
        noise = torch.randn((n_bl, n_t, n_ch, 4, 2), generator=g, dtype=torch.float32) * noise_sigma
        out += torch.view_as_complex(noise).to(dev)
    return out.cpu().numpy() if device == "cpu" else out
