"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module draws the observation geometry and the source catalogue only.  It
holds none of the method's arithmetic: no visibility model (Eq. 1), no phase
shift, no facet and no likelihood.  Model visibilities of the "observed" data
are produced by whichever side needs them (the oracle in the parity tests, the
library's own sky-model call in the benchmark).

Geometry follows the standard Earth-rotation synthesis relation between an
equatorial baseline (X, Y, Z) and (u, v, w) for hour angle H and declination
dec (Thompson, Moran & Swenson, eq. 4.1; cited by Sec. 2.2 of the paper).

Workloads (sizes of the paper's SKA-MID simulations, Sec. 4 and Sec. 5):
  small    : 64 antennas uniform in a 5 km-radius disk (2016 baselines), 60 time
             steps over +-4 h, 1 channel at 1.0 GHz, 10 sources in 0.1 x 0.1 deg.
  mid      : 197 antennas, radius log-uniform in [100 m, 75 km] (19306
             baselines), 240 x 60 s, 8 channels of 30 MHz centred 965..1175 MHz,
             200 sources in 0.5 x 0.5 deg.
  batched  : 197 antennas as above, 480 x 60 s (8 h), 16 channels of 15 MHz over
             1280..1520 MHz, 1000 sources in a 20' x 20' box.
Fluxes are log-uniform in 50..200 uJy, scalelengths log-normal (median 0.8",
sigma_ln 0.3) and e1, e2 ~ N(0, 0.3^2) redrawn until |e| < 0.8.  The
catalogue is ordered by decreasing flux, ties by index (Sec. 2.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299792458.0
ARCSEC = math.pi / 648000.0
DEG = math.pi / 180.0


@dataclasses.dataclass
class Observation:
    u: np.ndarray          # [n_rows] metres, float64
    v: np.ndarray
    w: np.ndarray
    freq_hz: np.ndarray    # [n_chan] float64, uniformly spaced
    n_ant: int
    n_bl: int
    n_time: int
    nu_ref_hz: float

    @property
    def n_rows(self) -> int:
        return int(self.u.shape[0])

    @property
    def n_chan(self) -> int:
        return int(self.freq_hz.shape[0])


@dataclasses.dataclass
class Catalogue:
    l: np.ndarray            # direction cosines, float64
    m: np.ndarray
    flux_jy: np.ndarray      # float64, decreasing
    alpha_arcsec: np.ndarray # true scalelength (arcsec)
    e1: np.ndarray           # true ellipticity
    e2: np.ndarray

    @property
    def n_src(self) -> int:
        return int(self.l.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    n_ant: int
    layout: str              # "disk" or "logradial"
    r_min_m: float
    r_max_m: float
    n_time: int
    dt_s: float              # seconds between time steps (0 -> spread over span)
    span_h: float            # hour-angle span (hours), centred on transit
    n_chan: int
    f_lo_hz: float           # lower band edge
    f_hi_hz: float           # upper band edge
    nu_ref_hz: float
    n_src: int
    field_rad: float         # side of the square source field
    sigma_jy: float          # noise per visibility component
    seed: int
    lat_rad: float = -30.7 * DEG
    dec_rad: float = -30.0 * DEG


WORKLOADS = {
    "small": Workload("small", 64, "disk", 0.0, 5000.0, 60, 0.0, 8.0, 1,
                      1.0e9, 1.0e9, 1.0e9, 10, 0.1 * DEG, 1e-6, 1),
    "mid": Workload("mid", 197, "logradial", 100.0, 75000.0, 240, 60.0, 4.0, 8,
                    950e6, 1190e6, 1.07e9, 200, 0.5 * DEG, 1e-6, 2),
    "batched": Workload("batched", 197, "logradial", 100.0, 75000.0, 480, 60.0, 8.0, 16,
                        1280e6, 1520e6, 1.4e9, 1000, 20.0 / 60.0 * DEG, 1e-6, 4),
}


def _streams(seed: int, n: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def antenna_enu(wl: Workload, rng: np.random.Generator) -> np.ndarray:
    """Antenna (east, north) positions in metres, [n_ant, 2]."""
    az = rng.uniform(0.0, 2.0 * math.pi, wl.n_ant)
    if wl.layout == "disk":
        r = wl.r_max_m * np.sqrt(rng.uniform(0.0, 1.0, wl.n_ant))
    elif wl.layout == "logradial":
        r = np.exp(rng.uniform(math.log(wl.r_min_m), math.log(wl.r_max_m), wl.n_ant))
    else:
        raise ValueError(wl.layout)
    return np.stack([r * np.sin(az), r * np.cos(az)], axis=1)


def hour_angles(wl: Workload) -> np.ndarray:
    """Hour angles (radians) of the time steps, centred on transit."""
    if wl.dt_s > 0:
        t = (np.arange(wl.n_time) - (wl.n_time - 1) / 2.0) * wl.dt_s
    else:
        span = wl.span_h * 3600.0
        t = -span / 2 + (np.arange(wl.n_time) + 0.5) * span / wl.n_time
    # sidereal rate: 2 pi per 86164.0905 s
    return t * (2.0 * math.pi / 86164.0905)


def baselines_xyz(enu: np.ndarray, lat: float) -> np.ndarray:
    """Equatorial baseline vectors (X, Y, Z) in metres for every antenna pair a < b."""
    n = enu.shape[0]
    a, b = np.triu_indices(n, k=1)
    d = enu[b] - enu[a]
    east, north = d[:, 0], d[:, 1]
    up = np.zeros_like(east)
    x = -math.sin(lat) * north + math.cos(lat) * up
    y = east
    z = math.cos(lat) * north + math.sin(lat) * up
    return np.stack([x, y, z], axis=1)


def uvw_rows(xyz: np.ndarray, ha: np.ndarray, dec: float):
    """(u, v, w) in metres, time-major rows: row = t * n_bl + baseline."""
    X = xyz[None, :, 0]
    Y = xyz[None, :, 1]
    Z = xyz[None, :, 2]
    sH = np.sin(ha)[:, None]
    cH = np.cos(ha)[:, None]
    sd, cd = math.sin(dec), math.cos(dec)
    u = sH * X + cH * Y
    v = -sd * cH * X + sd * sH * Y + cd * Z
    w = cd * cH * X - cd * sH * Y + sd * Z
    return u.reshape(-1).copy(), v.reshape(-1).copy(), w.reshape(-1).copy()


def channel_freqs(wl: Workload) -> np.ndarray:
    if wl.n_chan == 1:
        return np.array([0.5 * (wl.f_lo_hz + wl.f_hi_hz)], dtype=np.float64)
    width = (wl.f_hi_hz - wl.f_lo_hz) / wl.n_chan
    return wl.f_lo_hz + (np.arange(wl.n_chan) + 0.5) * width


def make_observation(wl: Workload) -> Observation:
    rng_ant, _, _ = _streams(wl.seed, 3)
    enu = antenna_enu(wl, rng_ant)
    xyz = baselines_xyz(enu, wl.lat_rad)
    u, v, w = uvw_rows(xyz, hour_angles(wl), wl.dec_rad)
    return Observation(u=u, v=v, w=w, freq_hz=channel_freqs(wl), n_ant=wl.n_ant,
                       n_bl=xyz.shape[0], n_time=wl.n_time, nu_ref_hz=wl.nu_ref_hz)


def make_catalogue(wl: Workload, n_src: int | None = None) -> Catalogue:
    _, rng_cat, _ = _streams(wl.seed, 3)
    n = wl.n_src if n_src is None else n_src
    half = wl.field_rad / 2.0
    l = rng_cat.uniform(-half, half, n)
    m = rng_cat.uniform(-half, half, n)
    flux = np.exp(rng_cat.uniform(math.log(50e-6), math.log(200e-6), n))
    alpha = 0.8 * np.exp(0.3 * rng_cat.standard_normal(n))
    e1 = np.empty(n)
    e2 = np.empty(n)
    for i in range(n):
        while True:
            a, b = rng_cat.normal(0.0, 0.3, 2)
            if a * a + b * b < 0.64:
                e1[i], e2[i] = a, b
                break
    order = np.argsort(-flux, kind="stable")
    return Catalogue(l=l[order], m=m[order], flux_jy=flux[order],
                     alpha_arcsec=alpha[order], e1=e1[order], e2=e2[order])


def noise(n_rows: int, n_chan: int, sigma: float, seed: int, dtype=np.float32) -> np.ndarray:
    """Gaussian noise N(0, sigma^2) on the real and imaginary parts, [n_rows, n_chan, 2]."""
    _, _, rng_noise = _streams(seed, 3)
    out = rng_noise.standard_normal((n_rows, n_chan, 2), dtype=np.float32)
    out *= np.float32(sigma)
    return out.astype(dtype, copy=False)


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def tiny(seed: int = 7, n_ant: int = 12, n_time: int = 9, n_chan: int = 3,
         n_src: int = 4, r_max_m: float = 3000.0) -> Workload:
    """A small custom workload for fast tests (several tiles, ragged tails)."""
    return Workload("tiny", n_ant, "disk", 0.0, r_max_m, n_time, 0.0, 6.0, n_chan,
                    990e6, 1010e6 + (n_chan - 1) * 0.0, 1.0e9, n_src, 0.05 * DEG, 1e-6, seed)
