"""Seeded synthetic inputs standing in for the paper's measurement sets.

The paper benchmarks on a MeerKAT L-band measurement set (Sec. 6) that is not available
here; these generators produce inputs with the same structure: an interferometer array with
earth-rotation uvw tracks, several frequency channels, complex visibilities and sparse point-
source images.  This module holds no arithmetic of the gridding method itself; the oracle
and the GPU path both consume what it returns.

Workloads (named by what they are):
  tiny        256^2 image, 0.05 deg pixels, 1e4 single-channel visibilities at 1 GHz with
              uniform random uvw (|u|, |v| <= 0.45 / pixel, w uniform in +-0.5 max|u|).
  wide_2k     2048^2 image, 20 arcsec pixels, 64 antennas (2016 baselines) x 62 time steps
              x 8 channels in 0.9-1.7 GHz = 999,936 visibilities.
  wide_8k     8192^2 image, 4 arcsec pixels, 128 antennas (8128 baselines), 193 time steps
              x 64 channels, truncated to 1,562,500 rows = 1e8 visibilities.
  diff_4k     4096^2 image, 4 arcsec pixels, 64 antennas x 310 time steps x 16 channels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SPEED_OF_LIGHT = 299792458.0
ARCSEC = math.pi / (180.0 * 3600.0)


@dataclass
class Observation:
    uvw: np.ndarray          # (nrows, 3) float64, metres
    freq: np.ndarray         # (nchan,) float64, Hz
    npix_x: int
    npix_y: int
    pixsize_x: float         # radians
    pixsize_y: float
    uv_scale: float = 1.0    # uniform scale applied to the array (see array_uvw)
    name: str = ""

    @property
    def nrows(self):
        return self.uvw.shape[0]

    @property
    def nchan(self):
        return self.freq.size

    @property
    def nvis(self):
        return self.nrows * self.nchan


def antenna_disk(n_ant: int, radius_m: float, rng) -> np.ndarray:
    """Antenna positions uniform in a disk, local (east, north, up=0) metres."""
    r = radius_m * np.sqrt(rng.uniform(0.0, 1.0, n_ant))
    t = rng.uniform(0.0, 2 * np.pi, n_ant)
    return np.stack([r * np.cos(t), r * np.sin(t), np.zeros(n_ant)], axis=1)


def earth_rotation_uvw(enu: np.ndarray, lat_rad: float, dec_rad: float,
                       hour_angles: np.ndarray) -> np.ndarray:
    """uvw (metres) of all baselines i < j over the hour angles (textbook equatorial
    rotation of the ENU baseline vectors).  Rows are ordered time-major."""
    i, j = np.triu_indices(enu.shape[0], k=1)
    b = enu[j] - enu[i]                                    # (nbl, 3) east, north, up
    X = -math.sin(lat_rad) * b[:, 1] + math.cos(lat_rad) * b[:, 2]
    Y = b[:, 0]
    Z = math.cos(lat_rad) * b[:, 1] + math.sin(lat_rad) * b[:, 2]
    H = hour_angles[:, None]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    u = np.sin(H) * X + np.cos(H) * Y
    v = -sd * np.cos(H) * X + sd * np.sin(H) * Y + cd * Z
    w = cd * np.cos(H) * X - cd * np.sin(H) * Y + sd * Z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


def array_observation(n_ant, n_time, n_chan, npix, pixsize, seed=0, radius_m=4000.0,
                      f_lo=0.9e9, f_hi=1.7e9, dec_deg=-30.0, lat_deg=-30.0, ha_hours=4.0,
                      max_rows=None, fill=0.45, name="") -> Observation:
    """Earth-rotation synthesis with an n_ant array in a disk of radius_m.

    The uvw are scaled uniformly by s = min(1, fill / (pixsize * max(|u|, |v|) at f_hi)) so
    that the longest baselines fall inside the uv grid of the requested pixel size (with the
    unscaled 4 km array most visibilities would alias); s is recorded in uv_scale."""
    rng = np.random.default_rng(seed)
    enu = antenna_disk(n_ant, radius_m, rng)
    ha = np.linspace(-ha_hours, ha_hours, n_time) * (np.pi / 12.0)
    uvw = earth_rotation_uvw(enu, math.radians(lat_deg), math.radians(dec_deg), ha)
    if max_rows is not None:
        uvw = uvw[:max_rows]
    freq = np.linspace(f_lo, f_hi, n_chan) if n_chan > 1 else np.array([f_lo])
    umax = np.abs(uvw[:, :2]).max() * freq.max() / SPEED_OF_LIGHT
    s = min(1.0, fill / (pixsize * umax))
    return Observation(np.ascontiguousarray(uvw * s), freq, npix, npix, pixsize, pixsize, s, name)


def tiny(seed=0) -> Observation:
    rng = np.random.default_rng(seed)
    npix, pix = 256, math.radians(0.05)
    f = 1e9
    n = 10_000
    umax = 0.45 / pix
    u = rng.uniform(-umax, umax, n)
    v = rng.uniform(-umax, umax, n)
    w = rng.uniform(-0.5 * umax, 0.5 * umax, n)
    uvw = np.stack([u, v, w], axis=1) * SPEED_OF_LIGHT / f
    return Observation(uvw, np.array([f]), npix, npix, pix, pix, 1.0, "tiny")


def wide_2k(seed=0) -> Observation:
    return array_observation(64, 62, 8, 2048, 20 * ARCSEC, seed=seed, name="wide_2k")


def wide_1k(seed=0) -> Observation:
    """Quarter-size variant of wide_2k (1024^2 at 40 arcsec, 64 antennas x 31 x 8 channels),
    small enough for profiler captures that replay each kernel many times."""
    return array_observation(64, 31, 8, 1024, 40 * ARCSEC, seed=seed, name="wide_1k")


def dense_1k(seed=0) -> Observation:
    """1024^2 at 40 arcsec with 64 antennas x 100 time steps x 8 channels (1.6e6 visibilities):
    about the visibilities per uv cell of wide_8k on a grid small enough for profiler replays."""
    return array_observation(64, 100, 8, 1024, 40 * ARCSEC, seed=seed, name="dense_1k")


def wide_8k(seed=0) -> Observation:
    return array_observation(128, 193, 64, 8192, 4 * ARCSEC, seed=seed, max_rows=1_562_500,
                             name="wide_8k")


def diff_4k(seed=0) -> Observation:
    return array_observation(64, 310, 16, 4096, 4 * ARCSEC, seed=seed, name="diff_4k")


WORKLOADS = {"tiny": tiny, "wide_1k": wide_1k, "dense_1k": dense_1k, "wide_2k": wide_2k,
             "wide_8k": wide_8k,
             "diff_4k": diff_4k}


def random_uvw_observation(nrows, nchan, npix_x, npix_y, fov_deg, seed=0, wfrac=0.5,
                           f_lo=0.9e9, f_hi=1.4e9, fill=0.45) -> Observation:
    """Uniform random uvw inside the uv grid (|u| dl <= fill), w in +-wfrac max|u|."""
    rng = np.random.default_rng(seed)
    psx = math.radians(fov_deg) / npix_x
    psy = math.radians(fov_deg) / npix_y
    freq = np.linspace(f_lo, f_hi, nchan) if nchan > 1 else np.array([f_lo])
    lam_min = SPEED_OF_LIGHT / freq.max()
    umax = fill / psx * lam_min
    vmax = fill / psy * lam_min
    uvw = np.stack([rng.uniform(-umax, umax, nrows), rng.uniform(-vmax, vmax, nrows),
                    rng.uniform(-wfrac * max(umax, vmax), wfrac * max(umax, vmax), nrows)], axis=1)
    return Observation(uvw, freq, npix_x, npix_y, psx, psy, 1.0, "random")


def point_source_image(npix_x, npix_y, frac=0.01, seed=0, dtype=np.float64) -> np.ndarray:
    """frac of the pixels hold point sources with log-normal(0, 1) flux; zero elsewhere."""
    rng = np.random.default_rng(seed + 1000)
    img = np.zeros((npix_x, npix_y), dtype=dtype)
    n = max(1, int(round(frac * npix_x * npix_y)))
    idx = rng.choice(npix_x * npix_y, size=n, replace=False)
    img.reshape(-1)[idx] = rng.lognormal(0.0, 1.0, n)
    return img


def gaussian_image(npix_x, npix_y, seed=0, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed + 2000).standard_normal((npix_x, npix_y)).astype(dtype)


def complex_normal(shape, seed=0, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed + 3000)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
