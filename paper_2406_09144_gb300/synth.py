"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds observation geometry and random draws only: antenna layouts,
Earth-rotation uvw tracks, channel frequencies, sky images, visibilities and
weights. It contains none of the measurement operator's arithmetic, so both the
FP64 oracle tests and the CUDA path take their inputs from here.

Shapes follow the VLA Cygnus A data (single channel, Tab. 1) and the MeerKAT
ESO 137-006 data (many rows, many channels, wide field, Tab. 2). The real data
sets are not available; these generators stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
C_LIGHT = 299_792_458.0  # m/s, used only to size pixels from a uv extent


# --------------------------------------------------------------------------
# arrays and tracks
# --------------------------------------------------------------------------

def vla_like_enu(seed: int = 1, n_per_arm: int = 9, arm_km: float = 21.0) -> np.ndarray:
    """Random-Y array: 3 arms 120 deg apart, radii U[0.05, 1] * arm_km, sorted. ENU metres [nant, 3]."""
    rng = np.random.default_rng(seed)
    pos = []
    for arm in range(3):
        az = math.radians(5.0 + 120.0 * arm)
        radii = np.sort(rng.uniform(0.05, 1.0, n_per_arm)) * arm_km * 1e3
        for r in radii:
            pos.append((r * math.sin(az), r * math.cos(az), rng.uniform(-5.0, 5.0)))
    return np.asarray(pos, dtype=np.float64)


def meerkat_like_enu(seed: int = 1, nant: int = 64, core_frac: float = 0.7,
                     core_km: float = 1.0, outer_km: float = 4.0) -> np.ndarray:
    """Dense core (70% of dishes within 1 km) plus outer dishes out to 4 km radius (baselines up
    to about 8 km, as for MeerKAT). ENU metres [nant, 3]."""
    rng = np.random.default_rng(seed)
    ncore = int(round(core_frac * nant))
    r_core = core_km * 1e3 * np.sqrt(rng.uniform(0.0, 1.0, ncore))
    r_out = rng.uniform(core_km, outer_km, nant - ncore) * 1e3
    r = np.concatenate([r_core, r_out])
    az = rng.uniform(0.0, 2.0 * math.pi, nant)
    up = rng.uniform(-10.0, 10.0, nant)
    return np.stack([r * np.sin(az), r * np.cos(az), up], axis=1)


def earth_rotation_uvw(enu: np.ndarray, lat_deg: float, dec_deg: float,
                       hours: float, step_s: float) -> np.ndarray:
    """uvw tracks (metres) of all baselines p<q over an hour-angle range centred on transit.

    Textbook Earth-rotation synthesis: ENU -> local equatorial XYZ at latitude lat,
    then the (H, dec) rotation to (u, v, w). Rows are time-major, baseline-minor,
    like a measurement set. Returns float64 [ntime * nbl, 3].
    """
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    xyz = np.stack([-math.sin(lat) * n + math.cos(lat) * u,
                    e,
                    math.cos(lat) * n + math.sin(lat) * u], axis=1)
    p, q = np.triu_indices(len(enu), k=1)
    b = xyz[q] - xyz[p]                                   # [nbl, 3]
    ntime = int(round(hours * 3600.0 / step_s))
    ha = (np.arange(ntime) - (ntime - 1) / 2.0) * step_s * (2.0 * math.pi / 86164.0905)
    sh, ch = np.sin(ha)[:, None], np.cos(ha)[:, None]
    bx, by, bz = b[None, :, 0], b[None, :, 1], b[None, :, 2]
    uu = sh * bx + ch * by
    vv = -math.sin(dec) * ch * bx + math.sin(dec) * sh * by + math.cos(dec) * bz
    ww = math.cos(dec) * ch * bx - math.cos(dec) * sh * by + math.sin(dec) * bz
    return np.stack([uu, vv, ww], axis=-1).reshape(-1, 3).astype(np.float64)


# --------------------------------------------------------------------------
# skies, visibilities, weights
# --------------------------------------------------------------------------

def sky_image(nx: int, ny: int, seed: int = 0, npoint: int = 20, nblob: int = 5,
              dtype=np.float64) -> np.ndarray:
    """Positive sky: point sources (log-uniform flux [1e-2, 1]) plus Gaussian blobs. [nx, ny]."""
    rng = np.random.default_rng(seed)
    img = np.zeros((nx, ny), dtype=np.float64)
    px = rng.integers(0, nx, npoint)
    py = rng.integers(0, ny, npoint)
    flux = 10.0 ** rng.uniform(-2.0, 0.0, npoint)
    np.add.at(img, (px, py), flux)
    gx = np.arange(nx)[:, None]
    gy = np.arange(ny)[None, :]
    for _ in range(nblob):
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        sig = rng.uniform(2.0, 8.0)
        amp = rng.uniform(1e-2, 1e-1)
        img += amp * np.exp(-((gx - cx) ** 2 + (gy - cy) ** 2) / (2.0 * sig * sig))
    return img.astype(dtype)


def random_skies(nsky: int, nx: int, ny: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Stack of independent seeded skies [nsky, nx, ny]."""
    return np.stack([sky_image(nx, ny, seed=seed + 7919 * i, dtype=dtype) for i in range(nsky)])


def complex_gaussian(shape, seed: int, sigma=1.0) -> np.ndarray:
    """Circular complex Gaussian with E|z|^2 = sigma^2 (Re, Im each sigma^2/2). complex128."""
    rng = np.random.default_rng(seed)
    s = np.asarray(sigma, dtype=np.float64) / math.sqrt(2.0)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * s


def baseline_sigmas(nrow: int, nbl: int, sigma: float, seed: int, spread: float = 0.2) -> np.ndarray:
    """Per-baseline noise level sigma * U[1-spread, 1+spread], repeated over time-major rows. [nrow]."""
    rng = np.random.default_rng(seed)
    sb = sigma * rng.uniform(1.0 - spread, 1.0 + spread, nbl)
    return np.resize(sb, nrow)


# --------------------------------------------------------------------------
# workload presets
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Observation:
    name: str
    uvw: np.ndarray          # [nrow, 3] metres
    freqs: np.ndarray        # [nchan] Hz
    weights: np.ndarray      # [nrow, nchan] float64 (1/sigma^2)
    sigma: np.ndarray        # [nrow, nchan] noise sigma
    nx: int
    ny: int
    pixsize: float           # radians, square pixels
    wterm: bool
    per_channel_sky: bool

    @property
    def nrow(self) -> int:
        return self.uvw.shape[0]

    @property
    def nchan(self) -> int:
        return self.freqs.shape[0]

    @property
    def nvis(self) -> int:
        return self.nrow * self.nchan

    @property
    def nsky(self) -> int:
        return self.nchan if self.per_channel_sky else 1


def _pixsize_from_uv(uvw: np.ndarray, fmax: float, factor: float = 2.2) -> float:
    umax = float(np.max(np.abs(uvw[:, :2]))) * fmax / C_LIGHT
    return 1.0 / (factor * umax)


def observation(name: str, seed_array: int = 1, seed_noise: int = 2, hours=None,
                step_s=None, npix=None) -> Observation:
    """Preset workloads.

    small   : 128^2, 1 ch at 1.4 GHz, VLA-like 27 antennas, 4 h at 10 s (505,440 rows), w = 0
    vla     : 1024^2 at 0.1", 1 ch 1.4 GHz, 27 antennas, 8 h at 2 s (5,054,400 rows), w-terms
    meerkat : 4096^2 at 2", 8 ch 909.5 + 107 i MHz, 64 antennas, 8 h at 8 s (7,257,600 rows)
    tiny    : 32^2, VLA-like, 20 min at 60 s, w-terms; for brute-force checks
    npix overrides the image side at the preset's pixel size (e.g. 3600 with the MeerKAT-like
    array: Tab. 2's 2 degree field of 3600^2 pixels of 2").
    """
    if name in ("small", "tiny"):
        enu = vla_like_enu(seed_array)
        h = 4.0 if name == "small" else 0.34
        st = 10.0 if name == "small" else 60.0
        uvw = earth_rotation_uvw(enu, 34.08, 40.7, hours or h, step_s or st)
        freqs = np.array([1.4e9])
        nx = ny = 128 if name == "small" else 32
        pix = _pixsize_from_uv(uvw, freqs.max())
        wterm = name == "tiny"
        if name == "small":
            uvw = uvw.copy()
            uvw[:, 2] = 0.0
        sig = np.full((uvw.shape[0], 1), 1e-2)
        per_chan = False
    elif name == "vla":
        enu = vla_like_enu(seed_array)
        uvw = earth_rotation_uvw(enu, 34.08, 40.7, hours or 8.0, step_s or 2.0)
        freqs = np.array([1.4e9])
        nx = ny = 1024
        pix = 0.1 * ARCSEC
        nbl = len(enu) * (len(enu) - 1) // 2
        sig = baseline_sigmas(uvw.shape[0], nbl, 1e-2, seed_noise)[:, None]
        wterm = True
        per_chan = False
    elif name in ("meerkat", "meerkat1"):
        enu = meerkat_like_enu(seed_array)
        uvw = earth_rotation_uvw(enu, -30.7, -60.5, hours or 8.0, step_s or 8.0)
        freqs = 909.5e6 + 107e6 * np.arange(8)
        if name == "meerkat1":  # the top channel alone (7,257,600 visibilities)
            freqs = freqs[-1:]
        nx = ny = 4096
        pix = 2.0 * ARCSEC
        nbl = len(enu) * (len(enu) - 1) // 2
        sb = baseline_sigmas(uvw.shape[0], nbl, 1e-2, seed_noise)
        sig = np.repeat(sb[:, None], len(freqs), axis=1)
        wterm = True
        per_chan = True
    else:
        raise ValueError(f"unknown observation preset {name!r}")
    sig = np.broadcast_to(sig, (uvw.shape[0], len(freqs))).astype(np.float64)
    if npix is not None:
        nx = ny = int(npix)
    return Observation(name=name, uvw=uvw, freqs=freqs, weights=1.0 / sig ** 2, sigma=sig,
                       nx=nx, ny=ny, pixsize=pix, wterm=wterm, per_channel_sky=per_chan)


def random_observation(nrow: int, nchan: int, nx: int, ny: int, pixsize: float, seed: int,
                       umax_frac: float = 0.35, wmax_cycles: float = 0.0, f0: float = 1.0e9,
                       per_channel_sky: bool = False, weights: bool = True) -> Observation:
    """Uniformly scattered uvw for small parity cases.

    |u|, |v| reach umax_frac / pixsize wavelengths at the top channel and w spans
    +-wmax_cycles / |n_min - 1| wavelengths, so the w phase spans about wmax_cycles
    turns at the field corner.
    """
    rng = np.random.default_rng(seed)
    freqs = f0 * (1.0 + 0.15 * np.arange(nchan))
    fmax = freqs.max()
    lmax = max(nx, ny) / 2 * pixsize
    t_corner = abs(math.sqrt(max(1.0 - 2 * lmax * lmax, 0.0)) - 1.0)
    uv = rng.uniform(-1.0, 1.0, (nrow, 2)) * umax_frac / pixsize * C_LIGHT / fmax
    wmax = wmax_cycles / max(t_corner, 1e-30) * C_LIGHT / fmax
    w = rng.uniform(-1.0, 1.0, nrow) * wmax
    uvw = np.concatenate([uv, w[:, None]], axis=1)
    wt = rng.uniform(0.5, 2.0, (nrow, nchan)) if weights else np.ones((nrow, nchan))
    return Observation(name="random", uvw=uvw, freqs=freqs, weights=wt, sigma=1.0 / np.sqrt(wt),
                       nx=nx, ny=ny, pixsize=pixsize, wterm=wmax_cycles > 0,
                       per_channel_sky=per_channel_sky)
