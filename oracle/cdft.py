"""ctypes front end of oracle/dft.c: sampled FP64 direct sums for large problems.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). ``build()`` compiles dft.c with gcc and
OpenMP into oracle/_dft.so; ``load()`` builds on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .measurement import uvw_to_wavelengths

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dft.c")
_LIB = os.path.join(_HERE, "_dft.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C direct sums (plain gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        D = ctypes.c_double
        C = ctypes.c_int
        lib.or_degrid.argtypes = [P, I, I, I, D, D, P, P, P, I, P, P, I, C, C, P]
        lib.or_grid.argtypes = [P, P, I, I, I, I, I, D, D, P, P, P, P, P, I, C, C, P]
        lib.or_psf.argtypes = [P, I, I, I, D, D, P, P, P, P, P, I, P]
        for f in (lib.or_degrid, lib.or_grid, lib.or_psf):
            f.restype = None
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def degrid_at(sky, uvw, freqs, dl, dm, rows, chans, wterm=True, nterm=True):
    """R (Eq. rime) at the visibilities (rows[i], chans[i]); complex128 [n]."""
    lib = load()
    sky = _f64(sky)
    if sky.ndim == 2:
        sky = sky[None]
    u, v, w = (_f64(a) for a in uvw_to_wavelengths(uvw, freqs))
    rows, chans = _i64(rows), _i64(chans)
    out = np.zeros(2 * len(rows))
    lib.or_degrid(_p(sky), sky.shape[0], sky.shape[1], sky.shape[2], dl, dm, _p(u), _p(v), _p(w),
                  u.shape[1], _p(rows), _p(chans), len(rows), int(wterm), int(nterm), _p(out))
    return out[0::2] + 1j * out[1::2]


def grid_at(vis, uvw, freqs, dl, dm, nx, ny, imgs, pix, weights=None, nsky=1, wterm=True,
            nterm=True):
    """R^dagger N^-1 (Eq. clean) at pixels pix[i] = jx * ny + jy of image imgs[i]; float64 [n]."""
    lib = load()
    y = np.asarray(vis, dtype=np.complex128)
    if weights is not None:
        y = y * np.asarray(weights, dtype=np.float64)
    yre, yim = _f64(y.real), _f64(y.imag)
    u, v, w = (_f64(a) for a in uvw_to_wavelengths(uvw, freqs))
    imgs, pix = _i64(imgs), _i64(pix)
    out = np.zeros(len(pix))
    lib.or_grid(_p(yre), _p(yim), u.shape[0], u.shape[1], nsky, nx, ny, dl, dm, _p(u), _p(v), _p(w),
                _p(imgs), _p(pix), len(pix), int(wterm), int(nterm), _p(out))
    return out


def psf_at(uvw, freqs, dl, dm, imgs, a, b, weights=None, nsky=1):
    """PSF (Sec. 3.3.2, unnormalised, w = 0) at pixel offsets (a[i], b[i]) of image imgs[i]."""
    lib = load()
    u, v, _ = (_f64(x) for x in uvw_to_wavelengths(uvw, freqs))
    wt = _f64(np.ones(u.shape) if weights is None else weights)
    imgs, a, b = _i64(imgs), _i64(a), _i64(b)
    out = np.zeros(len(a))
    lib.or_psf(_p(wt), u.shape[0], u.shape[1], nsky, dl, dm, _p(u), _p(v), _p(imgs), _p(a), _p(b),
               len(a), _p(out))
    return out


def psf_full(uvw, freqs, dl, dm, nx, ny, weights=None, nsky=1):
    """Whole [nsky, 2nx, 2ny] PSF from the C sums, laid out as oracle.measurement.psf."""
    A, B = np.meshgrid(np.arange(-nx, nx), np.arange(-ny, ny), indexing="ij")
    out = np.zeros((nsky, 2 * nx, 2 * ny))
    for s in range(nsky):
        vals = psf_at(uvw, freqs, dl, dm, np.full(A.size, s), A.ravel(), B.ravel(), weights, nsky)
        out[s] = vals.reshape(2 * nx, 2 * ny)
    out[:, 0, :] = 0.0
    out[:, :, 0] = 0.0
    return out
