"""CPU-only checks of the native library: it loads, exports every declared symbol, and its FFT
stage arithmetic (run on the host with the same code the kernels use) matches numpy.fft."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2406_09144_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_09144_gb300 import build
    build.build()
    return binding.load()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "fr_plan_create" in names and "fr_psf_apply" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) <= names


def test_error_strings(lib):
    assert lib.fr_strerror(0) == b"success"
    assert lib.fr_strerror(-1) == b"invalid argument"


def test_plan_create_rejects_bad_sizes_without_gpu(lib):
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    uvw = np.zeros((4, 3))
    f = np.array([1e9])
    # unknown flag bits
    r = lib.fr_plan_create(uvw.ctypes.data, 4, f.ctypes.data, 1, None, 64, 64, 1e-5, 1e-5, 1e-5,
                           64, None, ctypes.byref(h))
    assert r == -1 and not h.value
    # odd or out-of-range sides (any even side in [16, 4096] is accepted)
    for nx, ny in [(101, 64), (64, 33), (8192, 64), (64, 14)]:
        r = lib.fr_plan_create(uvw.ctypes.data, 4, f.ctypes.data, 1, None, nx, ny, 1e-5, 1e-5,
                               1e-5, 0, None, ctypes.byref(h))
        assert r == -4 and not h.value, (nx, ny)
    r = lib.fr_plan_create(uvw.ctypes.data, 4, f.ctypes.data, 1, None, 64, 64, 1e-5, 1e-5, 1e-9,
                           0, None, ctypes.byref(h))
    assert r == -4
    bad = uvw.copy()
    bad[1, 0] = np.nan
    r = lib.fr_plan_create(bad.ctypes.data, 4, f.ctypes.data, 1, None, 64, 64, 1e-5, 1e-5, 1e-5,
                           0, None, ctypes.byref(h))
    assert r == -1 and b"not finite" in lib.fr_last_error()
    # empty input: no rows, no channels, or an image below the 16-pixel minimum
    r = lib.fr_plan_create(uvw.ctypes.data, 0, f.ctypes.data, 1, None, 64, 64, 1e-5, 1e-5, 1e-5,
                           0, None, ctypes.byref(h))
    assert r == -1 and not h.value
    r = lib.fr_plan_create(uvw.ctypes.data, 4, f.ctypes.data, 0, None, 64, 64, 1e-5, 1e-5, 1e-5,
                           0, None, ctypes.byref(h))
    assert r == -1
    r = lib.fr_plan_create(uvw.ctypes.data, 4, f.ctypes.data, 1, None, 8, 64, 1e-5, 1e-5, 1e-5,
                           0, None, ctypes.byref(h))
    assert r == -4


# powers of two, the 3 2^k and 5 2^k lengths of the reduced-padding PSF transforms, and odd
# parts with several factors (radix-3 and radix-5 stages in sequence)
FFT_LENGTHS = [1 << lg for lg in range(1, 15)] + [3, 5, 6, 10, 48, 80, 96, 1536, 1280, 12288,
                                                  10240, 45, 225, 7200, 144, 240, 400, 720,
                                                  1200, 3600]


@pytest.mark.parametrize("n", FFT_LENGTHS)
@pytest.mark.parametrize("direction", [-1, 1, -2, 2])
def test_host_fft_stages_match_numpy(lib, n, direction):
    """Both stage schedules (16 points per thread, and +-2: 32 with a radix-32 opening stage)."""
    rng = np.random.default_rng(n)
    x = (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).astype(np.complex64)
    got = binding.selftest_fft_host(x, direction)
    ref = np.fft.fft(x.astype(np.complex128), axis=1) if direction < 0 else \
        np.fft.ifft(x.astype(np.complex128), axis=1) * n
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-6 * max(1, np.log2(n) / 4), err


def test_host_fft_rejects_other_lengths(lib):
    for n in (7, 14, 21 * 16, 1, 32768):
        with pytest.raises(binding.FastResolveError):
            binding.selftest_fft_host(np.zeros((1, max(n, 1)), np.complex64), -1)


def test_grid_length_rule():
    """The Python mirror of the library's transform-length rule (the oversampled grid of a side n
    is the shortest length >= 2n of the form 2^k, 3 2^k or 5 2^k; tests/test_gpu_sizes.py checks
    plans against it on the GPU)."""
    f = binding.fft_len_at_least
    assert [f(2 * n) for n in (16, 48, 80, 100, 34, 60, 1024, 3600, 4096)] == \
        [32, 96, 160, 256, 80, 128, 2048, 8192, 8192]
    for m in range(17, 16385, 37):
        L = f(m)
        assert L >= m
        c = L
        while c % 2 == 0:
            c //= 2
        assert c in (1, 3, 5)

