"""The allocation-free PSF convolution entry point, checked against fr_psf_apply and the oracle.

fr_psf_convolve_noalloc exists for callers that cannot allocate device memory (code embedded in
an application that owns the device-memory budget through its own pool, or running where a
cudaMalloc would synchronise the device or is not allowed). It keeps its intermediates in one
fixed device array inside the library, which every call shares. So this test calls it through
the C ABI several times in a row, with the image size changing between calls (a large image,
then a small one, then the large one again: no call may be disturbed by what an earlier call of
another layout left in the array), and compares every result with the plan-based fr_psf_apply
at the tolerance of the PSF-convolution parity tests, and with the FP64 oracle's direct linear
convolution of the same PSF image (the whole image at the small size, sampled pixels at the
large one).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6  # same bound as the PSF-convolution parity tests


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(nx, ny):
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.random_observation(4000, 1, nx, ny, 2e-3, seed=60)
    plan = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    return plan, psf


def _call(lib, psf, sky, nx, ny, batch):
    out = torch.full_like(sky, float("nan"))
    stream = torch.cuda.current_stream()
    rc = lib.fr_psf_convolve_noalloc(ctypes.c_void_p(psf.data_ptr()),
                                     ctypes.c_void_p(sky.data_ptr()), nx, ny, batch,
                                     ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.fr_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_convolution_across_changing_sizes():
    from paper_2406_09144_gb300 import build
    from paper_2406_09144_gb300.binding import load
    build.build()
    lib = load()
    cases = {(1024, 1024): _case(1024, 1024), (128, 64): _case(128, 64)}
    rng = np.random.default_rng(5)
    for call, (nx, ny, batch) in enumerate([(1024, 1024, 1), (128, 64, 3), (1024, 1024, 2),
                                            (128, 64, 1)]):
        plan, psf = cases[(nx, ny)]
        sky = torch.tensor(synth.random_skies(batch, nx, ny, seed=10 + call), dtype=torch.float32,
                           device="cuda")
        got = _call(lib, psf, sky, nx, ny, batch)
        assert np.all(np.isfinite(got))
        ref = plan.psf_apply(sky[:, None]).cpu().numpy()[:, 0]
        assert _rel(got, ref) <= TOL, (call, _rel(got, ref))
        P = psf.cpu().numpy()[0].astype(np.float64)
        s = sky.cpu().numpy().astype(np.float64)
        if nx * ny <= 128 * 64:
            refo = oracle.psf_apply(P[None], s)
            assert _rel(got, refo) <= TOL, (call, _rel(got, refo))
        else:
            for b in range(batch):
                pix = rng.integers(0, nx * ny, 64)
                refo = oracle.psf_apply_at(P, s[b], pix)
                assert _rel(got[b].reshape(-1)[pix], refo) <= TOL, (call, b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2406_09144_gb300.binding import load
    lib = load()
    dummy = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.fr_psf_convolve_noalloc(p, p, 2048, 1024, 1, p, None)
    assert rc == -1 and b"exceeds the fixed scratch" in lib.fr_last_error()
    # within 2^20 pixels, but the padded transform of 2 x 16384 points is longer than the FFT
    # passes take: refused up front with FR_EINVAL, nothing queued
    for nx, ny in ((16384, 64), (64, 16384)):
        rc = lib.fr_psf_convolve_noalloc(p, p, nx, ny, 1, p, None)
        assert rc == -1 and b"[16, 8192]" in lib.fr_last_error(), (nx, ny)
