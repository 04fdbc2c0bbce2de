"""The allocation-free PSF convolution entry point, checked against fr_psf_apply.

fr_psf_convolve_noalloc exists for callers that cannot allocate device memory (code embedded in
an application that owns the device-memory budget through its own pool, or running where a
cudaMalloc would synchronise the device or is not allowed). It keeps its intermediates in one
fixed device array inside the library, so this test calls it through the C ABI twice in a row
(the second call must not be disturbed by what the first left in that array) and compares both
results with the plan-based fr_psf_apply, at the tolerance the PSF-convolution parity tests use.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6  # same bound as the PSF-convolution parity tests


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny,batch", [(128, 64, 3), (1024, 1024, 1)])
def test_noalloc_convolution_matches_plan_path_on_two_calls(nx, ny, batch):
    from paper_2406_09144_gb300 import build
    from paper_2406_09144_gb300.binding import Plan, load
    build.build()
    lib = load()
    obs = synth.random_observation(4000, 1, nx, ny, 2e-3, seed=60)
    plan = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    stream = torch.cuda.current_stream()
    for call in range(2):
        sky = torch.tensor(synth.random_skies(batch, nx, ny, seed=10 + call), dtype=torch.float32,
                           device="cuda")
        ref = plan.psf_apply(sky[:, None]).cpu().numpy()[:, 0]
        out = torch.full_like(sky, float("nan"))
        rc = lib.fr_psf_convolve_noalloc(ctypes.c_void_p(psf.data_ptr()),
                                         ctypes.c_void_p(sky.data_ptr()), nx, ny, batch,
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.fr_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= TOL, (call, _rel(got, ref))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2406_09144_gb300.binding import load
    lib = load()
    dummy = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.fr_psf_convolve_noalloc(p, p, 2048, 1024, 1, p, None)
    assert rc == -1 and b"exceeds the fixed scratch" in lib.fr_last_error()
