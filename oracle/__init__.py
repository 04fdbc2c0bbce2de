"""Plain FP64 CPU oracle of the fast-resolve measurement operator.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import, call, link or execute anything under ``oracle/``.

Every function here evaluates a definition from the paper directly (direct sums,
no NUFFT, no blocking or fusion beyond chunking a vectorised sum), so a reader can
check it against the equations by eye. The measurement operator uses no FFT; the
noise model (``oracle.noise``) uses numpy's FFT because the paper defines its
periodic convolutions by FFTs, and solves the kernel fit as a numerical argmin. The oracle shares no code,
tables or constants with the CUDA path under ``paper_2406_09144_gb300/csrc``.

Sections and equations cited:
  Eq. (rime), Sec. 2       - measurement equation R
  Eq. (ham), Sec. 3.1.2    - likelihood Hamiltonian, N^-1 = visibility weights
  Eq. (clean), Sec. 3.2    - R^dagger N^-1 R I = R^dagger N^-1 V, dirty image, PSF
  Sec. 3.3.2               - PSF convolution on a 2x padded grid, and with reduced padding
                             (the PSF truncated to the window the padded grid holds)
  Algorithm 1              - major-cycle residual d = I^D - R^dagger N^-1 R I
  Eq. (ham_new), Sec. 3.3.1, Sec. 3.3.3 (oracle.noise) - noise kernel K = exp(xi) + eps,
                             its fit, N'^-1 and the fast-resolve Hamiltonian

Parity: every function is pinned by tests in tests/test_oracle_pins.py and
tests/test_oracle_noise_pins.py (closed forms, a special case equal to numpy.fft,
adjointness, the PSF identity, a library convolution, dense circulant algebra, a
kernel the fit must recover, and finite differences). No function is
parity-unpinned.
"""
from .measurement import (  # noqa: F401
    C_LIGHT,
    uvw_to_wavelengths,
    pixel_lm,
    direction_cosines,
    degrid,
    grid,
    psf,
    psf_apply,
    psf_apply_at,
    psf_window,
    truncate_psf,
    psf_apply_truncated,
    likelihood,
    likelihood_exact,
    residual_dirty,
    vis_residual_norm2,
)
from . import noise  # noqa: E402,F401
