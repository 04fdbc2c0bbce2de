"""Pins of the oracle's noise model and fast-resolve Hamiltonian (oracle/noise.py) against
closed forms, dense linear algebra and finite differences (Sec. 3.3.1 Eq. ham_new, Sec. 3.3.3)."""
import numpy as np

import oracle
from oracle import noise
from paper_2406_09144_gb300 import synth


def _even_positive(nx, ny, seed, floor):
    """A real, even (K(-k) = K(k)) transfer function bounded below by `floor`."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 2.0, (nx, ny))
    a = 0.5 * (a + a[(-np.arange(nx)) % nx][:, (-np.arange(ny)) % ny])
    return floor + a


def test_fit_recovers_a_positive_periodic_kernel():
    """If N' is itself a periodic convolution with transfer P > eps, the argmin is K = P."""
    nx, ny, eps = 8, 16, 1e-3
    P = _even_positive(nx, ny, 1, 0.1)
    n_delta = noise.periodic_convolve(noise.centre_delta(1, nx, ny), P[None])
    K = noise.fit_noise_kernel(n_delta, eps)
    assert np.allclose(K[0], P, rtol=1e-7, atol=1e-9)


def test_fit_stays_above_eps_where_the_target_transfer_is_smaller():
    """Where the target's transfer function is below eps (or negative), no K = exp(xi) + eps
    reaches it; the loss decreases towards K = eps there, and equals max(target, eps) elsewhere."""
    nx, ny, eps = 8, 8, 0.05
    P = _even_positive(nx, ny, 2, -0.5)  # some entries negative
    n_delta = noise.periodic_convolve(noise.centre_delta(1, nx, ny), P[None])
    K = noise.fit_noise_kernel(n_delta, eps)[0]
    assert np.all(K >= eps)
    above = P > eps + 1e-3
    assert np.allclose(K[above], P[above], rtol=1e-6)
    assert np.all(K[~above] < eps + 2e-3)


def test_noise_inverse_and_logdet_against_dense_circulant():
    """N'^-1 r by FFT equals the dense solve with the circulant matrix of the kernel, and
    1/2 sum ln(2 pi K) equals 1/2 ln det(2 pi N')."""
    nx, ny = 6, 4
    K = _even_positive(nx, ny, 3, 0.2)
    c = np.real(np.fft.ifft2(K))  # convolution kernel of N'
    n = nx * ny
    C = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            dx = (i // ny - j // ny) % nx
            dy = (i % ny - j % ny) % ny
            C[i, j] = c[dx, dy]
    r = np.random.default_rng(4).standard_normal((1, nx, ny))
    u = noise.noise_inverse(r, K[None])
    u_dense = np.linalg.solve(C, r.ravel()).reshape(1, nx, ny)
    assert np.allclose(u, u_dense, rtol=1e-10, atol=1e-12)
    sign, logdet = np.linalg.slogdet(2.0 * np.pi * C)
    assert sign > 0
    assert np.isclose(0.5 * np.sum(np.log(2.0 * np.pi * K)), 0.5 * logdet, rtol=1e-12)


def test_noise_inverse_undoes_the_covariance():
    nx, ny = 8, 8
    K = _even_positive(nx, ny, 5, 0.3)
    x = np.random.default_rng(6).standard_normal((2, nx, ny))
    assert np.allclose(noise.noise_inverse(noise.periodic_convolve(x, K[None]), K[None]), x,
                       rtol=1e-12, atol=1e-12)


def test_fit_of_a_coplanar_normal_operator_is_even_and_matches_the_psf_transfer():
    """At w = 0 and 1/n = 1 the exact N'(I_delta) is the PSF centred on the delta plus eps delta; its
    fitted kernel is real, even, and equals the periodic transfer of that image where it
    exceeds eps."""
    obs = synth.random_observation(300, 1, 16, 16, 5e-3, seed=7, wmax_cycles=0.0)
    eps = 1e-2
    w = obs.weights.astype(np.float64)
    n_delta = noise.noise_cov_of_delta(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 16, 16, eps,
                                       weights=w, wterm=False, nterm=False)
    # the exact normal operator of a centre delta is the (unnormalised) PSF centred there
    P = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 16, 16, weights=w)[0]
    centred = P[8:24, 8:24] + eps * noise.centre_delta(1, 16, 16)[0]
    assert np.allclose(n_delta[0], centred, rtol=1e-10, atol=1e-10 * P.max())
    K = noise.fit_noise_kernel(n_delta, eps)[0]
    flip = K[(-np.arange(16)) % 16][:, (-np.arange(16)) % 16]
    assert np.allclose(K, flip, rtol=1e-6, atol=1e-8 * K.max())
    z = np.real(np.fft.fft2(n_delta[0]) * np.conj(np.fft.fft2(noise.centre_delta(1, 16, 16)[0])))
    above = z > eps * 1.5
    # the numerical argmin stops once the loss (dominated by the largest K) stalls: 1e-7 of max
    assert np.allclose(K[above], z[above], rtol=0, atol=1e-7 * z.max())
    assert np.all(K[~above] < eps * 1.5 + 1e-7 * z.max())


def test_fast_hamiltonian_gradient_by_central_differences():
    nx = ny = 8
    rng = np.random.default_rng(8)
    obs = synth.random_observation(200, 1, nx, ny, 8e-3, seed=9, wmax_cycles=0.0)
    w = obs.weights.astype(np.float64)
    psf = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny, weights=w)
    K = _even_positive(nx, ny, 10, 0.5)[None]
    sky = rng.standard_normal((1, nx, ny))
    dirty = rng.standard_normal((1, nx, ny))
    H, logdet, g = noise.fast_hamiltonian(psf, sky, dirty, K)
    for k in range(3):
        d = rng.standard_normal((1, nx, ny))
        h = 0.5  # H is quadratic in the sky: the central difference is exact up to rounding
        Hp = noise.fast_hamiltonian(psf, sky + h * d, dirty, K)[0]
        Hm = noise.fast_hamiltonian(psf, sky - h * d, dirty, K)[0]
        assert np.isclose((Hp - Hm)[0] / (2 * h), np.sum(g * d), rtol=1e-9)
    # the value is the quadratic form of the residual
    r = dirty - oracle.psf_apply(psf, sky)
    assert np.isclose(H[0], 0.5 * np.sum(r * noise.noise_inverse(r, K)), rtol=1e-12)
    assert np.isclose(logdet[0], 0.5 * np.sum(np.log(2 * np.pi * K)))
