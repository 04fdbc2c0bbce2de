"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library FFT or
convolution on a special case that reduces to it, a different geometric route to the same
phase, adjointness, the PSF identity R^dagger N^-1 R = PSF * at w = 0 (Sec. 3.2, 3.3.2),
closed forms, invariants, and finite differences. A dropped term, a flipped sign, a shifted
pixel origin or a transposed axis in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.signal

import oracle
from oracle import cdft
from paper_2406_09144_gb300 import synth

C = oracle.C_LIGHT


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _grid_uvw(nx, ny, dl, dm, freq):
    """uvw (metres) whose u, v land exactly on the integer DFT frequencies a / (nx dl), b / (ny dm)."""
    A, B = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    u = A.ravel() / (nx * dl)
    v = B.ravel() / (ny * dm)
    lam = C / freq
    return np.stack([u * lam, v * lam, np.zeros_like(u)], axis=1), A.ravel(), B.ravel()


# ---------------------------------------------------------------- R: special cases and geometry

def test_degrid_on_integer_uv_grid_equals_numpy_fft2():
    """At w = 0, 1/n = 1 and u = a/(nx dl), v = b/(ny dm), Eq. (rime) is a 2D DFT of the image:
    V(a, b) = sum_j I_j exp(-2 pi i (a (jx - nx/2)/nx + b (jy - ny/2)/ny)) = (-1)^(a+b) fft2(I)[a, b].
    Pins the sign of the exponent, the pixel origin, x <-> u and the nu / c scaling."""
    nx, ny, dl, dm, f = 16, 12, 3e-3, 2e-3, 1.7e9
    sky = np.random.default_rng(0).standard_normal((nx, ny))
    uvw, A, B = _grid_uvw(nx, ny, dl, dm, f)
    vis = oracle.degrid(sky[None], uvw, [f], dl, dm, wterm=False, nterm=False)[:, 0]
    ref = np.fft.fft2(sky)[A, B] * (-1.0) ** (A + B)
    assert _rel(vis, ref) < 1e-12


def test_grid_on_integer_uv_grid_equals_numpy_ifft2():
    """The adjoint on the same special case is Re of an unnormalised inverse DFT."""
    nx, ny, dl, dm, f = 8, 16, 4e-3, 1e-3, 0.9e9
    rng = np.random.default_rng(1)
    uvw, A, B = _grid_uvw(nx, ny, dl, dm, f)
    y = rng.standard_normal(len(A)) + 1j * rng.standard_normal(len(A))
    d = oracle.grid(y[:, None], uvw, [f], dl, dm, nx, ny, wterm=False, nterm=False)[0]
    Y = np.zeros((nx, ny), complex)
    Y[A, B] = y * (-1.0) ** (A + B)
    ref = (np.fft.ifft2(Y) * nx * ny).real
    assert _rel(d, ref) < 1e-12


def test_degrid_equals_baseline_dot_direction_geometry():
    """Eq. (rime) from geometry: the phase of a source in direction s = (l, m, n) on baseline b
    (wavelengths) relative to the phase centre s0 = (0, 0, 1) is b . (s - s0); the amplitude
    carries 1/n. Pins the w sign relative to u, v, the (n - 1) and the 1/n factor (wide field)."""
    nx, ny, dl, dm = 8, 8, 0.04, 0.05
    rng = np.random.default_rng(2)
    sky = rng.uniform(0.0, 1.0, (nx, ny))
    uvw = rng.uniform(-40.0, 40.0, (50, 3))
    f = 3e8 * 1.3
    vis = oracle.degrid(sky[None], uvw, [f], dl, dm)[:, 0]
    b = uvw * f / C
    ref = np.zeros(len(b), complex)
    for jx in range(nx):
        for jy in range(ny):
            s = np.array([(jx - nx // 2) * dl, (jy - ny // 2) * dm, 0.0])
            s[2] = math.sqrt(1.0 - s[0] ** 2 - s[1] ** 2)
            ref += sky[jx, jy] / s[2] * np.exp(-2j * np.pi * (b @ (s - np.array([0.0, 0.0, 1.0]))))
    assert _rel(vis, ref) < 1e-12


def test_point_source_at_phase_centre_gives_flux():
    nx, ny = 10, 6
    sky = np.zeros((1, nx, ny))
    sky[0, nx // 2, ny // 2] = 2.5
    uvw = np.random.default_rng(3).uniform(-1e3, 1e3, (40, 3))
    vis = oracle.degrid(sky, uvw, [1e9, 2e9], 1e-3, 1e-3)
    assert np.allclose(vis, 2.5, atol=1e-13)


def test_hermitian_symmetry_of_real_sky():
    rng = np.random.default_rng(4)
    sky = rng.uniform(0, 1, (1, 12, 12))
    uvw = rng.uniform(-500, 500, (30, 3))
    a = oracle.degrid(sky, uvw, [1.2e9], 2e-3, 2e-3)
    b = oracle.degrid(sky, -uvw, [1.2e9], 2e-3, 2e-3)
    assert _rel(b, np.conj(a)) < 1e-12


def test_frequency_scaling_is_uvw_times_nu_over_c():
    rng = np.random.default_rng(5)
    sky = rng.uniform(0, 1, (1, 8, 8))
    uvw = rng.uniform(-500, 500, (20, 3))
    a = oracle.degrid(sky, uvw, [1.0e9], 3e-3, 3e-3)
    b = oracle.degrid(sky, 2.0 * uvw, [0.5e9], 3e-3, 3e-3)
    assert _rel(a, b) < 1e-12


# ---------------------------------------------------------------- adjointness

@pytest.mark.parametrize("nchan,per_channel", [(1, False), (3, False), (3, True)])
def test_adjointness(nchan, per_channel):
    """<R x, N^-1 y> = <x, R^dagger N^-1 y> under the real inner product (Eq. clean)."""
    obs = synth.random_observation(60, nchan, 10, 14, 2e-2, seed=6, wmax_cycles=3.0,
                                   per_channel_sky=per_channel)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((obs.nsky, obs.nx, obs.ny))
    y = rng.standard_normal((obs.nrow, nchan)) + 1j * rng.standard_normal((obs.nrow, nchan))
    rx = oracle.degrid(x, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    rty = oracle.grid(y, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.nx, obs.ny,
                      weights=obs.weights, nsky=obs.nsky)
    lhs = float(np.sum((np.conj(rx) * (obs.weights * y)).real))
    rhs = float(np.sum(x * rty))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


# ---------------------------------------------------------------- PSF

def _tiny_w0_obs(nrow=80, nx=12, ny=10, nchan=1, seed=8):
    obs = synth.random_observation(nrow, nchan, nx, ny, 1.5e-2, seed=seed, wmax_cycles=0.0)
    return obs


def test_psf_peak_is_weight_sum_and_psf_is_even():
    obs = _tiny_w0_obs(nchan=2)
    P = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.nx, obs.ny, obs.weights)[0]
    assert abs(P[obs.nx, obs.ny] - obs.weights.sum()) < 1e-10 * obs.weights.sum()
    # even about (nx, ny): P[nx + a, ny + b] == P[nx - a, ny - b] for the stored offsets
    inner = P[1:, 1:]
    assert np.allclose(inner, inner[::-1, ::-1], atol=1e-10)
    assert np.all(P[0, :] == 0.0) and np.all(P[:, 0] == 0.0)


def test_normal_operator_of_a_delta_is_the_shifted_psf():
    """At w = 0 with 1/n = 1, R^dagger N^-1 R delta_j0 = PSF centred on j0 (Eq. clean, Sec. 3.2)."""
    obs = _tiny_w0_obs()
    nx, ny, dl = obs.nx, obs.ny, obs.pixsize
    P = oracle.psf(obs.uvw, obs.freqs, dl, dl, nx, ny, obs.weights)[0]
    for j0 in [(nx // 2, ny // 2), (0, 0), (nx - 1, 3)]:
        d = np.zeros((1, nx, ny))
        d[0][j0] = 1.0
        vis = oracle.degrid(d, obs.uvw, obs.freqs, dl, dl, wterm=False, nterm=False)
        rr = oracle.grid(vis, obs.uvw, obs.freqs, dl, dl, nx, ny, weights=obs.weights,
                         wterm=False, nterm=False)[0]
        ref = P[nx - j0[0]:2 * nx - j0[0], ny - j0[1]:2 * ny - j0[1]]
        assert np.allclose(rr, ref, atol=1e-10 * obs.weights.sum())


def test_psf_convolution_equals_normal_operator_at_w0():
    """PSF * s == R^dagger N^-1 R s for every sky when w = 0 and 1/n = 1 (Sec. 3.3.2, coplanar)."""
    obs = _tiny_w0_obs(nchan=2, seed=9)
    nx, ny, dl = obs.nx, obs.ny, obs.pixsize
    s = np.random.default_rng(10).uniform(0, 1, (1, nx, ny))
    P = oracle.psf(obs.uvw, obs.freqs, dl, dl, nx, ny, obs.weights)
    conv = oracle.psf_apply(P, s)
    vis = oracle.degrid(s, obs.uvw, obs.freqs, dl, dl, wterm=False, nterm=False)
    rr = oracle.grid(vis, obs.uvw, obs.freqs, dl, dl, nx, ny, weights=obs.weights,
                     wterm=False, nterm=False)
    assert _rel(conv, rr) < 1e-12


def test_psf_apply_equals_scipy_linear_convolution():
    """The cropped linear convolution of Sec. 3.3.2 is the centre block of the full 2D convolution."""
    rng = np.random.default_rng(11)
    nx, ny = 9, 14
    P = rng.standard_normal((2 * nx, 2 * ny))
    s = rng.standard_normal((nx, ny))
    full = scipy.signal.convolve2d(s, P, mode="full")
    ref = full[nx:2 * nx, ny:2 * ny]
    assert _rel(oracle.psf_apply(P[None], s[None])[0], ref) < 1e-12


def test_sampled_psf_convolution_equals_scipy_linear_convolution():
    """psf_apply_at (single output pixels, for large images) against the same library
    convolution, at every pixel of a small rectangular image including its corners."""
    rng = np.random.default_rng(12)
    nx, ny = 7, 12
    P = rng.standard_normal((2 * nx, 2 * ny))
    s = rng.standard_normal((nx, ny))
    ref = scipy.signal.convolve2d(s, P, mode="full")[nx:2 * nx, ny:2 * ny]
    got = oracle.psf_apply_at(P, s, np.arange(nx * ny)).reshape(nx, ny)
    assert _rel(got, ref) < 1e-12


# ---------------------------------------------------- reduced padding (truncated PSF, Sec. 3.3.2)

def test_truncated_psf_with_full_padding_is_the_exact_convolution():
    """lx = 2nx, ly = 2ny keep every offset the cropped product reaches: no truncation."""
    rng = np.random.default_rng(30)
    nx, ny = 10, 12
    P = rng.standard_normal((2, 2 * nx, 2 * ny))
    s = rng.standard_normal((2, nx, ny))
    assert oracle.psf_window(nx, ny, 2 * nx, 2 * ny) == (nx - 1, ny - 1)
    assert _rel(oracle.psf_apply_truncated(P, s, 2 * nx, 2 * ny), oracle.psf_apply(P, s)) < 1e-14


def test_truncated_psf_delta_response_closed_form():
    """A unit sky pixel at q returns PSF(p - q) inside the window |p - q| <= (hx, hy) (edges
    included) and exactly zero outside it."""
    rng = np.random.default_rng(31)
    nx, ny, lx, ly = 12, 16, 15, 22
    hx, hy = oracle.psf_window(nx, ny, lx, ly)
    assert (hx, hy) == (3, 6)
    P = rng.uniform(1.0, 2.0, (1, 2 * nx, 2 * ny))  # no zero inside: every kept offset shows
    for q in [(0, 0), (nx - 1, ny - 1), (5, 7)]:
        s = np.zeros((1, nx, ny))
        s[0][q] = 1.0
        out = oracle.psf_apply_truncated(P, s, lx, ly)[0]
        for px in range(nx):
            for py in range(ny):
                a, b = px - q[0], py - q[1]
                want = P[0, nx + a, ny + b] if abs(a) <= hx and abs(b) <= hy else 0.0
                assert out[px, py] == want, (q, px, py)


def _periodic_kernel(P, nx, ny, lx, ly, hx, hy):
    K = np.zeros((lx, ly))
    for a in range(-hx, hx + 1):
        for b in range(-hy, hy + 1):
            K[a % lx, b % ly] += P[nx + a, ny + b]
    return K


@pytest.mark.parametrize("lx,ly", [(15, 22), (20, 24), (13, 17), (16, 30)])
def test_truncated_psf_equals_padded_fft_convolution(lx, ly):
    """The padded FFT convolution of Sec. 3.3.2, P^dag FFT^-1[FFT[K] . FFT[P s]] on an lx x ly
    grid with the periodic kernel K of the window, equals the truncated linear convolution
    (numpy.fft); one offset more than the window and the period wraps it onto the crop."""
    rng = np.random.default_rng(32)
    nx, ny = 12, 16
    P = rng.standard_normal((2 * nx, 2 * ny))
    s = rng.standard_normal((nx, ny))
    hx, hy = oracle.psf_window(nx, ny, lx, ly)
    pad = np.zeros((lx, ly))
    pad[:nx, :ny] = s

    def fftconv(hx_, hy_):
        K = _periodic_kernel(P, nx, ny, lx, ly, hx_, hy_)
        return np.real(np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(pad)))[:nx, :ny]

    ref = oracle.psf_apply_truncated(P[None], s[None], lx, ly)[0]
    assert _rel(fftconv(hx, hy), ref) < 1e-12
    if hx + 1 <= nx - 1:  # a wider window aliases: the window rule is the largest exact one
        wide = oracle.psf_apply(oracle.truncate_psf(P[None], hx + 1, hy), s[None])[0]
        assert _rel(fftconv(hx + 1, hy), wide) > 1e-3


def test_truncation_error_bounded_by_dropped_sidelobes():
    """|PSF_t * s - PSF * s| <= (sum of |PSF| outside the window) max|s| at every pixel (Young)."""
    obs = _tiny_w0_obs(nchan=1, seed=33)
    nx, ny, dl = obs.nx, obs.ny, obs.pixsize
    P = oracle.psf(obs.uvw, obs.freqs, dl, dl, nx, ny, obs.weights)
    s = np.random.default_rng(34).uniform(0, 1, (1, nx, ny))
    full = oracle.psf_apply(P, s)
    for lx, ly in [(nx + 2, ny + 3), (nx + nx // 2, 2 * ny), (2 * nx, ny + 4)]:
        hx, hy = oracle.psf_window(nx, ny, lx, ly)
        dropped = np.abs(P - oracle.truncate_psf(P, hx, hy)).sum()
        err = np.abs(oracle.psf_apply_truncated(P, s, lx, ly) - full).max()
        assert err <= dropped * s.max() * (1 + 1e-12)
        assert err > 0


def test_psf_per_channel_sums_to_mfs_psf():
    obs = _tiny_w0_obs(nchan=3, seed=12)
    a = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.nx, obs.ny, obs.weights, nsky=3)
    b = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.nx, obs.ny, obs.weights, nsky=1)
    assert _rel(a.sum(0), b[0]) < 1e-12


def test_wide_field_psf_deviation_bounded_by_n_term():
    """With the n-term on, R^dagger N^-1 R departs from PSF * by at most the 1 - n_min scale."""
    obs = synth.random_observation(60, 1, 10, 10, 2e-2, seed=13, wmax_cycles=0.0)
    nx, ny, dl = obs.nx, obs.ny, obs.pixsize
    s = np.random.default_rng(14).uniform(0, 1, (1, nx, ny))
    P = oracle.psf(obs.uvw, obs.freqs, dl, dl, nx, ny, obs.weights)
    conv = oracle.psf_apply(P, s)
    vis = oracle.degrid(s, obs.uvw, obs.freqs, dl, dl, wterm=False, nterm=True)
    rr = oracle.grid(vis, obs.uvw, obs.freqs, dl, dl, nx, ny, weights=obs.weights,
                     wterm=False, nterm=True)
    _, _, n = oracle.direction_cosines(nx, ny, dl, dl)
    dev = _rel(rr, conv)
    bound = 2.5 * (1.0 / np.nanmin(n) ** 2 - 1.0)
    assert 0.0 < dev <= bound


# ---------------------------------------------------------------- likelihood

def test_likelihood_gradient_central_differences():
    """L is quadratic, so a central difference along any direction equals <grad, e> up to rounding."""
    obs = _tiny_w0_obs(nx=8, ny=8, seed=15)
    rng = np.random.default_rng(16)
    P = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 8, 8, obs.weights)
    s = rng.uniform(0, 1, (2, 8, 8))
    d = rng.standard_normal((2, 8, 8)) * 10.0
    _, g = oracle.likelihood(P, s, d)
    for _ in range(3):
        e = rng.standard_normal((2, 8, 8))
        h = 1e-3
        lp, _ = oracle.likelihood(P, s + h * e, d)
        lm, _ = oracle.likelihood(P, s - h * e, d)
        fd = (lp - lm) / (2 * h)
        an = np.einsum("bij,bij->b", g, e)
        assert np.allclose(fd, an, rtol=1e-8, atol=1e-8 * np.abs(an).max())


def test_likelihood_equals_hamiltonian_minus_constant():
    """With d = R^dagger N^-1 V and PSF * = R^dagger N^-1 R (w = 0), the image-space likelihood
    equals Eq. (ham) minus the constant 1/2 V^dagger N^-1 V."""
    obs = _tiny_w0_obs(seed=17)
    nx, ny, dl = obs.nx, obs.ny, obs.pixsize
    rng = np.random.default_rng(18)
    V = rng.standard_normal((obs.nrow, 1)) + 1j * rng.standard_normal((obs.nrow, 1))
    d = oracle.grid(V, obs.uvw, obs.freqs, dl, dl, nx, ny, weights=obs.weights, wterm=False,
                    nterm=False)
    s = rng.uniform(0, 1, (1, nx, ny))
    P = oracle.psf(obs.uvw, obs.freqs, dl, dl, nx, ny, obs.weights)
    val, _ = oracle.likelihood(P, s, d)
    rs = oracle.degrid(s, obs.uvw, obs.freqs, dl, dl, wterm=False, nterm=False)
    ham = 0.5 * np.sum(obs.weights * np.abs(V - rs) ** 2)
    const = 0.5 * np.sum(obs.weights * np.abs(V) ** 2)
    assert abs(val[0] - (ham - const)) < 1e-10 * const
    val_exact, g_exact = oracle.likelihood_exact(s, d, obs.uvw, obs.freqs, dl, dl, obs.weights,
                                                 wterm=False, nterm=False)
    assert abs(val_exact - val[0]) < 1e-10 * const
    assert 2 * (ham - const) + 2 * const == pytest.approx(
        oracle.vis_residual_norm2(V, s, obs.uvw, obs.freqs, dl, dl, obs.weights, wterm=False,
                                  nterm=False), rel=1e-12)


def test_major_cycle_residual_vanishes_for_noiseless_data():
    """Algorithm 1: d = I^D - R^dagger N^-1 R I is zero when V = R I exactly."""
    obs = synth.random_observation(50, 2, 8, 8, 2e-2, seed=19, wmax_cycles=2.0)
    s = np.random.default_rng(20).uniform(0, 1, (1, 8, 8))
    V = oracle.degrid(s, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    dirty = oracle.grid(V, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 8, 8, weights=obs.weights)
    res = oracle.residual_dirty(dirty, s, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.weights)
    assert np.max(np.abs(res)) < 1e-10 * np.max(np.abs(dirty))
    assert oracle.vis_residual_norm2(V, s, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize,
                                     obs.weights) < 1e-20


# ---------------------------------------------------------------- C helper vs numpy definitions

def test_c_direct_sums_match_numpy_definitions():
    obs = synth.random_observation(70, 2, 10, 12, 2e-2, seed=21, wmax_cycles=4.0,
                                   per_channel_sky=True)
    dl = obs.pixsize
    rng = np.random.default_rng(22)
    sky = rng.uniform(0, 1, (2, 10, 12))
    vis = oracle.degrid(sky, obs.uvw, obs.freqs, dl, dl)
    rows = rng.integers(0, obs.nrow, 25)
    chans = rng.integers(0, 2, 25)
    got = cdft.degrid_at(sky, obs.uvw, obs.freqs, dl, dl, rows, chans)
    assert _rel(got, vis[rows, chans]) < 1e-12
    y = rng.standard_normal((obs.nrow, 2)) + 1j * rng.standard_normal((obs.nrow, 2))
    for nsky in (1, 2):
        dirty = oracle.grid(y, obs.uvw, obs.freqs, dl, dl, 10, 12, weights=obs.weights, nsky=nsky)
        imgs = rng.integers(0, nsky, 30)
        pix = rng.integers(0, 120, 30)
        got = cdft.grid_at(y, obs.uvw, obs.freqs, dl, dl, 10, 12, imgs, pix, obs.weights, nsky)
        assert _rel(got, dirty.reshape(nsky, -1)[imgs, pix]) < 1e-12
        P = oracle.psf(obs.uvw, obs.freqs, dl, dl, 10, 12, obs.weights, nsky=nsky)
        Pc = cdft.psf_full(obs.uvw, obs.freqs, dl, dl, 10, 12, obs.weights, nsky=nsky)
        assert _rel(Pc, P) < 1e-12
