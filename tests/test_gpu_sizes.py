"""GPU parity at image sides that are not powers of two (any even side in [16, 4096]), through
the C ABI, against the FP64 oracle.

The oversampled grid is the shortest FFT length of at least twice the side (2^k, 3 2^k or
5 2^k: sigma = 2 for sides of those forms, a little above 2 otherwise), the PSF keeps its
[2nx][2ny] layout on a grid of at least 4nx x 4ny, and the padded PSF transforms default to the
shortest length holding every offset of the cropped product (>= 2n - 1). Tolerances as in
test_gpu_parity: eps = 1e-5 for the NUFFT outputs, 2e-6 for the PSF convolution.
"""
import numpy as np
import pytest

import oracle
from oracle import cdft, noise
from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09144_gb300 import build, binding
    build.build()
    binding.load()
    cdft.build()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def make_plan(obs, eps=EPS, mfs=False):
    from paper_2406_09144_gb300.binding import Plan
    return Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=obs.weights, eps=eps,
                wterm=obs.wterm, mfs=mfs)


# nx, ny, wmax_cycles, nchan, per-channel, expected grid (Nu, Nv)
CASES = [
    (48, 80, 0.0, 1, False, (96, 160)),     # 3 2^4 x 5 2^4: sigma = 2, radix-3/5 grids
    (96, 40, 3.0, 2, True, (192, 80)),      # w-stacking on mixed-radix grids
    (100, 60, 0.02, 1, False, (256, 128)),  # sides of no FFT form: sigma 2.56 x 2.13, expansion
    (34, 66, 1.5, 2, False, (80, 160)),     # sigma 2.35 x 2.42, MFS
]


@pytest.mark.parametrize("case", CASES)
def test_r_and_rdag_match_oracle_at_other_sizes(case):
    nx, ny, wc, nchan, per, grid = case
    obs = synth.random_observation(1200, nchan, nx, ny, 2e-3, seed=90, wmax_cycles=wc,
                                   per_channel_sky=per)
    plan = make_plan(obs, mfs=not per)
    info = plan.info()
    assert (info["grid_nu"], info["grid_nv"]) == grid
    sky = synth.random_skies(obs.nsky, nx, ny, seed=91)
    ref = oracle.degrid(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, wterm=obs.wterm)
    got = plan.degrid(dev(sky)).cpu().numpy()
    assert rel(got, ref) <= EPS, rel(got, ref)
    vis = synth.complex_gaussian(plan.vis_shape, seed=92)
    refd = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                       weights=obs.weights.astype(np.float32), nsky=obs.nsky, wterm=obs.wterm)
    gotd = plan.grid(dev(vis, torch.complex64)).cpu().numpy()
    assert rel(gotd, refd) <= EPS, rel(gotd, refd)
    # the PSF ([2nx][2ny], unnormalised) and its norm
    _, psf, norm = plan.dirty_psf(want_dirty=False)
    refp = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                      weights=obs.weights.astype(np.float32), nsky=obs.nsky)
    assert rel(psf.cpu().numpy(), refp) <= EPS
    assert np.allclose(norm, refp[:, nx, ny], rtol=1e-6)


@pytest.mark.parametrize("nx,ny,lxy", [(48, 80, (96, 160)), (100, 60, (256, 128)),
                                       (34, 66, (80, 160))])
def test_psf_convolution_and_likelihood_at_other_sizes(nx, ny, lxy):
    obs = synth.random_observation(1000, 1, nx, ny, 2e-3, seed=93)
    plan = make_plan(obs, mfs=True)
    assert plan.psf_padding == lxy  # shortest supported lengths >= 2n - 1
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    P = psf.cpu().numpy().astype(np.float64)
    sky = synth.random_skies(3, nx, ny, seed=94)[:, None]
    got = plan.psf_apply(dev(sky)).cpu().numpy()
    assert rel(got[:, 0], oracle.psf_apply(P, sky[:, 0])) <= 2e-6
    d = np.random.default_rng(95).standard_normal(sky.shape) * 30.0
    val, grad = plan.likelihood_grad(dev(sky), dev(d))
    rv, rg = oracle.likelihood(P, sky[:, 0], d[:, 0])
    assert np.allclose(val, rv, rtol=1e-5, atol=1e-5 * np.abs(rv).max())
    assert rel(grad.cpu().numpy()[:, 0], rg) <= 1e-5
    # reduced padding on the same plan: the truncated convolution of the oracle
    lx = [L for L in (64, 80, 96, 128, 160, 192) if nx < L < lxy[0]][0]
    plan.set_psf_padding(lx, lxy[1])
    got = plan.psf_apply(dev(sky)).cpu().numpy()
    assert rel(got[:, 0], oracle.psf_apply_truncated(P, sky[:, 0], lx, lxy[1])) <= 2e-6


def test_noise_model_at_mixed_radix_size():
    """The noise passes transform the unpadded image: 48 x 80 (3 2^4 x 5 2^4) against the
    oracle's argmin fit and N'^-1; a side of no FFT form is refused."""
    from paper_2406_09144_gb300.binding import FastResolveError
    nx, ny = 48, 80
    obs = synth.random_observation(600, 1, nx, ny, 3e-3, seed=96)
    plan = make_plan(obs, mfs=True)
    w = obs.weights.astype(np.float32).astype(np.float64)
    eps_noise = 1e-3 * float(w.sum())
    plan.noise_fit(eps_noise)
    K = plan.noise_kernel().cpu().numpy()
    n_delta = noise.noise_cov_of_delta(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                                       eps_noise, weights=w, wterm=obs.wterm)
    K_ref = noise.fit_noise_kernel(n_delta, eps_noise)
    assert rel(K, K_ref) <= 5e-5, rel(K, K_ref)
    x = np.random.default_rng(97).standard_normal((2, 1, nx, ny))
    got = plan.noise_apply_inverse(dev(x)).cpu().numpy()
    ref = np.stack([noise.noise_inverse(x[b], K.astype(np.float64)) for b in range(2)])
    assert rel(got, ref) <= 2e-6
    o2 = synth.random_observation(300, 1, 100, 60, 3e-3, seed=98)
    p2 = make_plan(o2, mfs=True)
    with pytest.raises(FastResolveError):
        p2.noise_fit(1.0)


def test_noise_model_at_sides_with_several_odd_factors():
    """Noise passes at 144 = 9 x 16 (two radix-3 stages, 144-thread CTAs: a partial warp in the
    reductions) against the oracle's argmin fit; N'^-1 and the fast-resolve likelihood at
    144 x 240 (240 = 15 x 16) against the oracle with the GPU's kernel."""
    nx, ny = 144, 32
    obs = synth.random_observation(500, 1, nx, ny, 3e-3, seed=99)
    plan = make_plan(obs, mfs=True)
    w = obs.weights.astype(np.float32).astype(np.float64)
    eps_noise = 1e-3 * float(w.sum())
    logdet = plan.noise_fit(eps_noise)
    K = plan.noise_kernel().cpu().numpy()
    n_delta = noise.noise_cov_of_delta(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                                       eps_noise, weights=w, wterm=obs.wterm)
    K_ref = noise.fit_noise_kernel(n_delta, eps_noise)
    assert rel(K, K_ref) <= 5e-5, rel(K, K_ref)
    assert np.allclose(logdet, 0.5 * np.log(2 * np.pi * K_ref).sum(), rtol=1e-5)
    nx, ny = 144, 240
    obs = synth.random_observation(800, 1, nx, ny, 2e-3, seed=100)
    plan = make_plan(obs, mfs=True)
    plan.noise_fit(5.0)
    K = plan.noise_kernel().cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(101)
    x = rng.standard_normal((2, 1, nx, ny))
    got = plan.noise_apply_inverse(dev(x)).cpu().numpy()
    ref = np.stack([noise.noise_inverse(x[b], K) for b in range(2)])
    assert rel(got, ref) <= 2e-6, rel(got, ref)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    P = psf.cpu().numpy().astype(np.float64)
    sky = synth.random_skies(2, nx, ny, seed=102)[:, None]
    d = rng.standard_normal(sky.shape) * 40.0
    val, grad = plan.fast_likelihood_grad(dev(sky), dev(d))
    for b in range(2):
        H, _, g = noise.fast_hamiltonian(P, sky[b], d[b], K)
        assert abs(val[b] - H[0]) <= 1e-5 * abs(H[0]), (val[b], H[0])
        assert rel(grad[b].cpu().numpy(), g) <= 1e-5


@pytest.mark.slow
def test_tab2_field_3600_full_size_sampled():
    """Tab. 2's field: 3600^2 pixels of 2" (8192^2 grid, sigma 2.28) with the MeerKAT-like top
    channel (7,257,600 visibilities, w-stacking): 10^4 sampled visibilities of R and 10^3
    sampled pixels of R^dag against the FP64 direct sums, and sampled pixels of the PSF
    convolution (8192-point padded transforms)."""
    obs = synth.observation("meerkat1", npix=3600)
    plan = make_plan(obs, mfs=not obs.per_channel_sky)
    info = plan.info()
    assert (info["grid_nu"], info["grid_nv"]) == (8192, 8192)
    rng = np.random.default_rng(5)
    n = 3600
    sky = synth.sky_image(n, n, seed=6)[None]
    vis = plan.degrid(dev(sky)).cpu().numpy()
    rows = rng.integers(0, obs.nrow, 10_000)
    ref = cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows,
                         np.zeros(10_000, int))
    assert rel(vis[rows, 0], ref) <= EPS, rel(vis[rows, 0], ref)
    y = synth.complex_gaussian((obs.nrow, 1), seed=7)
    d = plan.grid(dev(y, torch.complex64)).cpu().numpy()
    pix = rng.integers(0, n * n, 1_000)
    w32 = obs.weights.astype(np.float32)
    refd = cdft.grid_at(y, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, n, n,
                        np.zeros(1_000, int), pix, weights=w32)
    assert rel(d.reshape(-1)[pix], refd) <= EPS, rel(d.reshape(-1)[pix], refd)
    # PSF convolution: per-pixel sums of the GPU PSF image
    assert plan.psf_padding == (8192, 8192)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    P = psf.cpu().numpy()[0].astype(np.float64)
    s = sky[0].astype(np.float64)
    out = plan.psf_apply(dev(sky[None])).cpu().numpy()[0, 0]
    pts = [(0, 0), (n - 1, n - 1), (17, n - 3)] + [tuple(q) for q in rng.integers(0, n, (20, 2))]
    refc = np.array([np.sum(P[px + 1:px + n + 1, py + 1:py + n + 1][::-1, ::-1] * s)
                     for px, py in pts])
    assert rel(np.array([out[q] for q in pts]), refc) <= 2e-6
    # the noise model at 3600 (225 x 16: radix 5, 5, 3, 3, 16; 225-thread CTAs): the fitted
    # kernel is real, bounded below by eps and even (the PSF is), N'^-1 matches the oracle's
    # FFT definition with that kernel, and the likelihood's gradient a central difference
    eps_noise = 1e-4 * float(w32.astype(np.float64).sum())
    plan.noise_fit(eps_noise)
    K = plan.noise_kernel().cpu().numpy()[0].astype(np.float64)
    assert np.all(K >= np.float32(eps_noise) * (1 - 1e-6))
    flip = K[(-np.arange(n)) % n][:, (-np.arange(n)) % n]
    assert rel(K, flip) <= 1e-4
    x = rng.standard_normal((1, 1, n, n))
    got = plan.noise_apply_inverse(dev(x)).cpu().numpy()[0]
    assert rel(got, noise.noise_inverse(x[0], K[None])) <= 2e-6
    dd = d[None, None] if d.ndim == 2 else d[None]
    val, g = plan.fast_likelihood_grad(dev(sky[None]), dev(dd))
    dirn = rng.standard_normal(sky[None].shape)
    h = 0.5
    vp = plan.fast_likelihood_grad(dev(sky[None] + h * dirn), dev(dd))[0][0]
    vm = plan.fast_likelihood_grad(dev(sky[None] - h * dirn), dev(dd))[0][0]
    gd = float(np.sum(g.cpu().numpy().astype(np.float64) * dirn))
    assert abs((vp - vm) / (2 * h) - gd) <= 1e-2 * abs(gd) + 1e-6 * abs(val[0])
