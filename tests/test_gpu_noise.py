"""GPU parity of the fast-resolve noise model and likelihood (Sec. 3.3.1 Eq. ham_new, Sec. 3.3.3)
against the FP64 oracle (oracle/noise.py), through the C ABI.

Tolerances: the kernel K inherits the NUFFT error of the exact N'(I_delta), one R and one
R^dagger at eps = 1e-5 (<= 2 eps), amplified by at most rho = sqrt(N) |N'(I_delta)| / |K|
(derived in the fit test; rho is about 1.0-1.1 here); N'^-1 and the likelihood with a given
kernel are FP32 FFT arithmetic (<= 2e-6 and 1e-5 relative)."""
import numpy as np
import pytest

import oracle
from oracle import noise
from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09144_gb300 import build, binding
    build.build()
    binding.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.float32)


def make(nrow=500, nchan=1, nx=32, ny=32, wc=0.0, per=False, seed=60):
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.random_observation(nrow, nchan, nx, ny, 3e-3, seed=seed, wmax_cycles=wc,
                                   per_channel_sky=per)
    plan = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5,
                wterm=obs.wterm, mfs=not per)
    return obs, plan


@pytest.mark.parametrize("wc,nchan,per,nx,ny", [(0.0, 1, False, 32, 32), (1.5, 2, True, 32, 64)])
def test_noise_kernel_fit_matches_oracle_argmin(wc, nchan, per, nx, ny):
    obs, plan = make(nchan=nchan, nx=nx, ny=ny, wc=wc, per=per)
    w = obs.weights.astype(np.float32).astype(np.float64)
    eps_noise = 1e-3 * float(w.sum()) / nchan
    logdet = plan.noise_fit(eps_noise)
    K = plan.noise_kernel().cpu().numpy()
    n_delta = noise.noise_cov_of_delta(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                                       eps_noise, weights=w, nsky=plan.nsky, wterm=obs.wterm)
    K_ref = noise.fit_noise_kernel(n_delta, eps_noise)
    # The loss of Sec. 3.3.3 separates per frequency: with D = FFT(I_delta), |D_k| = 1 and
    # z = FFT(N'(I_delta)) conj(D), its minimiser over K >= eps is K_k = max(Re z_k, eps),
    # 1-Lipschitz in z_k. By Parseval |K - K_ref| <= |z - z_ref| = sqrt(N) |N' - N'_ref| (I_delta),
    # so rel(K) <= rho rel(N'(I_delta)) with rho = sqrt(N) |N'_ref(I_delta)| / |K_ref|. The
    # library's N'(I_delta) is one R and one R^dagger N^-1 of the plan (<= 2 eps), measured here.
    delta = noise.centre_delta(plan.nsky, nx, ny)
    n_gpu = plan.grid(plan.degrid(dev(delta))).cpu().numpy() + eps_noise * delta
    rn = rel(n_gpu, n_delta)
    rho = np.sqrt(nx * ny) * np.linalg.norm(n_delta) / np.linalg.norm(K_ref)
    assert rn <= 2e-5, rn
    assert rel(K, K_ref) <= rho * rn * 1.01 + 1e-6, (rel(K, K_ref), rho, rn)
    assert rel(K, K_ref) <= 2e-5 * rho * 1.01 + 1e-6, (rel(K, K_ref), rho)
    assert np.all(K >= np.float32(eps_noise) * (1 - 1e-6))
    ref_logdet = 0.5 * np.log(2 * np.pi * K_ref).reshape(plan.nsky, -1).sum(1)
    assert np.allclose(logdet, ref_logdet, rtol=1e-5)


def test_noise_inverse_matches_oracle():
    obs, plan = make(nchan=2, per=True, nx=32, ny=64, wc=0.5)
    plan.noise_fit(10.0)
    K = plan.noise_kernel().cpu().numpy().astype(np.float64)
    x = np.random.default_rng(1).standard_normal((3, 2, 32, 64))
    got = plan.noise_apply_inverse(dev(x)).cpu().numpy()
    ref = np.stack([noise.noise_inverse(x[b], K) for b in range(3)])
    assert rel(got, ref) <= 2e-6, rel(got, ref)


def test_fast_likelihood_matches_oracle():
    obs, plan = make(nx=32, ny=32, wc=0.0)
    plan.noise_fit(5.0)
    K = plan.noise_kernel().cpu().numpy().astype(np.float64)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    psf = psf.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2)
    sky = rng.standard_normal((2, 1, 32, 32))
    dirty = rng.standard_normal((2, 1, 32, 32)) * 50.0
    val, grad = plan.fast_likelihood_grad(dev(sky), dev(dirty))
    for b in range(2):
        H, _, g = noise.fast_hamiltonian(psf, sky[b], dirty[b], K)
        assert abs(val[b] - H[0]) <= 1e-5 * abs(H[0]), (val[b], H[0])
        assert rel(grad[b].cpu().numpy(), g) <= 1e-5
    # end to end with the oracle's own PSF and kernel fit
    w = obs.weights.astype(np.float32).astype(np.float64)
    psf_o = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 32, 32, weights=w)
    K_o = noise.fit_noise_kernel(noise.noise_cov_of_delta(obs.uvw, obs.freqs, obs.pixsize,
                                                          obs.pixsize, 32, 32, 5.0, weights=w,
                                                          wterm=obs.wterm), 5.0)
    H_o, _, g_o = noise.fast_hamiltonian(psf_o, sky[0], dirty[0], K_o)
    assert abs(val[0] - H_o[0]) <= 1e-4 * abs(H_o[0])
    assert rel(grad[0].cpu().numpy(), g_o) <= 1e-4


def test_fast_likelihood_gradient_by_central_differences():
    obs, plan = make(nx=64, ny=32, wc=1.0, seed=61)
    plan.noise_fit(2.0)
    rng = np.random.default_rng(3)
    sky = rng.standard_normal((1, 64, 32))
    dirty = rng.standard_normal((1, 64, 32)) * 30.0
    _, g = plan.fast_likelihood_grad(dev(sky), dev(dirty))
    g = g.cpu().numpy().astype(np.float64)
    for k in range(2):
        d = rng.standard_normal((1, 64, 32))
        h = 1.0  # quadratic in the sky: exact up to FP32 rounding of the value
        vp = plan.fast_likelihood_grad(dev(sky + h * d), dev(dirty))[0][0]
        vm = plan.fast_likelihood_grad(dev(sky - h * d), dev(dirty))[0][0]
        assert abs((vp - vm) / (2 * h) - np.sum(g * d)) <= 1e-3 * np.linalg.norm(g) * np.linalg.norm(d)


def test_noise_model_errors():
    from paper_2406_09144_gb300.binding import FastResolveError, Plan
    obs, plan = make()
    x = dev(np.zeros((1, 32, 32)))
    with pytest.raises(FastResolveError):
        plan.fast_likelihood_grad(x, x)  # before the fit
    with pytest.raises(FastResolveError):
        plan.noise_fit(-1.0)
    o16 = synth.random_observation(100, 1, 16, 16, 3e-3, seed=62, wmax_cycles=0.0)
    p16 = Plan(o16.uvw, o16.freqs, 16, 16, o16.pixsize, weights=o16.weights, eps=1e-5)
    with pytest.raises(FastResolveError):
        p16.noise_fit(1.0)  # periodic 16-point transforms are below the FFT engine's range


def test_fast_likelihood_autograd():
    """torch.autograd through FastLikelihood: d/dsky is the kernel's gradient, d/ddirty is
    N'^-1 r (checked against the oracle's N'^-1 with the GPU kernel)."""
    from paper_2406_09144_gb300.autograd import fast_likelihood
    obs, plan = make(nx=32, ny=32, wc=0.5, seed=63)
    plan.noise_fit(3.0)
    K = plan.noise_kernel().cpu().numpy().astype(np.float64)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    psf = psf.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    sky = dev(rng.standard_normal((2, 1, 32, 32))).requires_grad_(True)
    dirty = dev(rng.standard_normal((2, 1, 32, 32)) * 20.0).requires_grad_(True)
    loss = (fast_likelihood(sky, dirty, plan) * torch.tensor([1.0, 2.0], dtype=torch.float64,
                                                              device="cuda")).sum()
    loss.backward()
    _, g = plan.fast_likelihood_grad(sky.detach(), dirty.detach())
    assert rel(sky.grad[0].cpu().numpy(), g[0].cpu().numpy()) <= 1e-6
    assert rel(sky.grad[1].cpu().numpy(), 2 * g[1].cpu().numpy()) <= 1e-6
    s64 = sky.detach().cpu().numpy().astype(np.float64)
    d64 = dirty.detach().cpu().numpy().astype(np.float64)
    for b, wgt in ((0, 1.0), (1, 2.0)):
        r = d64[b] - oracle.psf_apply(psf, s64[b])
        assert rel(dirty.grad[b].cpu().numpy(), wgt * noise.noise_inverse(r, K)) <= 1e-5


@pytest.mark.slow
def test_vla_full_size_noise_model():
    """VLA-like workload at full size: the fitted kernel is real, bounded below by eps and even
    (the PSF is), and the likelihood is a non-negative quadratic form whose gradient matches a
    central difference."""
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.observation("vla")
    plan = Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=obs.weights, eps=1e-5,
                wterm=obs.wterm, mfs=True)
    eps_noise = 1e-4 * float(obs.weights.astype(np.float64).sum())
    plan.noise_fit(eps_noise)
    K = plan.noise_kernel().cpu().numpy()[0].astype(np.float64)
    assert np.all(K >= np.float32(eps_noise) * (1 - 1e-6))
    flip = K[(-np.arange(1024)) % 1024][:, (-np.arange(1024)) % 1024]
    assert rel(K, flip) <= 1e-4
    rng = np.random.default_rng(4)
    sky = synth.sky_image(1024, 1024, seed=5)[None, None]
    dirty = plan.grid(torch.as_tensor(synth.complex_gaussian((obs.nrow, 1), seed=6)).to(
        "cuda", torch.complex64)).cpu().numpy()[None]
    val, g = plan.fast_likelihood_grad(dev(sky), dev(dirty))
    assert val[0] >= 0
    d = rng.standard_normal(sky.shape)
    h = 0.5
    vp = plan.fast_likelihood_grad(dev(sky + h * d), dev(dirty))[0][0]
    vm = plan.fast_likelihood_grad(dev(sky - h * d), dev(dirty))[0][0]
    gd = float(np.sum(g.cpu().numpy().astype(np.float64) * d))
    assert abs((vp - vm) / (2 * h) - gd) <= 1e-2 * abs(gd) + 1e-6 * abs(val[0])
