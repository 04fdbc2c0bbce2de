"""Autograd wrappers: backward passes against the FP64 oracle and central finite differences.

Tolerances: gradients against the oracle <= 1e-5 relative L2 (NUFFT accuracy eps). Central
differences of the linear (R, R^dagger) and quadratic (likelihood) losses are exact up to rounding
for any step, so the step is chosen where FP32 rounding of the loss values stays below the
1e-3 relative tolerance: 1.0 for the linear maps, 0.5 for the small likelihoods; at full size
(16 x 2048^2) the step is 1e-3 along the gradient direction (no cancellation in <grad, e>) and
0.1 along a random direction (1e-2, the FP32 rounding of sums over 4M pixels).
"""
import numpy as np
import pytest

import oracle
from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09144_gb300 import build, binding
    build.build()
    binding.load()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def small_plan(seed=70, nchan=2, per=True):
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.random_observation(900, nchan, 32, 32, 2e-3, seed=seed, wmax_cycles=2.0,
                                   per_channel_sky=per)
    w32 = obs.weights.astype(np.float32)
    return obs, w32, Plan(obs.uvw, obs.freqs, 32, 32, obs.pixsize, weights=w32, eps=1e-5,
                          mfs=not per)


def test_degrid_backward_is_R_dagger():
    from paper_2406_09144_gb300.autograd import degrid
    obs, _, plan = small_plan()
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal(plan.sky_shape)
    a = synth.complex_gaussian(plan.vis_shape, seed=2)
    at = torch.tensor(a, dtype=torch.complex64, device="cuda")
    x = torch.tensor(x0, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = (torch.conj(at) * degrid(x, plan)).real.sum()
    loss.backward()
    ref = oracle.grid(a, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 32, 32, nsky=obs.nsky)
    assert rel(x.grad.cpu().numpy(), ref) <= 1e-5
    # central difference along a random direction (the loss is linear)
    e = torch.tensor(rng.standard_normal(plan.sky_shape), dtype=torch.float32, device="cuda")
    h = 1.0
    with torch.no_grad():
        lp = (torch.conj(at) * plan.degrid(x + h * e)).real.double().sum()
        lm = (torch.conj(at) * plan.degrid(x - h * e)).real.double().sum()
    fd = float((lp - lm) / (2 * h))
    an = float((x.grad.double() * e.double()).sum())
    assert abs(fd - an) <= 1e-3 * abs(an)


def test_grid_backward_is_weighted_R():
    from paper_2406_09144_gb300.autograd import grid
    obs, w32, plan = small_plan(seed=71)
    rng = np.random.default_rng(3)
    y0 = synth.complex_gaussian(plan.vis_shape, seed=4)
    g = rng.standard_normal(plan.sky_shape)
    gt = torch.tensor(g, dtype=torch.float32, device="cuda")
    y = torch.tensor(y0, dtype=torch.complex64, device="cuda", requires_grad=True)
    loss = (gt * grid(y, plan)).sum()
    loss.backward()
    ref = w32 * oracle.degrid(g, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    assert rel(y.grad.cpu().numpy(), ref) <= 1e-5
    e = torch.tensor(synth.complex_gaussian(plan.vis_shape, seed=5), dtype=torch.complex64,
                     device="cuda")
    h = 1.0
    with torch.no_grad():
        lp = (gt.double() * plan.grid(y + h * e).double()).sum()
        lm = (gt.double() * plan.grid(y - h * e).double()).sum()
    fd = float((lp - lm) / (2 * h))
    an = float((y.grad.real.double() * e.real.double() + y.grad.imag.double() * e.imag.double()).sum())
    assert abs(fd - an) <= 1e-3 * abs(an)


@pytest.mark.parametrize("exact", [False, True])
def test_likelihood_backward(exact):
    from paper_2406_09144_gb300.autograd import psf_likelihood, exact_likelihood
    obs, w32, plan = small_plan(seed=72, nchan=1, per=False)
    rng = np.random.default_rng(6)
    s0 = synth.random_skies(3, 32, 32, seed=7)[:, None]
    d0 = rng.standard_normal(s0.shape) * 30.0
    s = torch.tensor(s0, dtype=torch.float32, device="cuda", requires_grad=True)
    d = torch.tensor(d0, dtype=torch.float32, device="cuda", requires_grad=True)
    f = exact_likelihood if exact else psf_likelihood
    val = f(s, d, plan)
    coef = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (val * coef).sum().backward()
    if exact:
        rv, rg = zip(*[oracle.likelihood_exact(s0[b], d0[b], obs.uvw, obs.freqs, obs.pixsize,
                                               obs.pixsize, weights=w32) for b in range(3)])
        rv, rg = np.array(rv), np.stack(rg)
    else:
        _, psf, _ = plan.dirty_psf(want_dirty=False)
        rv, rg = oracle.likelihood(psf.cpu().numpy().astype(np.float64), s0[:, 0], d0[:, 0])
        rg = rg[:, None]
    c = coef.cpu().numpy()
    assert np.allclose(val.detach().cpu().numpy(), rv, rtol=1e-5, atol=1e-5 * np.abs(rv).max())
    assert rel(s.grad.cpu().numpy(), rg * c[:, None, None, None]) <= 1e-5
    assert rel(d.grad.cpu().numpy(), -s0 * c[:, None, None, None]) <= 1e-6
    e = torch.tensor(rng.standard_normal(s0.shape), dtype=torch.float32, device="cuda")
    h = 0.5
    with torch.no_grad():
        lp = (f(s + h * e, d, plan) * coef).sum()
        lm = (f(s - h * e, d, plan) * coef).sum()
    fd = float((lp - lm) / (2 * h))
    an = float((s.grad.double() * e.double()).sum())
    assert abs(fd - an) <= 1e-3 * abs(an)


def test_batch16_2048_psf_likelihood_fd_and_sampled_oracle():
    """Differentiation at full size: 16 skies at 2048^2 through the PSF likelihood."""
    from paper_2406_09144_gb300.autograd import psf_likelihood
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.observation("vla")
    plan = Plan(obs.uvw, obs.freqs, 2048, 2048, obs.pixsize / 2, weights=obs.weights, eps=1e-5)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    gen = torch.Generator(device="cuda").manual_seed(0)
    s = torch.rand((16, 1, 2048, 2048), generator=gen, device="cuda").requires_grad_(True)
    d = torch.randn((16, 1, 2048, 2048), generator=gen, device="cuda") * 100.0
    val = psf_likelihood(s, d, plan)
    val.sum().backward()
    g0 = s.grad.detach()
    nrm = lambda t: t.double().pow(2).sum(dim=(1, 2, 3), keepdim=True).sqrt()
    for e, h, tol in ((g0 * (nrm(s.detach()) / nrm(g0)).float(), 1e-3, 1e-3),
                      (torch.randn(s.shape, generator=gen, device="cuda"), 0.1, 1e-2)):
        with torch.no_grad():
            fd = (psf_likelihood(s + h * e, d, plan) - psf_likelihood(s - h * e, d, plan)) / (2 * h)
            an = (g0.double() * e.double()).sum(dim=(1, 2, 3))
        assert torch.allclose(fd, an, rtol=tol, atol=tol * float(an.abs().max())), (fd, an)
    # FP64 oracle gradient PSF * s - d at sampled pixels of two batch elements
    P = psf.cpu().numpy()[0].astype(np.float64)
    rng = np.random.default_rng(8)
    g = s.grad.detach()
    for b in (0, 11):
        sb = s.detach()[b, 0].cpu().numpy().astype(np.float64)
        db = d[b, 0].cpu().numpy().astype(np.float64)
        gb = g[b, 0].cpu().numpy()
        for _ in range(6):
            px, py = rng.integers(0, 2048, 2)
            win = P[2048 + px - 2047:2048 + px + 1, 2048 + py - 2047:2048 + py + 1][::-1, ::-1]
            ref = float(np.sum(win * sb)) - db[px, py]
            scale = float(np.sum(np.abs(win * sb))) + abs(db[px, py])
            assert abs(gb[px, py] - ref) <= 2e-5 * scale, (gb[px, py], ref, scale)
