"""FR_DETERMINISTIC: bitwise reproducible outputs through the C ABI.

The gridders accumulate in 64-bit fixed point (order-independent integer atomics) and the
expansion terms are added to the image one after the other, so R^dag N^-1, the PSF build, the
major-cycle residual and the likelihood gradients come out the same bit for bit on every call
and in every plan built from the same inputs. The results stay within the NUFFT tolerance of the
FP64 oracle (eps = 1e-5) and within 1e-6 of the default (float-atomic) path.
"""
import numpy as np
import pytest

import oracle
from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2406_09144_gb300 import build, binding
    build.build()
    binding.load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def plans(obs, mfs):
    from paper_2406_09144_gb300.binding import Plan
    kw = dict(weights=obs.weights, eps=EPS, wterm=obs.wterm, mfs=mfs)
    return (Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, deterministic=True, **kw),
            Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, deterministic=True, **kw),
            Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, **kw))


# w = 0; w-stacking; the small-w expansion (term grids); per-channel skies
CASES = [(0.0, 1, False, 64, 64), (3.0, 2, False, 64, 32), (0.02, 1, False, 96, 64),
         (1.0, 2, True, 48, 80)]


@pytest.mark.parametrize("wc,nchan,per,nx,ny", CASES)
def test_gridding_is_bitwise_reproducible(wc, nchan, per, nx, ny):
    obs = synth.random_observation(2500, nchan, nx, ny, 2e-3, seed=110, wmax_cycles=wc,
                                   per_channel_sky=per)
    d1, d2, nd = plans(obs, mfs=not per)
    vis = dev(synth.complex_gaussian(d1.vis_shape, seed=111), torch.complex64)
    a = d1.grid(vis).cpu().numpy()
    sky = dev(synth.random_skies(d1.nsky, nx, ny, seed=112))
    d1.degrid(sky)  # the degridder shares the workspace
    b = d1.grid(vis).cpu().numpy()
    c = d2.grid(vis).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(a, c)
    ref = oracle.grid(vis.cpu().numpy().astype(np.complex128), obs.uvw, obs.freqs, obs.pixsize,
                      obs.pixsize, nx, ny, weights=obs.weights.astype(np.float32),
                      nsky=d1.nsky, wterm=obs.wterm)
    assert rel(a, ref) <= EPS, rel(a, ref)
    assert rel(a, nd.grid(vis).cpu().numpy()) <= 1e-6
    # the PSF build grids too: two deterministic plans give the same PSF and transfer function
    p1 = d1.dirty_psf(want_dirty=False)[1].cpu().numpy()
    p2 = d2.dirty_psf(want_dirty=False)[1].cpu().numpy()
    assert np.array_equal(p1, p2)
    assert np.array_equal(d1.psf_apply(sky).cpu().numpy(), d2.psf_apply(sky).cpu().numpy())
    # the major cycle and the exact likelihood gradient (R^dag N^-1 R inside)
    dirty = d1.grid(vis)
    r1 = d1.major_cycle(sky, dirty)[0].cpu().numpy()
    r2 = d1.major_cycle(sky, dirty)[0].cpu().numpy()
    assert np.array_equal(r1, r2)
    g1 = d1.likelihood_grad(sky, dirty, exact=True)[1].cpu().numpy()
    g2 = d2.likelihood_grad(sky, dirty, exact=True)[1].cpu().numpy()
    assert np.array_equal(g1, g2)


def test_fast_likelihood_is_bitwise_reproducible():
    obs = synth.random_observation(1500, 1, 64, 64, 2e-3, seed=113, wmax_cycles=0.5)
    d1, d2, _ = plans(obs, mfs=True)
    l1 = d1.noise_fit(3.0)
    l2 = d2.noise_fit(3.0)
    assert np.array_equal(d1.noise_kernel().cpu().numpy(), d2.noise_kernel().cpu().numpy())
    assert abs(l1[0] - l2[0]) <= 1e-12 * abs(l1[0])  # FP64 scalar sums: last bits may differ
    sky = dev(synth.random_skies(2, 64, 64, seed=114)[:, None])
    d = dev(np.random.default_rng(115).standard_normal((2, 1, 64, 64)) * 20.0)
    ga = d1.fast_likelihood_grad(sky, d)[1].cpu().numpy()
    gb = d2.fast_likelihood_grad(sky, d)[1].cpu().numpy()
    assert np.array_equal(ga, gb)
