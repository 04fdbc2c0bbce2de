"""GPU parity of the reduced-padding PSF convolution (Sec. 3.3.2) against the FP64 oracle,
through the C ABI.

fr_psf_set_padding(lx, ly) runs the PSF passes on an lx x ly padded grid (radix-3 and radix-5
transform lengths 3 2^k, 5 2^k next to the powers of two), which evaluates the linear
convolution with the PSF truncated to the window psf_window(nx, ny, lx, ly). The oracle is
oracle.psf_apply_truncated of the GPU's own PSF image (the PSF itself is pinned by
test_gpu_parity). Tolerances as for the full-padding convolution: FP32 FFTs only, <= 2e-6
relative L2; likelihood values <= 1e-5 relative.
"""
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


def make(nx, ny, nchan=2, per=True, nrow=1500, seed=80):
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.random_observation(nrow, nchan, nx, ny, 2e-3, seed=seed, wmax_cycles=0.0,
                                   per_channel_sky=per)
    plan = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5,
                wterm=obs.wterm, mfs=not per)
    return obs, plan


def psf_of(plan):
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    return psf.cpu().numpy().astype(np.float64)


def test_padded_lengths_helper():
    from paper_2406_09144_gb300.binding import padded_lengths
    assert padded_lengths(64) == [80, 96, 128]
    assert padded_lengths(1024) == [1280, 1536, 2048]
    assert padded_lengths(4096) == [5120, 6144, 8192]


# lx over padded_lengths(64), ly over padded_lengths(128): every radix mix on both axes
@pytest.mark.parametrize("lx,ly", [(80, 160), (96, 192), (128, 160), (96, 256), (80, 192),
                                   (128, 256)])
def test_reduced_padding_matches_oracle(lx, ly):
    nx, ny = 64, 128
    obs, plan = make(nx, ny)
    P = psf_of(plan)
    sky = synth.random_skies(4, nx, ny, seed=81).reshape(2, 2, nx, ny)
    sky[1, 1] = np.random.default_rng(82).standard_normal((nx, ny))  # signed, dense
    plan.set_psf_padding(lx, ly)
    assert plan.psf_padding == (lx, ly)
    got = plan.psf_apply(dev(sky)).cpu().numpy()
    for b in range(2):
        for c in range(2):  # image b * nsky + c uses the PSF of channel c
            ref = oracle.psf_apply_truncated(P[c:c + 1], sky[b, c:c + 1], lx, ly)[0]
            assert rel(got[b, c], ref) <= 2e-6, (b, c, rel(got[b, c], ref))


def test_restoring_full_padding_is_bitwise_the_default():
    nx, ny = 64, 64
    obs, plan = make(nx, ny, nchan=1, per=False)
    sky = dev(synth.random_skies(3, nx, ny, seed=83)[:, None])
    before = plan.psf_apply(sky).cpu().numpy()
    assert plan.psf_padding == (2 * nx, 2 * ny)
    plan.set_psf_padding(96, 80)
    reduced = plan.psf_apply(sky).cpu().numpy()
    assert rel(reduced, before) > 1e-6  # the truncation changes the result
    plan.set_psf_padding(2 * nx, 2 * ny)
    after = plan.psf_apply(sky).cpu().numpy()
    assert np.array_equal(before, after)


def test_reduced_padding_likelihoods_match_oracle():
    """Eq. ham with PSF_t (fr_likelihood_grad) and Eq. ham_new with PSF_t and the fitted noise
    kernel (fr_fast_likelihood_grad) against the oracle with the truncated PSF."""
    nx, ny, lx, ly = 64, 64, 96, 80
    obs, plan = make(nx, ny, nchan=1, per=False)
    P = psf_of(plan)
    plan.set_psf_padding(lx, ly)
    hx, hy = oracle.psf_window(nx, ny, lx, ly)
    Pt = oracle.truncate_psf(P, hx, hy)
    rng = np.random.default_rng(84)
    sky = synth.random_skies(3, nx, ny, seed=85)[:, None]
    d = rng.standard_normal(sky.shape) * 30.0
    val, grad = plan.likelihood_grad(dev(sky), dev(d))
    rv, rg = oracle.likelihood(Pt, sky[:, 0], d[:, 0])
    assert np.allclose(val, rv, rtol=1e-5, atol=1e-5 * np.abs(rv).max())
    assert rel(grad.cpu().numpy()[:, 0], rg) <= 1e-5
    plan.noise_fit(4.0)
    K = plan.noise_kernel().cpu().numpy().astype(np.float64)
    fv, fg = plan.fast_likelihood_grad(dev(sky), dev(d))
    for b in range(3):
        H, _, g = noise.fast_hamiltonian(Pt, sky[b], d[b], K)
        assert abs(fv[b] - H[0]) <= 1e-5 * abs(H[0]), (fv[b], H[0])
        assert rel(fg[b].cpu().numpy(), g) <= 1e-5


def test_padding_errors():
    from paper_2406_09144_gb300.binding import FastResolveError, Plan
    nx, ny = 64, 64
    obs, plan = make(nx, ny, nchan=1, per=False)
    for lx, ly, code in [(64, 128, -1), (130, 128, -1), (97, 128, -1), (112, 128, -4),
                         (128, 72, -4), (80, 60, -1)]:
        with pytest.raises(FastResolveError) as e:
            plan.set_psf_padding(lx, ly)
        assert e.value.code == code, (lx, ly, e.value.code)
        assert plan.psf_padding == (2 * nx, 2 * ny)  # unchanged
    nopsf = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5,
                 wterm=obs.wterm, mfs=True, no_psf=True)
    with pytest.raises(FastResolveError):
        nopsf.set_psf_padding(96, 96)


def _sampled_truncated(Pt, s, pix):
    """out(p) = sum_q PSF_t(p - q) s(q) at the pixels pix, one O(nx ny) dot product each."""
    nx, ny = s.shape
    out = []
    for px, py in pix:
        block = Pt[px + 1:px + nx + 1, py + 1:py + ny + 1][::-1, ::-1]
        out.append(float(np.sum(block * s)))
    return np.array(out)


@pytest.mark.slow
@pytest.mark.parametrize("lx,ly", [(1536, 1536), (1280, 1536)])
def test_vla_full_size_reduced_padding_sampled(lx, ly):
    """The VLA-like 1024^2 workload at full size: sampled pixels (corners and edges included)
    of the reduced-padding convolution against the oracle's per-pixel sums."""
    from paper_2406_09144_gb300.binding import Plan
    obs = synth.observation("vla")
    plan = Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=obs.weights, eps=1e-5,
                wterm=obs.wterm, mfs=True)
    P = psf_of(plan)[0]
    plan.set_psf_padding(lx, ly)
    nx, ny = obs.nx, obs.ny
    hx, hy = oracle.psf_window(nx, ny, lx, ly)
    Pt = oracle.truncate_psf(P, hx, hy)[0]
    s = synth.sky_image(nx, ny, seed=86)
    got = plan.psf_apply(dev(s[None, None])).cpu().numpy()[0, 0]
    rng = np.random.default_rng(87)
    pix = [(0, 0), (0, ny - 1), (nx - 1, 0), (nx - 1, ny - 1), (hx, hy), (nx - 1 - hx, 7)]
    pix += [tuple(p) for p in rng.integers(0, [nx, ny], size=(250, 2))]
    ref = _sampled_truncated(Pt, s, pix)
    g = np.array([got[p] for p in pix])
    assert rel(g, ref) <= 2e-6, rel(g, ref)
    # the truncation error against the whole PSF is what the reduced padding trades for speed
    full = _sampled_truncated(P, s, pix)
    assert rel(ref, full) > 0
