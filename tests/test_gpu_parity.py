"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative L2 over the whole output unless stated):
  * R, R^dagger N^-1, PSF (NUFFT outputs): <= eps = 1e-5 (the accuracy the plan is built for);
  * PSF convolution against the oracle's direct linear convolution of the GPU's own PSF:
    <= 2e-6 (FP32 FFTs only, no NUFFT);
  * adjointness <Rx, y> = <x, R^dagger y>, both sides on the GPU: <= 1e-6 relative;
  * likelihood value: <= 1e-5 relative; gradient: <= 1e-5 relative L2.
"""
import numpy as np
import pytest

import oracle
from oracle import cdft
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


def make_plan(obs, eps=EPS, mfs=False, nterm=True, wterm=None, **kw):
    from paper_2406_09144_gb300.binding import Plan
    return Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=obs.weights, eps=eps,
                wterm=obs.wterm if wterm is None else wterm, nterm=nterm, mfs=mfs, **kw)


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


CASES = [
    # nrow, nchan, nx, ny, wmax_cycles, per_channel
    (1500, 1, 32, 32, 0.0, False),
    (1200, 1, 32, 64, 3.0, False),
    (700, 2, 64, 32, 6.0, True),
    (600, 3, 32, 32, 2.0, False),
]


@pytest.mark.parametrize("case", CASES)
def test_degrid_matches_oracle(case):
    nrow, nchan, nx, ny, wc, per = case
    obs = synth.random_observation(nrow, nchan, nx, ny, 2e-3, seed=31, wmax_cycles=wc,
                                   per_channel_sky=per)
    plan = make_plan(obs, mfs=not per)
    sky = synth.random_skies(obs.nsky, nx, ny, seed=5)
    ref = oracle.degrid(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, wterm=obs.wterm)
    got = plan.degrid(dev(sky)).cpu().numpy()
    assert rel(got, ref) <= EPS, rel(got, ref)


@pytest.mark.parametrize("case", CASES)
def test_grid_matches_oracle(case):
    nrow, nchan, nx, ny, wc, per = case
    obs = synth.random_observation(nrow, nchan, nx, ny, 2e-3, seed=32, wmax_cycles=wc,
                                   per_channel_sky=per)
    plan = make_plan(obs, mfs=not per)
    vis = synth.complex_gaussian((nrow, nchan), seed=9)
    ref = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny,
                      weights=obs.weights.astype(np.float32), nsky=obs.nsky, wterm=obs.wterm)
    got = plan.grid(dev(vis, torch.complex64)).cpu().numpy()
    assert rel(got, ref) <= EPS, rel(got, ref)
    # unweighted
    ref1 = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny, nsky=obs.nsky,
                       wterm=obs.wterm)
    got1 = plan.grid(dev(vis, torch.complex64), apply_weights=False).cpu().numpy()
    assert rel(got1, ref1) <= EPS


@pytest.mark.parametrize("wc,nchan,per", [(0.003, 1, False), (0.02, 2, True), (0.05, 3, False)])
def test_small_w_expansion_matches_oracle(wc, nchan, per):
    """A w-phase far below one turn takes the truncated expansion in w instead of w-stacking;
    R, R^dagger and a point source's closed form must still match the oracle."""
    obs = synth.random_observation(1400, nchan, 64, 32, 2e-3, seed=44, wmax_cycles=wc,
                                   per_channel_sky=per)
    plan = make_plan(obs, mfs=not per)
    info = plan.info()
    assert info["dw"] == 0.0 and info["wplanes_max"] < info["support"] + 1
    sky = synth.random_skies(obs.nsky, 64, 32, seed=12)
    ref = oracle.degrid(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    assert rel(plan.degrid(dev(sky)).cpu().numpy(), ref) <= EPS
    vis = synth.complex_gaussian(plan.vis_shape, seed=13)
    refd = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 64, 32,
                       weights=obs.weights.astype(np.float32), nsky=obs.nsky)
    assert rel(plan.grid(dev(vis, torch.complex64)).cpu().numpy(), refd) <= EPS
    pt = np.zeros((obs.nsky, 64, 32))
    pt[:, 3, 29] = 1.0
    refp = oracle.degrid(pt, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    assert rel(plan.degrid(dev(pt)).cpu().numpy(), refp) <= EPS


@pytest.mark.parametrize("wc,eps,min_terms,W", [(0.12, 1e-5, 5, 7), (0.02, 1e-3, 1, 5),
                                                 (0.02, 1e-6, 1, 8)])
def test_small_w_expansion_term_counts_and_supports(wc, eps, min_terms, W):
    """Expansions that need two gridding passes (more than 4 terms, padded interleaved term
    grids when the count is odd), and the smallest and largest kernel supports."""
    obs = synth.random_observation(1100, 1, 64, 32, 2e-3, seed=46, wmax_cycles=wc)
    plan = make_plan(obs, eps=eps)
    info = plan.info()
    assert info["dw"] == 0.0 and info["support"] == W
    assert min_terms <= info["wplanes_max"] < W + 1
    tol = max(eps, 2e-6)  # FP32 arithmetic floors the achievable error near 1e-6
    sky = synth.random_skies(1, 64, 32, seed=14)
    ref = oracle.degrid(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    assert rel(plan.degrid(dev(sky)).cpu().numpy(), ref) <= tol
    vis = synth.complex_gaussian(plan.vis_shape, seed=15)
    refd = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 64, 32,
                       weights=obs.weights.astype(np.float32), nsky=1)
    got = plan.grid(dev(vis, torch.complex64)).cpu().numpy()
    assert rel(got, refd) <= tol
    # a second call leaves the same result (the term grids are cleared by the post-pass)
    assert rel(plan.grid(dev(vis, torch.complex64)).cpu().numpy(), got) <= 1e-6


def test_grid_twice_is_identical_workspace_stays_clean():
    obs = synth.random_observation(900, 1, 32, 32, 2e-3, seed=33, wmax_cycles=2.0)
    plan = make_plan(obs)
    vis = dev(synth.complex_gaussian((900, 1), seed=3), torch.complex64)
    a = plan.grid(vis).cpu().numpy()
    sky = dev(synth.random_skies(1, 32, 32, seed=1))
    plan.degrid(sky)  # degrid writes the shared grid workspace
    b = plan.grid(vis).cpu().numpy()
    assert rel(b, a) < 1e-6


def test_adjointness_on_gpu():
    obs = synth.random_observation(2000, 2, 64, 64, 2e-3, seed=34, wmax_cycles=4.0,
                                   per_channel_sky=True)
    plan = make_plan(obs)
    rng = np.random.default_rng(1)
    x = dev(rng.standard_normal(plan.sky_shape))
    y = dev(synth.complex_gaussian(plan.vis_shape, seed=2), torch.complex64)
    rx = plan.degrid(x).cpu().numpy().astype(np.complex128)
    rty = plan.grid(y, apply_weights=False).cpu().numpy().astype(np.float64)
    lhs = float(np.sum((np.conj(rx) * y.cpu().numpy()).real))
    rhs = float(np.sum(x.cpu().numpy() * rty))
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), np.linalg.norm(rx) * np.linalg.norm(y.cpu().numpy()))


def test_psf_and_norm_match_oracle():
    obs = synth.random_observation(1500, 2, 32, 32, 2e-3, seed=35, wmax_cycles=1.0,
                                   per_channel_sky=True)
    plan = make_plan(obs)
    _, psf, norm = plan.dirty_psf(want_dirty=False)
    w32 = obs.weights.astype(np.float32)
    ref = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 32, 32, w32, nsky=2)
    assert rel(psf.cpu().numpy(), ref) <= EPS
    assert np.allclose(norm, w32.astype(np.float64).sum(0), rtol=1e-12)
    assert np.allclose(norm, ref[:, 32, 32], rtol=1e-5)


def test_dirty_image_matches_grid():
    obs = synth.random_observation(800, 1, 32, 32, 2e-3, seed=36, wmax_cycles=1.0)
    plan = make_plan(obs)
    vis = dev(synth.complex_gaussian((800, 1), seed=4), torch.complex64)
    dirty, _, _ = plan.dirty_psf(vis, want_psf=False)
    assert rel(dirty.cpu().numpy(), plan.grid(vis).cpu().numpy()) < 1e-7


@pytest.mark.parametrize("nx,ny,batch", [(32, 32, 1), (32, 64, 3), (64, 16, 2), (128, 128, 2)])
def test_psf_apply_matches_direct_convolution(nx, ny, batch):
    # a 16-pixel axis has a 32-cell grid, so the kernel footprint limits |v| to ~0.3 / pixsize
    obs = synth.random_observation(1000, 1, nx, ny, 2e-3, seed=37, umax_frac=0.3)
    plan = make_plan(obs)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    P = psf.cpu().numpy().astype(np.float64)
    sky = synth.random_skies(batch, nx, ny, seed=8)[:, None]
    got = plan.psf_apply(dev(sky)).cpu().numpy()
    ref = oracle.psf_apply(P, sky[:, 0])[:, None]
    assert rel(got, ref) <= 2e-6, rel(got, ref)


def test_psf_convolution_equals_normal_operator_at_w0():
    """PSF * s vs R^dagger N^-1 R s at w = 0, 1/n = 1 (Sec. 3.3.2 exact for coplanar arrays)."""
    obs = synth.random_observation(3000, 1, 64, 64, 2e-3, seed=38)
    plan = make_plan(obs, nterm=False, wterm=False)
    sky = dev(synth.random_skies(1, 64, 64, seed=11))
    a = plan.psf_apply(sky).cpu().numpy()
    b = plan.grid(plan.degrid(sky)).cpu().numpy()
    assert rel(a, b) <= 2 * EPS


def test_likelihood_approx_matches_oracle():
    obs = synth.random_observation(1200, 1, 32, 32, 2e-3, seed=39)
    plan = make_plan(obs)
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    P = psf.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    sky = synth.random_skies(4, 32, 32, seed=2)[:, None]
    d = rng.standard_normal(sky.shape) * 50.0
    val, grad = plan.likelihood_grad(dev(sky), dev(d))
    rv, rg = oracle.likelihood(P, sky[:, 0], d[:, 0])
    assert np.allclose(val, rv, rtol=1e-5, atol=1e-5 * np.abs(rv).max())
    assert rel(grad.cpu().numpy()[:, 0], rg) <= 1e-5


def test_likelihood_exact_and_major_cycle_match_oracle():
    obs = synth.random_observation(900, 2, 32, 32, 2e-3, seed=40, wmax_cycles=2.0,
                                   per_channel_sky=True)
    plan = make_plan(obs)
    sky = synth.random_skies(2, 32, 32, seed=3)
    w32 = obs.weights.astype(np.float32)
    V = synth.complex_gaussian((900, 2), seed=5)
    dirty = oracle.grid(V, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 32, 32, weights=w32,
                        nsky=2, wterm=obs.wterm)
    rv, rg = oracle.likelihood_exact(sky, dirty, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize,
                                     weights=w32, wterm=obs.wterm)
    val, grad = plan.likelihood_grad(dev(sky[None]), dev(dirty[None]), exact=True)
    assert abs(val[0] - rv) <= 1e-5 * max(abs(rv), 1.0)
    assert rel(grad.cpu().numpy()[0], rg) <= EPS
    resid, rn2, chi2 = plan.major_cycle(dev(sky), dev(dirty), vis=dev(V, torch.complex64))
    rres = oracle.residual_dirty(dirty, sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize,
                                 weights=w32, wterm=obs.wterm)
    assert rel(resid.cpu().numpy(), rres) <= EPS
    assert abs(rn2 - float(np.sum(rres ** 2))) <= 2 * EPS * float(np.sum(rres ** 2))
    rchi = oracle.vis_residual_norm2(V, sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize,
                                     weights=w32, wterm=obs.wterm)
    assert abs(chi2 - rchi) <= 1e-5 * rchi


# ------------------------------------------------------------------ edge cases

def test_point_source_closed_form():
    """A unit point source gives V_k = exp(-2 pi i (u l0 + v m0 + w (n0 - 1))) / n0 exactly."""
    obs = synth.random_observation(1000, 1, 64, 64, 3e-3, seed=41, wmax_cycles=5.0)
    plan = make_plan(obs)
    sky = np.zeros((1, 64, 64))
    j0 = (40, 13)
    sky[0][j0] = 1.0
    got = plan.degrid(dev(sky)).cpu().numpy()[:, 0]
    l0, m0 = (j0[0] - 32) * obs.pixsize, (j0[1] - 32) * obs.pixsize
    n0 = np.sqrt(1 - l0 * l0 - m0 * m0)
    u, v, w = (x[:, 0] for x in oracle.uvw_to_wavelengths(obs.uvw, obs.freqs))
    ref = np.exp(-2j * np.pi * (u * l0 + v * m0 + w * (n0 - 1))) / n0
    assert rel(got, ref) <= EPS


def test_dropped_and_flagged_visibilities():
    obs = synth.random_observation(500, 1, 32, 32, 2e-3, seed=42, wmax_cycles=1.0)
    uvw = obs.uvw.copy()
    lam = oracle.C_LIGHT / obs.freqs[0]
    uvw[:7, 0] = 0.499 / obs.pixsize * lam  # footprint leaves the grid
    w = obs.weights.copy()
    w[10:20] = 0.0  # flagged
    from paper_2406_09144_gb300.binding import Plan, FastResolveError
    with pytest.raises(FastResolveError):
        Plan(uvw, obs.freqs, 32, 32, obs.pixsize, weights=w, eps=EPS)
    plan = Plan(uvw, obs.freqs, 32, 32, obs.pixsize, weights=w, eps=EPS, drop_oob=True)
    assert plan.info()["nvis_dropped"] == 7
    sky = synth.random_skies(1, 32, 32, seed=6)
    got = plan.degrid(dev(sky)).cpu().numpy()
    assert np.all(got[:7] == 0)
    ref = oracle.degrid(sky, uvw[7:], obs.freqs, obs.pixsize, obs.pixsize)
    assert rel(got[7:], ref) <= EPS
    vis = synth.complex_gaussian((500, 1), seed=7)
    g = plan.grid(dev(vis, torch.complex64)).cpu().numpy()
    rg = oracle.grid(vis[7:], uvw[7:], obs.freqs, obs.pixsize, obs.pixsize, 32, 32,
                     weights=w[7:].astype(np.float32))
    assert rel(g, rg) <= EPS


def test_all_visibilities_dropped():
    """Degenerate plan: every footprint leaves the grid and is dropped. R gives zeros, R^dagger
    a zero image, and the PSF (no weight) is zero."""
    obs = synth.random_observation(64, 1, 32, 32, 2e-3, seed=47, wmax_cycles=1.0)
    uvw = obs.uvw.copy()
    lam = oracle.C_LIGHT / obs.freqs[0]
    uvw[:, 0] = 0.499 / obs.pixsize * lam
    from paper_2406_09144_gb300.binding import Plan
    plan = Plan(uvw, obs.freqs, 32, 32, obs.pixsize, weights=obs.weights, eps=EPS, drop_oob=True)
    assert plan.info()["nvis_dropped"] == 64
    sky = synth.random_skies(1, 32, 32, seed=8)
    assert np.all(plan.degrid(dev(sky)).cpu().numpy() == 0)
    vis = dev(synth.complex_gaussian((64, 1), seed=9), torch.complex64)
    assert np.all(plan.grid(vis).cpu().numpy() == 0)
    _, psf, norm = plan.dirty_psf(want_dirty=False)
    assert np.all(psf.cpu().numpy() == 0) and np.all(norm == 0)


def test_single_visibility_at_origin():
    """A single visibility y at u = v = w = 0 grids to D_j = Re(y) / n_j (closed form)."""
    from paper_2406_09144_gb300.binding import Plan
    plan = Plan(np.zeros((1, 3)), [1e9], 32, 32, 1e-2, eps=EPS)
    y = dev(np.array([[2.0 - 1.0j]]), torch.complex64)
    d = plan.grid(y).cpu().numpy()[0]
    _, _, n = oracle.direction_cosines(32, 32, 1e-2, 1e-2)
    assert rel(d, 2.0 / n) <= EPS


def test_plan_info_and_footprint():
    obs = synth.random_observation(500, 2, 32, 32, 2e-3, seed=43, wmax_cycles=3.0,
                                   per_channel_sky=True)
    plan = make_plan(obs)
    info = plan.info()
    assert info["nsky"] == 2 and info["grid_nu"] == 64 and info["support"] >= 5
    assert info["wplanes_total"] >= 2 * info["support"]
    res, ws = plan.footprint()
    assert res > 0 and ws > 0
    plan.check()


# ------------------------------------------------------------------ the PSF chain, oracle PSF

@pytest.mark.parametrize("nchan,per", [(1, False), (2, True)])
def test_psf_convolution_chain_against_oracle_psf(nchan, per):
    """The whole PSF path against the oracle alone: the FP64 oracle PSF (Sec. 3.3.2, direct
    sums) convolved with each sky by the oracle's direct linear convolution, against
    fr_psf_apply, whose PSF the library grids itself (NUFFT at eps) and whose convolution runs
    on its own FFT passes."""
    nx, ny = 64, 48
    obs = synth.random_observation(2000, nchan, nx, ny, 2e-3, seed=70, per_channel_sky=per)
    plan = make_plan(obs, mfs=not per)
    w32 = obs.weights.astype(np.float32)
    P = oracle.psf(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, nx, ny, weights=w32,
                   nsky=plan.nsky)
    sky = synth.random_skies(2 * plan.nsky, nx, ny, seed=71).reshape(2, plan.nsky, nx, ny)
    got = plan.psf_apply(dev(sky)).cpu().numpy()
    ref = np.stack([oracle.psf_apply(P[k:k + 1], sky[:, k]) for k in range(plan.nsky)], axis=1)
    assert rel(got, ref) <= EPS, rel(got, ref)


# ------------------------------------------------------------------ full size

NVIS_SAMPLE = 10_000   # sampled visibilities, each an O(N_pix) FP64 direct sum
NPIX_SAMPLE = 1_000    # sampled pixels, each an O(N_vis) FP64 direct sum


@pytest.mark.slow
def test_small_full_brute_force():
    """Plain method, small (128^2, 1 channel at 1.4 GHz, 505,440 visibilities, w = 0): every
    output of R, R^dagger N^-1 and the PSF convolution against the FP64 direct sums. At w = 0
    with 1/n = 1 the PSF convolution equals R^dagger N^-1 R exactly (Sec. 3.3.2), so its oracle
    is the direct R followed by the direct R^dagger N^-1."""
    obs = synth.observation("small")
    assert obs.nrow == 505_440 and not obs.wterm
    plan = make_plan(obs)
    n = obs.nx
    sky = synth.sky_image(n, n, seed=0)[None]
    rows, chans = np.arange(obs.nrow), np.zeros(obs.nrow, int)
    vis = plan.degrid(dev(sky)).cpu().numpy()
    ref = cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows, chans,
                         wterm=False)
    assert rel(vis[:, 0], ref) <= EPS, rel(vis[:, 0], ref)
    w32 = obs.weights.astype(np.float32)
    pix = np.arange(n * n)
    y = synth.complex_gaussian((obs.nrow, 1), seed=1)
    d = plan.grid(dev(y, torch.complex64)).cpu().numpy()
    refd = cdft.grid_at(y, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, n, n,
                        np.zeros(n * n, int), pix, weights=w32, wterm=False)
    assert rel(d.reshape(-1), refd) <= EPS, rel(d.reshape(-1), refd)
    conv = plan.psf_apply(dev(sky[None])).cpu().numpy()[0, 0]
    v0 = cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows, chans,
                        wterm=False, nterm=False)
    refc = cdft.grid_at(v0[:, None], obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, n, n,
                        np.zeros(n * n, int), pix, weights=w32, wterm=False, nterm=False)
    assert rel(conv.reshape(-1), refc) <= EPS, rel(conv.reshape(-1), refc)


def _sampled_psf_checks(plan, obs, sky, dirty, rng, npix_psf, npix_conv):
    """The PSF image at sampled offsets against the oracle's direct sums (<= eps), and the
    likelihood gradient PSF * s - d of the benchmark's call at sampled pixels against the
    oracle's direct linear convolution of that PSF image (<= 2e-6: FP32 FFTs only)."""
    nx, ny = obs.nx, obs.ny
    w32 = obs.weights.astype(np.float32)
    _, grad = plan.likelihood_grad(dev(sky[None]), dev(dirty[None]), want_value=False)
    grad = grad.cpu().numpy()[0]
    _, psf, _ = plan.dirty_psf(want_dirty=False)
    for k in range(plan.nsky):
        P = psf[k].cpu().numpy().astype(np.float64)
        a = rng.integers(-nx + 1, nx, npix_psf)
        b = rng.integers(-ny + 1, ny, npix_psf)
        refp = cdft.psf_at(obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, np.full(npix_psf, k),
                           a, b, weights=w32, nsky=plan.nsky)
        assert rel(P[a + nx, b + ny], refp) <= EPS, (k, rel(P[a + nx, b + ny], refp))
        pix = rng.integers(0, nx * ny, npix_conv)
        refc = oracle.psf_apply_at(P, sky[k], pix) - dirty[k].reshape(-1)[pix]
        assert rel(grad[k].reshape(-1)[pix], refc) <= 2e-6, (k, rel(grad[k].reshape(-1)[pix], refc))


@pytest.mark.slow
def test_vla_full_size_sampled():
    """VLA-like workload at full size (1024^2, 5,054,400 visibilities, w-terms, PSF convolution
    on the 2048^2 padded grid) in the launch configuration the benchmark times: 10^4 sampled
    visibilities of R and 10^3 sampled pixels of R^dagger N^-1 against the FP64 direct sums,
    and the PSF and the likelihood gradient at sampled points."""
    obs = synth.observation("vla")
    plan = make_plan(obs)
    rng = np.random.default_rng(0)
    n = obs.nx
    sky = synth.sky_image(n, n, seed=0)[None]
    vis = plan.degrid(dev(sky)).cpu().numpy()
    rows = rng.integers(0, obs.nrow, NVIS_SAMPLE)
    ref = cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows,
                         np.zeros(NVIS_SAMPLE, int))
    assert rel(vis[rows, 0], ref) <= EPS, rel(vis[rows, 0], ref)
    y = synth.complex_gaussian((obs.nrow, 1), seed=1)
    d = plan.grid(dev(y, torch.complex64)).cpu().numpy()
    pix = rng.integers(0, n * n, NPIX_SAMPLE)
    w32 = obs.weights.astype(np.float32)
    refd = cdft.grid_at(y, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, n, n,
                        np.zeros(NPIX_SAMPLE, int), pix, weights=w32)
    assert rel(d.reshape(-1)[pix], refd) <= EPS, rel(d.reshape(-1)[pix], refd)
    _sampled_psf_checks(plan, obs, sky, d.reshape(1, n, n), rng, NPIX_SAMPLE, 300)


@pytest.mark.slow
def test_meerkat_all_channels_full_size_sampled():
    """MeerKAT-like multi-channel workload at full size, the benchmark's default: 8 channels of
    4096^2 skies (w-stacking on 8192^2 grids, 58,060,800 visibilities) and the PSF likelihood on
    8192^2 padded grids, in the benchmark's launch configuration. 10^4 visibilities sampled over
    all rows and channels, 10^3 pixels over all 8 images, against the FP64 direct sums; the PSF
    images and the likelihood gradient at sampled points."""
    obs = synth.observation("meerkat")
    plan = make_plan(obs, mfs=not obs.per_channel_sky)
    assert plan.nsky == 8 and plan.info()["wplanes_max"] > plan.info()["support"]
    rng = np.random.default_rng(2)
    n = obs.nx
    sky = synth.random_skies(8, n, n, seed=3)
    vis = plan.degrid(dev(sky)).cpu().numpy()
    rows = rng.integers(0, obs.nrow, NVIS_SAMPLE)
    chans = rng.integers(0, 8, NVIS_SAMPLE)
    ref = cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows, chans)
    assert rel(vis[rows, chans], ref) <= EPS, rel(vis[rows, chans], ref)
    del vis
    y = synth.complex_gaussian((obs.nrow, 8), seed=4)
    d = plan.grid(dev(y, torch.complex64)).cpu().numpy()
    imgs = rng.integers(0, 8, NPIX_SAMPLE)
    pix = rng.integers(0, n * n, NPIX_SAMPLE)
    w32 = obs.weights.astype(np.float32)
    refd = cdft.grid_at(y, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, n, n, imgs, pix,
                        weights=w32, nsky=8)
    got = d.reshape(8, -1)[imgs, pix]
    assert rel(got, refd) <= EPS, rel(got, refd)
    _sampled_psf_checks(plan, obs, sky, d, rng, 200, 40)
