"""Major/minor inference loop of Alg. 1 (Sec. 3.3.4) on the library's operators.

    I^D = R^dagger N^-1 V                                   (exact, fr_grid)
    d_0 = I^D
    for i in 0 .. n_major - 1:
        minor cycle: estimate I_i from d_i = PSF * (I - I_{i-1}) + n'      (Eq. ham_new)
        major cycle: d_{i+1} = I^D - R^dagger N^-1 R I_i                    (exact, fr_major_cycle)

The paper's minor cycle is MGVI/geoVI variational inference (Sec. 3.3.5), outside this
library. As a stand-in this module takes the maximum a posteriori sky under a positive
log-normal prior, I = exp(phi) with phi ~ N(mu, sigma^2) per pixel, minimising
Eq. ham_new (fr_fast_likelihood_grad) plus the prior with L-BFGS in torch. Every operator call
runs in the library's CUDA kernels; torch holds the parameters and runs the optimiser.
"""
import math

import numpy as np


def reconstruct(plan, vis, n_major=3, n_minor=25, eps_noise=None, prior_mean=None,
                prior_sigma=3.0, psf_padding=None, stream=None):
    """Run Alg. 1. vis: device complex64 [nrow, nchan] (user order). Returns (sky, history),
    history = [{"major": i, "resid_norm2": |d_{i+1}|^2, "minor_value": last H + prior}].

    eps_noise: the white-noise variance of Eq. N_new (default: 1e-4 of the PSF peak, i.e. of
    the summed weights per image). prior_mean: mu of the log-sky (default: ln of 1e-3 of the
    dirty image's maximum over the PSF peak). psf_padding: (lx, ly) for the minor cycles' PSF
    convolutions (reduced padding, Sec. 3.3.2; the plan's setting is restored afterwards);
    the major cycles stay exact, so they correct what the truncated PSF misses.
    """
    import torch

    if psf_padding is not None:
        saved = plan.psf_padding
        plan.set_psf_padding(*psf_padding, stream=stream)
        try:
            return reconstruct(plan, vis, n_major, n_minor, eps_noise, prior_mean, prior_sigma,
                               None, stream)
        finally:
            plan.set_psf_padding(*saved, stream=stream)

    dirty = plan.grid(vis, stream=stream)
    _, psf, norm = plan.dirty_psf(want_dirty=False, stream=stream)
    peak = float(np.max(norm))
    if eps_noise is None:
        eps_noise = 1e-4 * peak
    plan.noise_fit(eps_noise, stream=stream)
    flux = max(float(dirty.max()) / peak, 1e-30)  # a point source's flux from its dirty peak
    if prior_mean is None:
        prior_mean = math.log(flux * 1e-3)
    # the optimiser's trial steps are kept finite: no pixel above 100 times that flux
    phi_max = math.log(flux * 100.0)
    phi = torch.full(dirty.shape, prior_mean, dtype=torch.float32, device=dirty.device,
                     requires_grad=True)
    inv_var = 1.0 / (prior_sigma * prior_sigma)
    # the optimiser sees the objective divided by the PSF peak (the summed weights), which
    # keeps its curvature estimates in range; the minimiser is the same
    scale = 1.0 / peak
    prev = torch.zeros_like(dirty)
    d = dirty
    history = []
    sky = torch.exp(torch.clamp(phi.detach(), max=phi_max))
    for i in range(n_major):
        opt = torch.optim.LBFGS([phi], max_iter=n_minor, history_size=10,
                                line_search_fn="strong_wolfe")
        last = {}

        def closure():
            opt.zero_grad()
            with torch.no_grad():
                capped = phi > phi_max
                s = torch.exp(torch.clamp(phi, max=phi_max))
                val, g = plan.fast_likelihood_grad(s - prev, d, stream=stream)
                dp = phi - prior_mean
                prior = 0.5 * inv_var * float(torch.sum(dp.double() * dp.double()))
                phi.grad = scale * (torch.where(capped, torch.zeros_like(g), g * s) + inv_var * dp)
            last["value"] = float(val[0]) + prior
            return torch.tensor(scale * last["value"], dtype=torch.float64)

        opt.step(closure)
        sky = torch.exp(torch.clamp(phi.detach(), max=phi_max))
        # major cycle: residual of the dirty image against the exact normal operator
        d, rn2, _ = plan.major_cycle(sky, dirty, stream=stream)
        prev = sky
        history.append({"major": i, "resid_norm2": rn2, "minor_value": last.get("value")})
    return sky, history
