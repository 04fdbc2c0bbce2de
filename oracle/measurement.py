"""FP64 direct-sum definitions of R, R^dagger, the PSF, PSF convolution and the likelihood.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the product path never imports this.

Conventions (readings where the paper is silent):
  * pixel (jx, jy) of an [nx, ny] image sits at l = (jx - nx//2) * dl, m = (jy - ny//2) * dm;
    the array is row-major with jy fastest and x <-> l <-> u;
  * the integral over the sky in Eq. (rime) is a plain sum over pixels (brightness per pixel);
  * pixels with l^2 + m^2 >= 1 contribute nothing;
  * gains G are 1 (scalar, calibrated data);
  * a sky stack has nsky = 1 (one image for all channels; R^dagger sums channels) or
    nsky = nchan (one image per channel; R^dagger keeps channels apart).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0  # m/s


def uvw_to_wavelengths(uvw, freqs):
    """Baseline coordinates in units of the observing wavelength, Eq. (rime): k = uvw * nu / c.

    uvw [nrow, 3] metres, freqs [nchan] Hz -> (u, v, w), each [nrow, nchan] float64.
    """
    uvw = np.asarray(uvw, dtype=np.float64)
    scale = np.asarray(freqs, dtype=np.float64)[None, :] / C_LIGHT
    return uvw[:, 0:1] * scale, uvw[:, 1:2] * scale, uvw[:, 2:3] * scale


def pixel_lm(nx, ny, dl, dm):
    """Sky coordinates of pixel centres: l [nx], m [ny] (radians, direction cosines)."""
    l = (np.arange(nx, dtype=np.float64) - nx // 2) * dl
    m = (np.arange(ny, dtype=np.float64) - ny // 2) * dm
    return l, m


def direction_cosines(nx, ny, dl, dm):
    """l, m, n = sqrt(1 - l^2 - m^2) on the pixel grid, each [nx, ny]; n = nan outside the unit disc."""
    l, m = pixel_lm(nx, ny, dl, dm)
    L, M = np.meshgrid(l, m, indexing="ij")
    r2 = L * L + M * M
    n = np.where(r2 < 1.0, np.sqrt(np.maximum(1.0 - r2, 0.0)), np.nan)
    return L, M, n


def _sky_terms(nx, ny, dl, dm, wterm, nterm):
    """Per-pixel flat arrays (l, m, n - 1 or 0, 1/n or 1, inside-disc mask) for Eq. (rime)."""
    L, M, n = direction_cosines(nx, ny, dl, dm)
    inside = np.isfinite(n)
    nn = np.where(inside, n, 1.0)
    t = (nn - 1.0) if wterm else np.zeros_like(nn)
    amp = (1.0 / nn) if nterm else np.ones_like(nn)
    amp = np.where(inside, amp, 0.0)
    return L.ravel(), M.ravel(), t.ravel(), amp.ravel()


def _sky_for_channel(sky, c):
    return sky[0] if sky.shape[0] == 1 else sky[c]


def degrid(sky, uvw, freqs, dl, dm, wterm=True, nterm=True, chunk=256):
    """R, Eq. (rime) with G = 1:

        V_k = sum_j I_j / n_j * exp(-2 pi i (u_k l_j + v_k m_j + w_k (n_j - 1)))

    sky [nsky, nx, ny] (nsky in {1, nchan}) -> vis [nrow, nchan] complex128.
    wterm=False sets the w phase to zero; nterm=False sets 1/n to 1.
    """
    sky = np.asarray(sky, dtype=np.float64)
    if sky.ndim == 2:
        sky = sky[None]
    nsky, nx, ny = sky.shape
    u, v, w = uvw_to_wavelengths(uvw, freqs)
    nrow, nchan = u.shape
    if nsky not in (1, nchan):
        raise ValueError("nsky must be 1 or nchan")
    l, m, t, amp = _sky_terms(nx, ny, dl, dm, wterm, nterm)
    vis = np.zeros((nrow, nchan), dtype=np.complex128)
    for c in range(nchan):
        a = _sky_for_channel(sky, c).ravel() * amp
        for k0 in range(0, nrow, chunk):
            k1 = min(nrow, k0 + chunk)
            phase = (np.outer(u[k0:k1, c], l) + np.outer(v[k0:k1, c], m)
                     + np.outer(w[k0:k1, c], t))
            vis[k0:k1, c] = np.exp(-2j * np.pi * phase) @ a
    return vis


def grid(vis, uvw, freqs, dl, dm, nx, ny, weights=None, nsky=1, wterm=True, nterm=True,
         chunk=4096):
    """R^dagger N^-1 applied to visibilities: the adjoint of R under the real inner product
    (the sky is real), with N^-1 the visibility weights (Sec. 3.1.2, Eq. clean):

        D_j = Re sum_k w_k y_k exp(+2 pi i (u_k l_j + v_k m_j + w_k (n_j - 1))) / n_j

    vis [nrow, nchan] complex, weights [nrow, nchan] or None (= 1).
    nsky = 1 sums all channels into one image; nsky = nchan keeps one image per channel.
    Returns [nsky, nx, ny] float64.
    """
    vis = np.asarray(vis, dtype=np.complex128)
    u, v, w = uvw_to_wavelengths(uvw, freqs)
    nrow, nchan = u.shape
    if nsky not in (1, nchan):
        raise ValueError("nsky must be 1 or nchan")
    y = vis if weights is None else vis * np.asarray(weights, dtype=np.float64)
    l, m, t, amp = _sky_terms(nx, ny, dl, dm, wterm, nterm)
    out = np.zeros((nsky, nx * ny), dtype=np.float64)
    for c in range(nchan):
        acc = np.zeros(nx * ny, dtype=np.complex128)
        for k0 in range(0, nrow, chunk):
            k1 = min(nrow, k0 + chunk)
            for j0 in range(0, nx * ny, chunk):
                j1 = min(nx * ny, j0 + chunk)
                phase = (np.outer(l[j0:j1], u[k0:k1, c]) + np.outer(m[j0:j1], v[k0:k1, c])
                         + np.outer(t[j0:j1], w[k0:k1, c]))
                acc[j0:j1] += np.exp(2j * np.pi * phase) @ y[k0:k1, c]
        out[0 if nsky == 1 else c] += (acc * amp).real
    return out.reshape(nsky, nx, ny)


def psf(uvw, freqs, dl, dm, nx, ny, weights=None, nsky=1):
    """Point spread function on the 2x padded grid (Sec. 3.2 and 3.3.2), neglecting wide-field
    effects (w = 0, 1/n = 1), unnormalised so that PSF * I equals R^dagger N^-1 R I at w = 0:

        PSF(a, b) = sum_k w_k cos(2 pi (u_k a dl + v_k b dm)),  a in [-nx, nx), b in [-ny, ny)

    stored at index (a + nx, b + ny), so offset 0 sits at (nx, ny). The row a = -nx and the
    column b = -ny are never reached by the cropped linear convolution and are set to zero,
    which makes the stored PSF exactly even about (nx, ny). Returns [nsky, 2nx, 2ny].
    """
    u, v, _ = uvw_to_wavelengths(uvw, freqs)
    nrow, nchan = u.shape
    wt = np.ones((nrow, nchan)) if weights is None else np.asarray(weights, dtype=np.float64)
    a = np.arange(-nx, nx, dtype=np.float64) * dl
    b = np.arange(-ny, ny, dtype=np.float64) * dm
    A, B = np.meshgrid(a, b, indexing="ij")
    A, B = A.ravel(), B.ravel()
    out = np.zeros((nsky, 4 * nx * ny), dtype=np.float64)
    chunk = 4096
    for c in range(nchan):
        acc = np.zeros(4 * nx * ny)
        for k0 in range(0, nrow, chunk):
            k1 = min(nrow, k0 + chunk)
            phase = np.outer(A, u[k0:k1, c]) + np.outer(B, v[k0:k1, c])
            acc += np.cos(2.0 * np.pi * phase) @ wt[k0:k1, c]
        out[0 if nsky == 1 else c] += acc
    out = out.reshape(nsky, 2 * nx, 2 * ny)
    out[:, 0, :] = 0.0
    out[:, :, 0] = 0.0
    return out


def psf_apply(psf_img, sky):
    """Linear (non-circular) convolution of each sky with the PSF, cropped to the sky
    (Sec. 3.3.2: the padded FFT convolution evaluates exactly this):

        out_b(p) = sum_{q in sky} PSF(p - q) s_b(q)

    psf_img [npsf, 2nx, 2ny] with npsf = 1 (shared) or npsf = B; sky [B, nx, ny].
    """
    sky = np.asarray(sky, dtype=np.float64)
    if sky.ndim == 2:
        sky = sky[None]
    psf_img = np.asarray(psf_img, dtype=np.float64)
    if psf_img.ndim == 2:
        psf_img = psf_img[None]
    nb, nx, ny = sky.shape
    out = np.zeros_like(sky)
    for bi in range(nb):
        P = psf_img[0 if psf_img.shape[0] == 1 else bi]
        s = sky[bi]
        for qx in range(nx):
            for qy in range(ny):
                val = s[qx, qy]
                if val != 0.0:
                    # offsets p - q for p in [0, nx) x [0, ny) at index (p - q) + (nx, ny)
                    out[bi] += val * P[nx - qx:2 * nx - qx, ny - qy:2 * ny - qy]
    return out


def psf_apply_at(psf_img, sky, pix):
    """The linear convolution of psf_apply at chosen output pixels only (Sec. 3.3.2), each an
    O(nx ny) sum, for checks of large images:

        out(p) = sum_{q in sky} PSF(p - q) s(q),   p = (pix // ny, pix % ny)

    psf_img [2nx, 2ny] (offset (a, b) at index (a + nx, b + ny)), sky [nx, ny]; float64 [n].
    """
    P = np.asarray(psf_img, dtype=np.float64)
    s = np.asarray(sky, dtype=np.float64)
    nx, ny = s.shape
    out = np.empty(len(pix))
    for i, k in enumerate(np.asarray(pix, dtype=np.int64)):
        px, py = int(k) // ny, int(k) % ny
        # offsets p - q for q in [0, nx) x [0, ny): index (px - qx + nx, py - qy + ny)
        window = P[px + 1:px + nx + 1, py + 1:py + ny + 1][::-1, ::-1]
        out[i] = float(np.sum(window * s))
    return out


def psf_window(nx, ny, lx, ly):
    """Half-widths (hx, hy) of the PSF window a zero-padded lx x ly grid holds without
    wrap-around (reduced padding, Sec. 3.3.2): hx = min(lx - nx, nx - 1), hy likewise.
    lx = 2nx, ly = 2ny give (nx - 1, ny - 1): every offset of the cropped product."""
    return min(lx - nx, nx - 1), min(ly - ny, ny - 1)


def truncate_psf(psf_img, hx, hy):
    """The PSF image with the sidelobes at offsets |a| > hx or |b| > hy set to zero (the
    reduced padding of Sec. 3.3.2 neglects them). psf_img [npsf, 2nx, 2ny] (offset (a, b) at
    index (a + nx, b + ny)) -> same shape, float64."""
    P = np.array(psf_img, dtype=np.float64)
    if P.ndim == 2:
        P = P[None]
    _, nx2, ny2 = P.shape
    a = np.arange(nx2) - nx2 // 2
    b = np.arange(ny2) - ny2 // 2
    keep = (np.abs(a)[:, None] <= hx) & (np.abs(b)[None, :] <= hy)
    return P * keep[None]


def psf_apply_truncated(psf_img, sky, lx, ly):
    """PSF convolution with reduced padding (Sec. 3.3.2) on an lx x ly padded grid: the linear
    convolution of psf_apply with the PSF truncated to the window psf_window(nx, ny, lx, ly).

        out_b(p) = sum_{q in sky} PSF_t(p - q) s_b(q)
    """
    sky = np.asarray(sky, dtype=np.float64)
    nx, ny = sky.shape[-2:]
    hx, hy = psf_window(nx, ny, lx, ly)
    return psf_apply(truncate_psf(psf_img, hx, hy), sky)


def likelihood(psf_img, sky, dirty):
    """Likelihood in image space with the PSF approximation R^dagger N^-1 R ~ PSF * (Sec. 3.3.2):
    Eq. (ham) expanded with Eq. (clean) and constants dropped,

        L(s) = 1/2 s^T (PSF * s) - s^T d,    grad L = PSF * s - d.

    sky, dirty [B, nx, ny]; returns (L [B] float64, grad [B, nx, ny] float64).
    """
    sky = np.asarray(sky, dtype=np.float64)
    dirty = np.asarray(dirty, dtype=np.float64)
    conv = psf_apply(psf_img, sky)
    val = 0.5 * np.einsum("bij,bij->b", sky, conv) - np.einsum("bij,bij->b", sky, dirty)
    return val, conv - dirty


def likelihood_exact(sky, dirty, uvw, freqs, dl, dm, weights=None, wterm=True, nterm=True):
    """Same likelihood with the exact normal operator R^dagger N^-1 R in place of the PSF.

    sky, dirty [nsky, nx, ny] (nsky in {1, nchan}); returns (L scalar, grad [nsky, nx, ny]).
    """
    sky = np.asarray(sky, dtype=np.float64)
    nsky, nx, ny = sky.shape
    vis = degrid(sky, uvw, freqs, dl, dm, wterm=wterm, nterm=nterm)
    rr = grid(vis, uvw, freqs, dl, dm, nx, ny, weights=weights, nsky=nsky, wterm=wterm,
              nterm=nterm)
    val = 0.5 * float(np.sum(sky * rr)) - float(np.sum(sky * dirty))
    return val, rr - dirty


def residual_dirty(dirty, sky, uvw, freqs, dl, dm, weights=None, wterm=True, nterm=True):
    """Major-cycle residual of Algorithm 1: d = I^D - R^dagger N^-1 R I."""
    sky = np.asarray(sky, dtype=np.float64)
    nsky, nx, ny = sky.shape
    vis = degrid(sky, uvw, freqs, dl, dm, wterm=wterm, nterm=nterm)
    rr = grid(vis, uvw, freqs, dl, dm, nx, ny, weights=weights, nsky=nsky, wterm=wterm,
              nterm=nterm)
    return np.asarray(dirty, dtype=np.float64) - rr


def vis_residual_norm2(vis, sky, uvw, freqs, dl, dm, weights=None, wterm=True, nterm=True):
    """Data-space misfit of Eq. (ham): (V - R I)^dagger N^-1 (V - R I) = sum_k w_k |V_k - (R I)_k|^2."""
    model = degrid(sky, uvw, freqs, dl, dm, wterm=wterm, nterm=nterm)
    r = np.asarray(vis, dtype=np.complex128) - model
    wt = 1.0 if weights is None else np.asarray(weights, dtype=np.float64)
    return float(np.sum(wt * (r.real ** 2 + r.imag ** 2)))
