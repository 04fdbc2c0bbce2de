"""FP64 oracle of the fast-resolve noise model and likelihood (test infrastructure only).

Sec. 3.3.1 (Eq. ham_new, Eq. N_new): the image-space likelihood
    H(I^D | I) = 1/2 (I^D - R'I)^T N'^-1 (I^D - R'I) + 1/2 ln|2 pi N'|,
    N' = R^dagger N^-1 R + eps 1.
Sec. 3.3.2: R'I ~ PSF * I (the padded, linear convolution of measurement.psf_apply).
Sec. 3.3.3: N' is replaced by a periodic convolution on the nx x ny image with the real,
positive transfer function K = exp(xi) + eps,
    N'(x) ~ FFT^-1[K . FFT(x)],   N'^-1(x) ~ FFT^-1[K^-1 . FFT(x)],
with xi fitted to the exact N' applied to a centre delta:
    xi = argmin_xi || N'(I_delta) - FFT^-1[(exp xi + eps) . FFT(I_delta)] ||^2.

The FFTs are the paper's own definition of these operators (numpy.fft, unnormalised forward,
1/N inverse). The fit is the argmin itself, solved numerically as a bound-constrained linear
least-squares problem on the dense operator.
"""
import numpy as np

from . import measurement as M


def centre_delta(nsky, nx, ny):
    """I_delta: a unit point source in the centre pixel (nx/2, ny/2) of every image."""
    d = np.zeros((nsky, nx, ny))
    d[:, nx // 2, ny // 2] = 1.0
    return d


def normal_operator(sky, uvw, freqs, dl, dm, weights=None, wterm=True, nterm=True):
    """Exact R^dagger N^-1 R sky (direct sums of Eq. rime and its adjoint)."""
    sky = np.asarray(sky, dtype=np.float64)
    nsky, nx, ny = sky.shape
    vis = M.degrid(sky, uvw, freqs, dl, dm, wterm=wterm, nterm=nterm)
    return M.grid(vis, uvw, freqs, dl, dm, nx, ny, weights=weights, nsky=nsky, wterm=wterm,
                  nterm=nterm)


def noise_cov_of_delta(uvw, freqs, dl, dm, nx, ny, eps_noise, weights=None, nsky=1, wterm=True,
                       nterm=True):
    """N'(I_delta) = R^dagger N^-1 R I_delta + eps I_delta (Eq. N_new), [nsky, nx, ny]."""
    delta = centre_delta(nsky, nx, ny)
    return normal_operator(delta, uvw, freqs, dl, dm, weights, wterm, nterm) + eps_noise * delta


def periodic_convolve(x, K):
    """FFT^-1[K . FFT(x)] per image (x [B, nx, ny], K [B or 1, nx, ny]); the real part."""
    return np.real(np.fft.ifft2(np.asarray(K) * np.fft.fft2(x, axes=(-2, -1)), axes=(-2, -1)))


def noise_inverse(x, K):
    """N'^-1 x ~ FFT^-1[K^-1 . FFT(x)] (Sec. 3.3.3, periodic boundaries)."""
    return periodic_convolve(x, 1.0 / np.asarray(K))


def fit_noise_kernel(n_delta, eps_noise):
    """K = exp(xi) + eps with xi the argmin of Sec. 3.3.3, one kernel per image.

    n_delta [nsky, nx, ny] = N'(I_delta). The model FFT^-1[K . FFT(I_delta)] is linear in K, so
    the loss is a linear least-squares problem in K over K > eps; its argmin over xi is the
    bound-constrained minimiser with K >= eps (K = eps being the limit xi -> -inf). It is
    solved on the dense operator (columns FFT^-1[e_k . FFT(I_delta)], real and imaginary parts
    stacked) by scipy.optimize.lsq_linear, after dividing the target and eps by
    s = max|n_delta| (the argmin scales with them).
    """
    from scipy import optimize

    n_delta = np.asarray(n_delta, dtype=np.float64)
    nsky, nx, ny = n_delta.shape
    N = nx * ny
    D = np.fft.fft2(centre_delta(1, nx, ny)[0])
    cols = np.fft.ifft2(np.eye(N).reshape(N, nx, ny) * D[None], axes=(1, 2)).reshape(N, N).T
    A = np.concatenate([cols.real, cols.imag])  # [2N, N]: image residual (re, im) per K_k
    out = np.empty_like(n_delta)
    for s in range(nsky):
        scale = float(np.max(np.abs(n_delta[s]))) or 1.0
        b = np.concatenate([n_delta[s].ravel() / scale, np.zeros(N)])
        eps = eps_noise / scale
        res = optimize.lsq_linear(A, b, bounds=(eps, np.inf), method="bvls", tol=1e-15,
                                  lsmr_tol="auto")
        out[s] = res.x.reshape(nx, ny) * scale
    return out


def fast_hamiltonian(psf_img, sky, dirty, K):
    """Eq. ham_new with R' = PSF * (padded, linear) and N'^-1 from the kernel K:

        r = I^D - PSF * I,   H = 1/2 r^T N'^-1 r,   logdet = 1/2 sum_k ln(2 pi K_k),
        grad_I H = -PSF * (N'^-1 r)    (PSF * is self-adjoint: the PSF is even).

    sky, dirty [B, nx, ny]; K [B or 1, nx, ny]. Returns (H [B], logdet [B or 1], grad).
    """
    sky = np.asarray(sky, dtype=np.float64)
    dirty = np.asarray(dirty, dtype=np.float64)
    r = dirty - M.psf_apply(psf_img, sky)
    u = noise_inverse(r, K)
    H = 0.5 * np.einsum("bij,bij->b", r, u)
    logdet = 0.5 * np.sum(np.log(2.0 * np.pi * np.asarray(K).reshape(np.asarray(K).shape[0], -1)),
                          axis=1)
    grad = -M.psf_apply(psf_img, u)
    return H, logdet, grad
