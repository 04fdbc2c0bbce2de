/* fastresolve: GB300-native measurement operator of fast-resolve (arXiv 2406.09144).
 *
 * C ABI of libfastresolve.so. Every entry point is extern "C", takes plain pointers and sizes,
 * and returns 0 on success or a negative FR_E* code; fr_last_error() then gives a message
 * (thread-local). All compute runs in the library's own CUDA kernels for sm_103a; there is no
 * CPU fallback.
 *
 * Operators (paper sections and equations):
 *   R          Eq. (rime), Sec. 2: sky -> visibilities, scalar gains G = 1,
 *              V_k = sum_j I_j / n_j exp(-2 pi i (u_k l_j + v_k m_j + w_k (n_j - 1)))
 *   R^dag N^-1 Eq. (clean), Sec. 3.2: weighted back-projection (dirty image), N^-1 = weights
 *              (Sec. 3.1.2), the adjoint of R under the real inner product (the sky is real)
 *   PSF *      Sec. 3.3.2: R^dag N^-1 R ~ convolution with the PSF, evaluated exactly (linear,
 *              not circular) by zero padding to 2nx x 2ny
 *   likelihood Eq. (ham) expanded with Eq. (clean): L(s) = 1/2 s^T (PSF * s) - s^T d,
 *              grad = PSF * s - d; the exact variant uses R^dag N^-1 R (Algorithm 1 major cycle)
 *
 * Conventions:
 *   - sky images are float32 [nsky][nx][ny], row-major, y fastest; pixel (jx, jy) sits at
 *     l = (jx - nx/2) * pixsize_x, m = (jy - ny/2) * pixsize_y;
 *   - nsky = nchan (one image per channel) by default, nsky = 1 with FR_MFS (one image for all
 *     channels; R^dag sums channels);
 *   - visibilities are complex64 [nrow][nchan] (fr_cf32), weights float32 [nrow][nchan];
 *   - uvw are metres, freqs Hz; u, v, w in wavelengths are uvw * nu / c, c = 299792458 m/s,
 *     scaled in FP64.
 *
 * Ownership: fr_plan_create copies its host inputs; the plan owns all device-resident data
 * (sorted visibility coordinates, permutation, correction tables, PSF and its transfer
 * function) and per-stream workspaces. Every other pointer argument is a caller-owned DEVICE
 * buffer (e.g. torch.Tensor.data_ptr()), contiguous, in the layout stated; the library never
 * frees it. Host outputs are marked "host". Calls are asynchronous on `stream` (a cudaStream_t,
 * NULL = legacy default stream) unless they return host values, in which case they synchronise
 * that stream before returning. A plan is immutable after creation; calls on one plan from
 * different host threads must use different streams.
 */
#ifndef FASTRESOLVE_H
#define FASTRESOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fr_plan *fr_plan_t;
typedef struct {
  float re, im;
} fr_cf32;

/* return codes */
#define FR_OK 0
#define FR_EINVAL (-1)        /* bad argument: size, null pointer, NaN/Inf coordinate, uv outside the grid */
#define FR_ENOMEM (-2)        /* device or host allocation failed */
#define FR_ECUDA (-3)         /* a CUDA runtime/driver call failed */
#define FR_EUNSUPPORTED (-4)  /* size outside the supported range (see fr_plan_create) */
#define FR_ETIMEOUT (-5)      /* a bounded device-side wait gave up; the call's output is invalid */

/* plan flags */
#define FR_WTERM 1u          /* apply the w-term exp(-2 pi i w (n - 1)) of Eq. (rime) */
#define FR_NTERM 2u          /* apply the 1/n factor of Eq. (rime) */
#define FR_MFS 4u            /* one sky image for all channels (nsky = 1) */
#define FR_DROP_OOB 8u       /* drop visibilities whose kernel footprint leaves the grid instead of failing */
#define FR_NO_PSF 16u        /* skip building the PSF (fr_psf_apply / approximate likelihood unavailable) */
/* bitwise reproducible outputs: the gridders (R^dag, the PSF build, the exact likelihood and
 * major cycle) accumulate in 64-bit fixed point, whose integer sums do not depend on the order
 * of the atomic adds, and the expansion terms are added to the image one after the other.
 * Every contribution is rounded once to a multiple of 2^-61 M n (M the call's largest
 * contribution, n its visibility count): far below FP32 resolution. Slower gridding (fixed-point
 * shared memory holds fewer CTAs per SM); FP64 scalar outputs (likelihood values, norms) still
 * sum per-CTA partials in arrival order and may differ in the last bits. */
#define FR_DETERMINISTIC 32u

/* Build a plan (plan time, Sec. 3.3.4: done once per observation).
 *   uvw      host float64 [nrow][3] metres
 *   freqs    host float64 [nchan] Hz, all > 0
 *   weights  host float32 [nrow][nchan] (N^-1 as visibility weights, Sec. 3.1.2), >= 0;
 *            NULL means all ones; weight 0 marks flagged data
 *   nx, ny   image size; even, in [16, 4096]. The oversampled grid is the shortest FFT length
 *            of at least 2 nx (2 ny) of the form 2^k, 3 2^k or 5 2^k (sigma = 2 for sides of those
 *            forms, at most 2.56 otherwise); fr_plan_get_info reports it
 *   pixsize_x, pixsize_y  pixel size in radians (direction cosines), > 0
 *   eps      requested relative L2 accuracy of R and R^dag, in [1e-6, 1e-2]
 *   flags    FR_WTERM | FR_NTERM | FR_MFS | FR_DROP_OOB | FR_NO_PSF | FR_DETERMINISTIC
 *            (other bits: FR_EINVAL)
 *   stream   stream for the plan's device work; the call synchronises it before returning
 *   out      receives the plan handle
 * Errors: FR_EINVAL for bad sizes/pointers, non-finite uvw or freqs, negative weights, or a
 * visibility whose gridding-kernel footprint leaves the oversampled grid (|u| too close to
 * 1 / (2 pixsize_x)) unless FR_DROP_OOB; FR_EUNSUPPORTED for sizes outside the range above;
 * FR_ENOMEM, FR_ECUDA. On error *out is NULL. */
int fr_plan_create(const double *uvw, int64_t nrow, const double *freqs, int32_t nchan,
                   const float *weights, int32_t nx, int32_t ny, double pixsize_x,
                   double pixsize_y, double eps, uint32_t flags, void *stream, fr_plan_t *out);

/* R, Eq. (rime): sky [nsky][nx][ny] (device) -> vis [nrow][nchan] (device, overwritten). */
int fr_degrid(fr_plan_t plan, const float *sky, fr_cf32 *vis, void *stream);

/* N^-1 R: R of Eq. (rime) followed by the inverse noise covariance of Eq. (ham), i.e. every
 * visibility times its weight (the plan's weights; 1 without weights; dropped visibilities 0).
 * It is the adjoint of fr_grid with weights (R^dag N^-1 = (N^-1 R)^dag for the real sky): the
 * backward pass of a weighted gridding call. Layouts and errors as fr_degrid. */
int fr_degrid_weighted(fr_plan_t plan, const float *sky, fr_cf32 *vis, void *stream);

/* R^dag (N^-1 if apply_weights != 0), Eq. (clean): vis [nrow][nchan] (device) ->
 * dirty [nsky][nx][ny] (device, overwritten): D_j = Re sum_k w_k y_k exp(+2 pi i phase_kj) / n_j. */
int fr_grid(fr_plan_t plan, const fr_cf32 *vis, int32_t apply_weights, float *dirty, void *stream);

/* Dirty image I^D = R^dag N^-1 V (Algorithm 1, first step) and the PSF (Sec. 3.3.2).
 *   dirty    device [nsky][nx][ny] or NULL
 *   psf      device [nsky][2nx][2ny] or NULL; unnormalised PSF(a, b) = sum_k w_k
 *            cos(2 pi (u_k a dx + v_k b dy)) at w = 0, offset (a, b) stored at (a + nx, b + ny);
 *            row 0 and column 0 are zero (never used by the cropped convolution)
 *   psf_norm host [nsky] or NULL: sum of weights per image = PSF at offset 0 (FP64)
 * vis may be NULL when dirty is NULL. */
int fr_dirty_psf(fr_plan_t plan, const fr_cf32 *vis, float *dirty, float *psf, double *psf_norm,
                 void *stream);

/* PSF convolution (Sec. 3.3.2): out = P^dag FFT^-1[FFT[PSF] . FFT[P sky]], i.e. the linear
 * convolution out(p) = sum_q PSF_t(p - q) sky(q) cropped to the image, on the lx x ly padded
 * grid set by fr_psf_set_padding (default 2nx x 2ny: PSF_t = PSF, the exact convolution).
 *   sky, out  device [batch][nsky][nx][ny]; image b*nsky + s uses the PSF of image s.
 *   batch     >= 1 */
int fr_psf_apply(fr_plan_t plan, const float *sky, int32_t batch, float *out, void *stream);

/* Reduced padding (Sec. 3.3.2): the PSF convolution of fr_psf_apply, fr_likelihood_grad
 * (exact == 0), fr_fast_likelihood_grad and the serving path runs on an lx x ly zero-padded
 * grid with the PSF truncated to offsets |a| <= hx = min(lx - nx, nx - 1), |b| <= hy =
 * min(ly - ny, ny - 1) (sidelobes beyond them neglected):
 *   out(p) = sum_q PSF_t(p - q) sky(q),  PSF_t(a, b) = PSF(a, b) inside the window, else 0,
 * which the lx-periodic transforms compute exactly. Smaller lx, ly move fewer bytes and lose
 * the truncated sidelobes; lx >= 2nx - 1, ly >= 2ny - 1 keep the whole PSF.
 *   lx, ly  even, nx < lx <= max(2nx, default lx), likewise ly; each 2^k (32..16384), 3 2^k
 *           (48..6144) or 5 2^k (80..5120). The default (set at plan creation) is the shortest
 *           such length >= 2nx - 1 (2nx for sides of those forms): the whole PSF.
 * Rebuilds the plan's transfer function in place on `stream` and synchronises it: no PSF call
 * on this plan may be in flight on any stream, and CUDA graphs captured before keep the old
 * lengths (capture again). Errors: FR_EINVAL (range, parity, FR_NO_PSF plan), FR_EUNSUPPORTED
 * (a length of another form), FR_ENOMEM, FR_ECUDA; on error the previous padding stays. */
int fr_psf_set_padding(fr_plan_t plan, int32_t lx, int32_t ly, void *stream);

/* The current padded lengths (host outputs). FR_EINVAL for a FR_NO_PSF plan. */
int fr_psf_padding(fr_plan_t plan, int32_t *lx, int32_t *ly);

/* Likelihood value and gradient (Eq. ham with Eq. clean, constants dropped):
 *   L_b = 1/2 s_b^T (A s_b) - s_b^T d_b,  grad_b = A s_b - d_b
 * with A = PSF * (exact == 0, Sec. 3.3.2) or A = R^dag N^-1 R (exact != 0, Algorithm 1).
 *   sky, dirty, grad  device [batch][nsky][nx][ny]; grad may alias neither input
 *   value             host float64 [batch] (sum over the nsky images of element b); may be NULL
 * Reductions are FP64. Synchronises `stream` when value != NULL. */
int fr_likelihood_grad(fr_plan_t plan, const float *sky, const float *dirty, int32_t batch,
                       int32_t exact, float *grad, double *value, void *stream);

/* Major-cycle residual of Algorithm 1 and residual norms (FP64 reductions):
 *   resid = dirty - R^dag N^-1 R sky   (device [nsky][nx][ny], may be NULL)
 *   resid_norm2  host float64: sum of resid^2 over all pixels (may be NULL)
 *   vis, vis_chi2: if vis != NULL, vis_chi2 (host float64) = sum_k w_k |V_k - (R sky)_k|^2,
 *   the data term of Eq. (ham).
 * Synchronises `stream` when a host output is requested. */
int fr_major_cycle(fr_plan_t plan, const float *sky, const float *dirty, float *resid,
                   double *resid_norm2, const fr_cf32 *vis, double *vis_chi2, void *stream);

/* Noise model of the fast-resolve likelihood (Sec. 3.3.3, Eq. N_new). Fits, per image, the
 * transfer function K = exp(xi) + eps_noise of a periodic convolution on the nx x ny image that
 * stands in for N' = R^dag N^-1 R + eps_noise 1: xi minimises
 * || N'(I_delta) - FFT^-1[K . FFT(I_delta)] ||^2 with I_delta a unit point source in the centre
 * pixel (nx/2, ny/2), and N'(I_delta) is evaluated with the exact R and R^dag of the plan. The
 * minimiser is computed exactly: by Parseval the loss separates per frequency, and
 * K_k = max(Re(FFT(N' I_delta)_k conj(FFT(I_delta)_k)), eps_noise) (the bound eps_noise is the
 * limit xi -> -inf where the target is smaller). The kernel stays resident in the plan.
 *   eps_noise  > 0, the variance of the added white noise (Eq. N_new)
 *   logdet     host float64 [nsky] or NULL: 1/2 sum_k ln(2 pi K_k), the ln|2 pi N'| / 2 term of
 *              Eq. ham_new (constant in the sky)
 * The noise passes transform the unpadded image: nx and ny must each be 2^k (>= 32), 3 2^k
 * (>= 48), 5 2^k (>= 80) or c 2^k (a multiple of 16, >= 144) with c in {9, 15, 25, 45, 75,
 * 225}, which includes 3600 (FR_EUNSUPPORTED otherwise). Synchronises `stream`. */
int fr_noise_fit(fr_plan_t plan, double eps_noise, double *logdet, void *stream);

/* The fitted kernel K (not its inverse): device float32 [nsky][nx][ny] in numpy.fft.fft2 order
 * (kx, ky). FR_EINVAL before fr_noise_fit. */
int fr_noise_kernel(fr_plan_t plan, float *K, void *stream);

/* N'^-1 x ~ FFT^-1[K^-1 . FFT(x)] per image (periodic boundaries, Sec. 3.3.3).
 *   x, out  device float32 [batch][nsky][nx][ny]; image (b, k) uses the kernel of sky k.
 * FR_EINVAL before fr_noise_fit. */
int fr_noise_apply_inverse(fr_plan_t plan, const float *x, int32_t batch, float *out,
                           void *stream);

/* The fast-resolve likelihood, Eq. ham_new with R' = PSF * (Sec. 3.3.2) and N'^-1 from the
 * fitted kernel, for a batch of skies against their dirty images or major-cycle residuals d:
 *   r = d - PSF * sky,   value_b = 1/2 r_b^T N'^-1 r_b,   grad_b = -PSF * (N'^-1 r_b)
 * (the ln|2 pi N'| term is constant in the sky and returned by fr_noise_fit).
 *   sky, dirty, grad  device float32 [batch][nsky][nx][ny]; grad may alias neither input
 *   value      host float64 [batch] or NULL (synchronises `stream` when given)
 * FR_EINVAL before fr_noise_fit or for a plan created with FR_NO_PSF. */
int fr_fast_likelihood_grad(fr_plan_t plan, const float *sky, const float *dirty, int32_t batch,
                            float *grad, double *value, void *stream);

/* The same as fr_fast_likelihood_grad, and with ninv_resid non-NULL also N'^-1 r (device
 * float32 [batch][nsky][nx][ny], the vector the likelihood's gradient with respect to the dirty
 * image d is made of: dH/dd = N'^-1 r). ninv_resid may alias neither input nor grad. */
int fr_fast_likelihood_grad_resid(fr_plan_t plan, const float *sky, const float *dirty,
                                  int32_t batch, float *grad, float *ninv_resid, double *value,
                                  void *stream);

/* PSF convolutions of several plans in one launch per pass (serving: many jobs' minor-cycle
 * convolutions of Sec. 3.3.2 batched into shared launches). The plans must have PSFs and equal
 * nx, ny and PSF padding (fr_psf_padding); their images form one flat batch, and each image is
 * convolved with its own plan's PSF exactly as fr_psf_apply does it (same passes, same
 * arithmetic).
 *   plans    host array of nplans (1 <= nplans <= 16) plan handles
 *   skies    host array of device pointers, plan j's float32 [batches[j]][nsky_j][nx][ny]
 *   batches  host int32 [nplans], each >= 1
 *   outs     host array of device pointers, plan j's output, same layout as its sky
 *   scratch  device memory owned by the caller, 16-byte aligned, at least
 *            fr_psf_group_scratch_bytes bytes; the call allocates nothing
 * FR_EINVAL for mismatched plans, null pointers or a short or misaligned scratch. */
int fr_psf_group_scratch_bytes(const fr_plan_t *plans, int32_t nplans, const int32_t *batches,
                               size_t *bytes);
int fr_psf_apply_group(const fr_plan_t *plans, int32_t nplans, const float *const *skies,
                       const int32_t *batches, float *const *outs, void *scratch,
                       size_t scratch_bytes, void *stream);

/* Allocates the per-stream workspace of `plan` for calls on `stream` (fr_degrid, fr_grid,
 * fr_dirty_psf and the PSF convolutions of up to `batch` skies) without computing anything, so
 * that later calls on that stream allocate nothing (a server prepares a job this way before
 * capturing its calls in a CUDA graph). Optional: the calls allocate on first use otherwise. */
int fr_plan_prepare(fr_plan_t plan, int32_t batch, void *stream);

/* Allocation-free PSF convolution. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory, such as code embedded in an application that owns
 * the whole device-memory budget through its own pool, or code running where a cudaMalloc would
 * implicitly synchronise the device or is not allowed. It computes the same linear convolution
 * as fr_psf_apply, out_b(p) = sum_q psf(p - q) sky_b(q) cropped to the image, but takes the PSF
 * image itself instead of a plan and allocates nothing: every intermediate lives in one
 * file-scope device array of 32 MiB compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *   psf   device float32 [2nx][2ny], offset (a, b) stored at (a + nx, b + ny) as fr_dirty_psf
 *         writes it (row 0 and column 0 are not used)
 *   sky   device float32 [batch][nx][ny];  out: device float32 [batch][nx][ny]
 *   nx, ny powers of two in [16, 8192] with nx * ny <= 2^20 (FR_EINVAL with a message
 *         otherwise, before any work is queued)
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture. All calls share the one array and it keeps
 * the last call's contents; each call writes every intermediate before reading it. Calls that
 * overlap on the GPU (different streams, or different host threads) race on the array and must
 * be serialised by the caller. */
int fr_psf_convolve_noalloc(const float *psf, const float *sky, int32_t nx, int32_t ny,
                            int32_t batch, float *out, void *stream);

/* Plan parameters chosen at creation (for reports and tests). */
typedef struct {
  int32_t nx, ny, nsky, nchan;
  int64_t nrow, nvis;
  int32_t grid_nu, grid_nv;        /* oversampled grid (>= 2 nx, 2 ny; see fr_plan_create) */
  int32_t support;                 /* gridding kernel support W in cells */
  double beta;                     /* exponential-of-semicircle kernel shape */
  int32_t wplanes_total;           /* sum over images of the w-planes */
  int32_t wplanes_max;             /* most w-planes of any image */
  double dw;                       /* w-plane spacing in wavelengths (0 without FR_WTERM) */
  int64_t nvis_dropped;            /* visibilities dropped under FR_DROP_OOB */
  int64_t work_items;              /* (tile, plane) work items over all planes */
  uint32_t flags;
} fr_plan_info;
int fr_plan_get_info(fr_plan_t plan, fr_plan_info *info);

/* Device memory held by the plan: resident data and the largest per-stream workspace. */
int fr_plan_footprint(fr_plan_t plan, size_t *resident_bytes, size_t *workspace_bytes);

/* Synchronise `stream` and report a device-side failure recorded by earlier calls on it
 * (FR_ETIMEOUT after a bounded wait gave up), then clear it. */
int fr_plan_check(fr_plan_t plan, void *stream);

/* Release the plan and all its device memory. Synchronises the device. NULL is ignored. */
void fr_plan_destroy(fr_plan_t plan);

const char *fr_strerror(int code);
const char *fr_last_error(void);

/* Number of kernel launches made by this library on the calling thread since the last reset
 * (for launch accounting in benchmarks). */
uint64_t fr_launch_count(int reset);

/* Per-kernel-class launch timing for roofline reports (not part of the method). When enabled,
 * every kernel launch of the library is bracketed by CUDA events on its launching stream and
 * tagged with its algorithmic byte count (the bytes the operation must move at the API dtypes).
 * fr_profile_enable(1) clears the accumulators; fr_profile_read synchronises on the recorded
 * events and writes, for categories 0 .. ncat-1, the summed milliseconds, algorithmic bytes and
 * launch counts (any output may be NULL); it returns the number of categories. Categories:
 * 0 fft_rows, 1 fft_cols, 2 degrid, 3 grid, 4 psf_rows, 5 psf_cols, 6 vis_prep, 7 reduce;
 * fr_profile_category(c) gives the name. */
void fr_profile_enable(int on);
int fr_profile_read(double *ms, double *bytes, uint64_t *launches, int32_t ncat);
const char *fr_profile_category(int32_t cat);

/* Host-only check of the FFT passes' Stockham index and butterfly arithmetic: transforms
 * `batch` sequences of n complex values in place (interleaved float32 re, im) on the CPU
 * with the same stage code and radix schedule the kernels use. dir = -1 forward, +1 inverse
 * (unnormalised), on the schedule of 16 points per thread; dir = -2 / +2 the same on the
 * schedule of 32 points per thread (a radix-32 opening stage for powers of two >= 512).
 * Returns FR_EINVAL unless 2 <= n <= 16384 with n = 2^k 3^a 5^b. Test support; needs no GPU. */
int fr_selftest_fft_host(float *data, int32_t n, int32_t batch, int32_t dir);

/* Test support for the error path of the bounded device waits (no counterpart in the paper):
 * launches on `stream` one CTA that arms its mbarrier for a transfer exactly as the degridder
 * does but issues no copy, so its bounded wait gives up (after about 0.3 s); the CTA records
 * the timeout in the plan's status word and returns with no copy in flight. The next
 * fr_plan_check on that stream then returns FR_ETIMEOUT and clears the word. Nothing faults and
 * the context stays usable. */
int fr_selftest_wait_timeout(fr_plan_t plan, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FASTRESOLVE_H */
