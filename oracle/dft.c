/* Direct-sum FP64 evaluation of R, R^dagger and the PSF at selected outputs.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load this library; the CUDA product path never does.
 *
 * These are the same definitions as oracle/measurement.py, written as plain loops so that
 * sampled checks at full problem size (one O(N) or O(M) sum per output) finish in seconds on
 * the host cores. One OpenMP thread per selected output; no blocking, no recurrences, no FFT.
 *
 *   R       (Eq. rime, G = 1):  V_k = sum_j I_j / n_j exp(-2 pi i (u l + v m + w (n - 1)))
 *   R^dag N^-1 (Eq. clean):     D_j = Re sum_k y_k exp(+2 pi i (u l + v m + w (n - 1))) / n_j
 *   PSF (Sec. 3.2, 3.3.2):      P(a, b) = sum_k w_k cos(2 pi (u a dl + v b dm))
 *
 * u, v, w are given in wavelengths ([nrow][nchan], row-major), already scaled by nu / c.
 * Pixel (jx, jy) sits at l = (jx - nx/2) dl, m = (jy - ny/2) dm (integer division).
 */
#include <math.h>
#include <stdint.h>

static const double TWO_PI = 6.283185307179586476925286766559;

/* exp(-2 pi i phase) with phase in cycles; the integer part is removed first so that sin/cos
 * see an argument in [-pi, pi]. */
static inline void cis_neg(double phase, double *re, double *im) {
    double f = phase - nearbyint(phase);
    *re = cos(TWO_PI * f);
    *im = -sin(TWO_PI * f);
}

static inline void pixel_terms(int64_t jx, int64_t jy, int64_t nx, int64_t ny, double dl, double dm,
                               int wterm, int nterm, double *l, double *m, double *t, double *amp) {
    *l = (double)(jx - nx / 2) * dl;
    *m = (double)(jy - ny / 2) * dm;
    double r2 = (*l) * (*l) + (*m) * (*m);
    if (r2 >= 1.0) { *t = 0.0; *amp = 0.0; return; }
    double n = sqrt(1.0 - r2);
    *t = wterm ? (n - 1.0) : 0.0;
    *amp = nterm ? 1.0 / n : 1.0;
}

/* R at selected visibilities (sel_row[i], sel_chan[i]) -> out[2*i] (re), out[2*i+1] (im).
 * sky is [nsky][nx][ny]; nsky == 1 uses image 0 for every channel, else image = channel. */
void or_degrid(const double *sky, int64_t nsky, int64_t nx, int64_t ny, double dl, double dm,
               const double *u, const double *v, const double *w, int64_t nchan,
               const int64_t *sel_row, const int64_t *sel_chan, int64_t nsel,
               int wterm, int nterm, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nsel; ++i) {
        int64_t k = sel_row[i] * nchan + sel_chan[i];
        const double *img = sky + (nsky == 1 ? 0 : sel_chan[i]) * nx * ny;
        double uk = u[k], vk = v[k], wk = w[k];
        double sre = 0.0, sim = 0.0;
        for (int64_t jx = 0; jx < nx; ++jx) {
            for (int64_t jy = 0; jy < ny; ++jy) {
                double I = img[jx * ny + jy];
                if (I == 0.0) continue;
                double l, m, t, amp;
                pixel_terms(jx, jy, nx, ny, dl, dm, wterm, nterm, &l, &m, &t, &amp);
                double cr, ci;
                cis_neg(uk * l + vk * m + wk * t, &cr, &ci);
                sre += I * amp * cr;
                sim += I * amp * ci;
            }
        }
        out[2 * i] = sre;
        out[2 * i + 1] = sim;
    }
}

/* R^dagger of the (already weighted) visibilities y at selected pixels.
 * Output i is image sel_img[i] (a channel when nsky == nchan; 0 sums all channels when
 * nsky == 1), pixel sel_pix[i] = jx * ny + jy. */
void or_grid(const double *yre, const double *yim, int64_t nrow, int64_t nchan, int64_t nsky,
             int64_t nx, int64_t ny, double dl, double dm,
             const double *u, const double *v, const double *w,
             const int64_t *sel_img, const int64_t *sel_pix, int64_t nsel,
             int wterm, int nterm, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nsel; ++i) {
        int64_t jx = sel_pix[i] / ny, jy = sel_pix[i] % ny;
        double l, m, t, amp;
        pixel_terms(jx, jy, nx, ny, dl, dm, wterm, nterm, &l, &m, &t, &amp);
        int64_t c0 = (nsky == 1) ? 0 : sel_img[i];
        int64_t c1 = (nsky == 1) ? nchan : sel_img[i] + 1;
        double acc = 0.0;
        for (int64_t r = 0; r < nrow; ++r) {
            for (int64_t c = c0; c < c1; ++c) {
                int64_t k = r * nchan + c;
                double cr, ci;
                cis_neg(u[k] * l + v[k] * m + w[k] * t, &cr, &ci);
                /* Re(y * exp(+2 pi i phase)) with exp(+..) = conj(exp(-..)) = (cr, -ci) */
                acc += yre[k] * cr + yim[k] * ci;
            }
        }
        out[i] = acc * amp;
    }
}

/* PSF at selected offsets (sel_a[i], sel_b[i]) in pixels, for image sel_img[i] (as in or_grid).
 * wt is [nrow][nchan]. */
void or_psf(const double *wt, int64_t nrow, int64_t nchan, int64_t nsky, double dl, double dm,
            const double *u, const double *v,
            const int64_t *sel_img, const int64_t *sel_a, const int64_t *sel_b, int64_t nsel,
            double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nsel; ++i) {
        double da = (double)sel_a[i] * dl, db = (double)sel_b[i] * dm;
        int64_t c0 = (nsky == 1) ? 0 : sel_img[i];
        int64_t c1 = (nsky == 1) ? nchan : sel_img[i] + 1;
        double acc = 0.0;
        for (int64_t r = 0; r < nrow; ++r) {
            for (int64_t c = c0; c < c1; ++c) {
                int64_t k = r * nchan + c;
                double cr, ci;
                cis_neg(u[k] * da + v[k] * db, &cr, &ci);
                acc += wt[k] * cr;
            }
        }
        out[i] = acc;
    }
}
