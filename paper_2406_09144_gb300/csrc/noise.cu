// Fast-resolve noise model (Sec. 3.3.3) and likelihood (Eq. ham_new, Sec. 3.3.1):
//   N'(x) ~ FFT^-1[K . FFT(x)] on the periodic nx x ny image, K = exp(xi) + eps > 0 real,
//   N'^-1(x) ~ FFT^-1[K^-1 . FFT(x)].
// Three passes per image (complex transforms of the real image):
//   NK1 (image rows, length ny, forward): x[jx][.] -> HT[ky][jx] (transposed store);
//   NK2 (HT rows, length nx): forward, multiply by 1/K (stored KT[ky][kx]), inverse, transposed
//       back to H[jx][ky];
//   NK3 (H rows, length ny, inverse): out = sgn Re(.)/(nx ny); optional FP64 epilogue
//       value += 1/2 sgn t . out per batch element (the quadratic form of Eq. ham_new).
// The kernel fit: K minimises || N'(I_delta) - FFT^-1[K . FFT(I_delta)] ||^2 over K > eps; by
// Parseval the loss separates per frequency, |z_k - K_k|^2 with z_k = FFT(N' I_delta)_k
// conj(FFT(I_delta)_k) (|FFT(I_delta)_k| = 1 for the centre delta), so the minimiser is
// K_k = Re z_k where that exceeds eps and the limit K_k -> eps elsewhere. NKF (HT rows, forward)
// forms it from the forward transform of N'(I_delta) and accumulates 1/2 sum ln(2 pi K).
#include "noise_ops.cuh"

namespace fr {

static int nk1(int len, const NK1Op& op, int n, const float2* tw, cudaStream_t s) {
  if (noise_extra_len(len)) return nk1_extra(len, op, n, tw, s);
  FR_LEN_DISPATCH(len, run_nk1, op, n, tw, s);
}
static int nk2(int len, const NK2Op& op, int n, const float2* tw, cudaStream_t s) {
  if (noise_extra_len(len)) return nk2_extra(len, op, n, tw, s);
  FR_LEN_DISPATCH(len, run_nk2, op, n, tw, s);
}
static int nk3(int len, const NK3Op& op, int n, const float2* tw, cudaStream_t s) {
  if (noise_extra_len(len)) return nk3_extra(len, op, n, tw, s);
  FR_LEN_DISPATCH(len, run_nk3, op, n, tw, s);
}
static int nkf(int len, const NKFOp& op, int n, const float2* tw, cudaStream_t s) {
  if (noise_extra_len(len)) return nkf_extra(len, op, n, tw, s);
  FR_LEN_DISPATCH(len, run_nkf, op, n, tw, s);
}

bool noise_len_supported(int L) { return fft_len_supported(L) || noise_extra_len(L); }

int noise_kernel_passes(const float* n_delta, int nx, int ny, int nsky, float eps, float2* ht,
                        float* kinv, double* logdet, const float2* tw_y, const float2* tw_x,
                        cudaStream_t s) {
  const double px = (double)nsky * nx * ny;
  NK1Op o1;
  o1.x = n_delta;
  o1.ht = ht;
  o1.nx = nx;
  o1.ny = ny;
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + px * 8.0);
    FR_TRY(nk1(ny, o1, nsky, tw_y, s));
  }
  NKFOp of;
  of.ht = ht;
  of.kinv = kinv;
  of.logdet = logdet;
  of.eps = eps;
  of.nx = nx;
  of.ny = ny;
  ProfScope ps(PC_PSF_COLS, s, px * 8.0 + px * 4.0);
  return nkf(nx, of, nsky, tw_x, s);
}

int noise_inverse_passes(const float* x, int nx, int ny, int nimg, int nsky, const float* kinv,
                         float2* ht, float2* h, float* out, float sgn, const float* t,
                         double* value, const float2* tw_y, const float2* tw_x, cudaStream_t s) {
  const double px = (double)nimg * nx * ny;
  NK1Op o1;
  o1.x = x;
  o1.ht = ht;
  o1.nx = nx;
  o1.ny = ny;
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + px * 8.0);
    FR_TRY(nk1(ny, o1, nimg, tw_y, s));
  }
  NK2Op o2;
  o2.ht = ht;
  o2.h = h;
  o2.kinv = kinv;
  o2.nx = nx;
  o2.ny = ny;
  o2.nsky = nsky;
  {
    ProfScope ps(PC_PSF_COLS, s, px * 16.0 + (double)nsky * nx * ny * 4.0);
    FR_TRY(nk2(nx, o2, nimg, tw_x, s));
  }
  NK3Op o3;
  o3.h = h;
  o3.out = out;
  o3.t = t;
  o3.value = value;
  o3.scale = 1.f / ((float)nx * (float)ny);
  o3.sgn = sgn;
  o3.nx = nx;
  o3.ny = ny;
  o3.nsky = nsky;
  ProfScope ps(PC_PSF_ROWS, s, px * 8.0 + px * 4.0 + (t ? px * 4.0 : 0.0));
  return nk3(ny, o3, nimg, tw_y, s);
}

}  // namespace fr
