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
#include "fft_engine.cuh"

namespace fr {

struct NK1Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  const float* x;  // [nimg][nx][ny]
  float2* ht;      // [nimg][ny][nx]
  int nx, ny;
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return ny; }
  __device__ float2 load(int jx, int i) const {
    return make_float2(__ldg(&x[((size_t)blockIdx.y * nx + jx) * ny + i]), 0.f);
  }
  __device__ double store(int jx, int ky, SeqView s) const {
    ht[((size_t)blockIdx.y * ny + ky) * nx + jx] = s[ky];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int ky, SeqView s) const { return s[ky]; }
  __device__ void store_group(int jx0, int ky, const float2* v, int n) const {
    store_run(ht + ((size_t)blockIdx.y * ny + ky) * nx + jx0, v, n);
  }
};

struct NK2Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool TWO = true;
  const float2* ht;   // [nimg][ny][nx]
  float2* h;          // [nimg][nx][ny]
  const float* kinv;  // [nsky][ny][nx]: 1 / K, transposed
  int nx, ny, nsky;
  __host__ __device__ int nseq() const { return ny; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int ky, int i) const {
    return ht[((size_t)blockIdx.y * ny + ky) * nx + i];
  }
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2* s, int q0) const {
    const float* KI = kinv + (size_t)(blockIdx.y % nsky) * ny * L;
    for (int idx = threadIdx.x; idx < B * L; idx += NT) {
      const int c = idx / L, kx = idx % L;
      if (q0 + c < ny) {
        const float k = __ldg(&KI[(size_t)(q0 + c) * L + kx]);
        float2& z = s[c * LP + spad(kx)];
        z.x *= k;
        z.y *= k;
      }
    }
  }
  __device__ double store(int ky, int jx, SeqView s) const {
    h[((size_t)blockIdx.y * nx + jx) * ny + ky] = s[jx];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int jx, SeqView s) const { return s[jx]; }
  __device__ void store_group(int ky0, int jx, const float2* v, int n) const {
    store_run(h + ((size_t)blockIdx.y * nx + jx) * ny + ky0, v, n);
  }
};

struct NK3Op : OpBase {
  const float2* h;  // [nimg][nx][ny]
  float* out;       // [nimg][nx][ny]
  const float* t;   // [nimg][nx][ny] for the value epilogue, or null
  double* value;    // [nimg / nsky]
  float scale, sgn;
  int nx, ny, nsky;
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return ny; }
  __device__ float2 load(int jx, int i) const {
    return h[((size_t)blockIdx.y * nx + jx) * ny + i];
  }
  __device__ double store(int jx, int jy, SeqView s) const {
    const size_t a = ((size_t)blockIdx.y * nx + jx) * ny + jy;
    const float u = s[jy].x * scale;
    out[a] = sgn * u;
    return t ? 0.5 * (double)__ldg(&t[a]) * (double)u : 0.0;
  }
  __device__ void finish(int, double acc) const {
    if (!t) return;
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      acc = lane < nw ? red[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) atomicAdd(&value[blockIdx.y / nsky], acc);
    }
  }
};

// forward transform of the HT rows of N'(I_delta) -> 1/K (transposed) and 1/2 sum ln(2 pi K)
struct NKFOp : OpBase {
  const float2* ht;  // [nsky][ny][nx]
  float* kinv;       // [nsky][ny][nx]
  double* logdet;    // [nsky]
  float eps;
  int nx, ny;
  __host__ __device__ int nseq() const { return ny; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int ky, int i) const {
    return ht[((size_t)blockIdx.y * ny + ky) * nx + i];
  }
  __device__ double store(int ky, int kx, SeqView s) const {
    // FFT(I_delta)_k = (-1)^(kx + ky) for the delta at (nx/2, ny/2)
    const float re = ((kx + ky) & 1) ? -s[kx].x : s[kx].x;
    const float K = fmaxf(re, eps);
    kinv[((size_t)blockIdx.y * ny + ky) * nx + kx] = 1.f / K;
    return 0.5 * log(2.0 * M_PI * (double)K);
  }
  __device__ void finish(int, double acc) const {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      acc = lane < nw ? red[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) atomicAdd(&logdet[blockIdx.y], acc);
    }
  }
};

template <int LEN>
static int run_nk1(const NK1Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, nimg, tw, s); }
template <int LEN>
static int run_nk2(const NK2Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, 1>(op, nimg, tw, s); }
template <int LEN>
static int run_nk3(const NK3Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, nimg, tw, s); }
template <int LEN>
static int run_nkf(const NKFOp& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, nimg, tw, s); }
static int nk1(int len, const NK1Op& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_nk1, op, n, tw, s); }
static int nk2(int len, const NK2Op& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_nk2, op, n, tw, s); }
static int nk3(int len, const NK3Op& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_nk3, op, n, tw, s); }
static int nkf(int len, const NKFOp& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_nkf, op, n, tw, s); }

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
