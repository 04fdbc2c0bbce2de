// Pass operations of the noise model (Sec. 3.3.3), shared by noise.cu and noise_extra.cu; the
// passes and the kernel fit are described in noise.cu.
#pragma once
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
    if (t) block_sum_atomic(&value[blockIdx.y / nsky], acc);
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
  __device__ void finish(int, double acc) const { block_sum_atomic(&logdet[blockIdx.y], acc); }
};

template <int LEN>
static int run_nk1(const NK1Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, nimg, tw, s); }
template <int LEN>
static int run_nk2(const NK2Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, 1>(op, nimg, tw, s); }
template <int LEN>
static int run_nk3(const NK3Op& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, nimg, tw, s); }
template <int LEN>
static int run_nkf(const NKFOp& op, int nimg, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, nimg, tw, s); }

// the lengths of FR_NOISE_EXTRA_DISPATCH (noise_extra.cu)
bool noise_extra_len(int L);
int nk1_extra(int len, const NK1Op& op, int n, const float2* tw, cudaStream_t s);
int nk2_extra(int len, const NK2Op& op, int n, const float2* tw, cudaStream_t s);
int nk3_extra(int len, const NK3Op& op, int n, const float2* tw, cudaStream_t s);
int nkf_extra(int len, const NKFOp& op, int n, const float2* tw, cudaStream_t s);

}  // namespace fr
