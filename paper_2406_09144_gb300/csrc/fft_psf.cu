// PSF convolution on the 2x padded grid (Sec. 3.3.2):
//   out = P^dag FFT^-1[ T . FFT[P s] ],  T = FFT[ifftshift(PSF)] / (4 nx ny)  (real: PSF even)
// in three passes over a half spectrum (the sky and the PSF are real):
//   P1 (rows, length 2ny): two real rows per complex transform, zero padded from ny to 2ny;
//      the half spectra (ny + 1 bins) of both rows are separated by Hermitian symmetry;
//   P2 (columns, length 2nx): rows >= nx are zero padding; forward FFT, multiply by T, inverse
//      FFT, keep rows [0, nx) (the crop P^dag along x);
//   P3 (rows, length 2ny): Hermitian extension of two half spectra into one complex inverse
//      FFT, keep columns [0, ny) (the crop along y). In likelihood mode the epilogue forms
//      grad = conv - d and accumulates L = 1/2 s.conv - s.d in FP64 (Eq. ham with Eq. clean).
// The transfer function is built the same way from the PSF image (rows, then a forward
// column pass), once per plan.
#include "fft_engine.cuh"

namespace fr {

struct P1Op {
  const float* src;  // real rows, row rho at src + rho * in_pitch
  int in_len, in_pitch;
  float2* h;         // half spectra, row rho at h + rho * hp
  int hp, nrows, nyh;
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return nyh + 1; }
  __device__ float2 load(int r, int i) const {
    if (i >= in_len) return make_float2(0.f, 0.f);
    const size_t a = (size_t)(2 * r) * in_pitch + i;
    return make_float2(__ldg(&src[a]), __ldg(&src[a + in_pitch]));
  }
  __device__ double store(int r, int k, SeqView v) const {
    const int L = 2 * nyh;
    const float2 z = v[k], zm = v[(L - k) & (L - 1)];
    const float2 x1 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    const float2 x2 = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    h[(size_t)(2 * r) * hp + k] = x1;
    h[(size_t)(2 * r + 1) * hp + k] = x2;
    return 0.0;
  }
  __device__ void finish(int, double) const {}
};

struct P2Op {
  float2* h;
  int hp, nx, nyh, nsky;
  const float* transfer;  // [nsky][2nx][nyh + 1]
  __host__ __device__ int ncol() const { return nyh + 1; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int i, int q) const {
    if (i >= nx) return make_float2(0.f, 0.f);
    return h[((size_t)blockIdx.y * nx + i) * hp + q];
  }
  template <int B, int NT, int L>
  __device__ void after_load(int) const {}
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2* s, int col0) const {
    const int nq = nyh + 1;
    const float* T = transfer + (size_t)(blockIdx.y % nsky) * (size_t)(2 * nx) * nq;
    for (int idx = threadIdx.x; idx < B * L; idx += NT) {
      const int p = idx / B, c = idx % B;
      const int q = col0 + c;
      if (q < nq) {
        const float t = __ldg(&T[(size_t)p * nq + q]);
        float2& z = s[c * LP + spad(p)];
        z.x *= t;
        z.y *= t;
      }
    }
  }
  __device__ void store(int o, int q, SeqView s) const {
    h[((size_t)blockIdx.y * nx + o) * hp + q] = s[o];
  }
};

struct P3Op {
  const float2* h;
  int hp, nyh, nrows;
  float* out;          // [nrows][nyh]: the convolution, or grad in likelihood mode
  const float* sky;    // likelihood mode only
  const float* dirty;  // likelihood mode only (null: plain convolution)
  double* value;       // [nrows / (nx * nsky)]
  int nx, nsky, B;     // B: row pairs per CTA of this instantiation
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return nyh; }
  __device__ float2 load(int r, int k) const {
    const int L = 2 * nyh;
    float2 x1, x2;
    const float2* h0 = h + (size_t)(2 * r) * hp;
    const float2* h1 = h0 + hp;
    if (k <= nyh) {
      x1 = h0[k];
      x2 = h1[k];
      if (k == 0 || k == nyh) {
        x1.y = 0.f;
        x2.y = 0.f;
      }
    } else {
      const int km = L - k;
      x1 = cconj(h0[km]);
      x2 = cconj(h1[km]);
    }
    return make_float2(x1.x - x2.y, x1.y + x2.x);
  }
  __device__ bool single_element(int seq0) const {
    const int rho0 = 2 * seq0;
    const int rho1 = min(2 * (seq0 + B), nrows) - 1;
    const int per = nx * nsky;
    return rho0 / per == rho1 / per;
  }
  __device__ double store(int r, int n, SeqView v) const {
    const float2 z = v[n];
    const size_t a0 = (size_t)(2 * r) * nyh + n, a1 = a0 + nyh;
    if (!dirty) {
      out[a0] = z.x;
      out[a1] = z.y;
      return 0.0;
    }
    const float s0 = __ldg(&sky[a0]), s1 = __ldg(&sky[a1]);
    const float d0 = __ldg(&dirty[a0]), d1 = __ldg(&dirty[a1]);
    out[a0] = z.x - d0;
    out[a1] = z.y - d1;
    const double c = (0.5 * (double)s0 * z.x - (double)s0 * d0) + (0.5 * (double)s1 * z.y - (double)s1 * d1);
    if (single_element(blockIdx.x * B)) return c;
    atomicAdd(&value[(2 * r) / (nx * nsky)], c);
    return 0.0;
  }
  __device__ void finish(int seq0, double acc) const {
    if (!dirty || !single_element(seq0)) return;
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      acc = lane < nw ? red[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) atomicAdd(&value[(2 * seq0) / (nx * nsky)], acc);
    }
  }
};

// forward column transform of the PSF half spectra -> real transfer function
struct TOp {
  const float2* h;
  int hp, nx2, nyh;
  float* transfer;
  float scale;
  __host__ __device__ int ncol() const { return nyh + 1; }
  __host__ __device__ int nout() const { return nx2; }
  __device__ float2 load(int i, int q) const { return h[((size_t)blockIdx.y * nx2 + i) * hp + q]; }
  template <int B, int NT, int L>
  __device__ void after_load(int) const {}
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2*, int) const {}
  __device__ void store(int p, int q, SeqView s) const {
    // ifftshift by nx2/2, ny: multiply by (-1)^(p + q); the result is real (PSF even)
    const float sg = ((p + q) & 1) ? -scale : scale;
    transfer[((size_t)blockIdx.y * nx2 + p) * (nyh + 1) + q] = sg * s[p].x;
  }
};

template <int LG>
static int run_p1(const P1Op& op, const float2* tw, cudaStream_t s) {
  return launch_rows<LG, -1>(op, tw, s);
}
template <int LG>
static int run_p2(const P2Op& op, int nimg, const float2* tw, cudaStream_t s) {
  ColOp<LG, P2Op> c;
  static_cast<P2Op&>(c) = op;
  return launch_cols<LG, -1, 1, true>(c, nimg, tw, s);
}
template <int LG>
static int run_p3(const P3Op& op, const float2* tw, cudaStream_t s) {
  P3Op o = op;
  o.B = FftCfg<LG>::B;
  return launch_rows<LG, 1>(o, tw, s);
}
template <int LG>
static int run_t(const TOp& op, int nimg, const float2* tw, cudaStream_t s) {
  ColOp<LG, TOp> c;
  static_cast<TOp&>(c) = op;
  return launch_cols<LG, -1, -1, false>(c, nimg, tw, s);
}
static int p1(int lg, const P1Op& op, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p1, op, tw, s); }
static int p2(int lg, const P2Op& op, int n, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p2, op, n, tw, s); }
static int p3(int lg, const P3Op& op, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p3, op, tw, s); }
static int pt(int lg, const TOp& op, int n, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_t, op, n, tw, s); }

int psf_apply_passes(const PsfArgs& a, float2* h, const float2* tw_rows, const float2* tw_cols,
                     cudaStream_t s) {
  const int nrows = a.nimg * a.nx;
  const double px = (double)nrows * a.ny, hs = (double)nrows * (a.ny + 1);
  P1Op o1{a.sky, a.ny, a.ny, h, a.hp, nrows, a.ny};
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + hs * 8.0);
    FR_TRY(p1(ilog2(2 * a.ny), o1, tw_rows, s));
  }
  P2Op o2{h, a.hp, a.nx, a.ny, a.nsky, a.transfer};
  {
    // half spectra in and out, transfer function (2nx x (ny+1) floats) once per image
    ProfScope ps(PC_PSF_COLS, s, hs * 16.0 + (double)a.nimg * 2 * a.nx * (a.ny + 1) * 4.0);
    FR_TRY(p2(ilog2(2 * a.nx), o2, a.nimg, tw_cols, s));
  }
  P3Op o3{h, a.hp, a.ny, nrows, a.out, a.sky, a.dirty, a.value, a.nx, a.nsky, 1};
  ProfScope ps(PC_PSF_ROWS, s, hs * 8.0 + px * (a.dirty ? 12.0 : 4.0));
  return p3(ilog2(2 * a.ny), o3, tw_rows, s);
}

int build_transfer(int nx, int ny, int nsky, const float* psf, float2* h, int hp, float* transfer,
                   const float2* tw_rows, const float2* tw_cols, cudaStream_t s) {
  const int nrows = nsky * 2 * nx;
  P1Op o1{psf, 2 * ny, 2 * ny, h, hp, nrows, ny};
  FR_TRY(p1(ilog2(2 * ny), o1, tw_rows, s));
  TOp ot{h, hp, 2 * nx, ny, transfer, (float)(1.0 / (4.0 * nx * (double)ny))};
  return pt(ilog2(2 * nx), ot, nsky, tw_cols, s);
}

}  // namespace fr
