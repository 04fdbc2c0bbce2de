// PSF convolution on the 2x padded grid (Sec. 3.3.2):
//   out = P^dag FFT^-1[ T . FFT[P s] ],  T = FFT[ifftshift(PSF)] / (4 nx ny)  (real: PSF even)
// in three passes over half spectra (the sky and the PSF are real), each reading contiguous
// sequences:
//   P1 (sky rows, length 2ny): two real rows per complex transform, zero padded from ny to 2ny;
//      both rows' half spectra (ny + 1 bins) are separated by Hermitian symmetry and stored
//      transposed, HT[img][q][jx];
//   P2 (HT rows, length 2nx): rows >= nx are zero padding; forward FFT, multiply by T (stored
//      transposed as TT[q][p]), inverse FFT, keep [0, nx) (the crop P^dag along x), stored
//      transposed back to H[img][jx][q];
//   P3 (H row pairs, length 2ny): Hermitian extension of two half spectra into one complex
//      inverse FFT, keep [0, ny) (the crop along y). In likelihood mode the epilogue forms
//      grad = conv - d and accumulates L = 1/2 s.conv - s.d in FP64 (Eq. ham with Eq. clean).
// The transfer function is built once per plan from the PSF image: P1 on the PSF rows, then a
// forward transform of the HT rows.
#include "fft_engine.cuh"

namespace fr {

struct P1Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  const float* src;  // real rows, row rho at src + rho * in_pitch
  int in_len, in_pitch;
  float2* ht;        // [img][nyh + 1][rows_img]
  int rows_img, nrows, nyh;
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
    const int rho = 2 * r;
    const int img = rho / rows_img, jx = rho - img * rows_img;
    float2* dst = ht + ((size_t)img * (nyh + 1) + k) * rows_img + jx;
    dst[0] = x1;
    dst[1] = x2;
    return 0.0;
  }
};

struct P2Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool TWO = true;
  const float2* ht;       // [img][nyh + 1][nx]
  float2* h;              // [img][nx][hp]
  int hp, nx, nyh, nsky;
  const float* transfer;  // [nsky][nyh + 1][2nx]
  __host__ __device__ int nseq() const { return nyh + 1; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int q, int i) const {
    if (i >= nx) return make_float2(0.f, 0.f);
    return ht[((size_t)blockIdx.y * (nyh + 1) + q) * nx + i];
  }
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2* s, int q0) const {
    const int nq = nyh + 1;
    const float* T = transfer + (size_t)(blockIdx.y % nsky) * nq * L;
    for (int idx = threadIdx.x; idx < B * L; idx += NT) {
      const int c = idx / L, p = idx % L;
      if (q0 + c < nq) {
        const float t = __ldg(&T[(size_t)(q0 + c) * L + p]);
        float2& z = s[c * LP + spad(p)];
        z.x *= t;
        z.y *= t;
      }
    }
  }
  __device__ double store(int q, int o, SeqView s) const {
    h[((size_t)blockIdx.y * nx + o) * hp + q] = s[o];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int o, SeqView s) const { return s[o]; }
  __device__ void store_group(int q0, int o, const float2* v, int n) const {
    store_run(h + ((size_t)blockIdx.y * nx + o) * hp + q0, v, n);
  }
};

struct P3Op : OpBase {
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
    const double c = (0.5 * (double)s0 * z.x - (double)s0 * d0) +
                     (0.5 * (double)s1 * z.y - (double)s1 * d1);
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

// forward transform of the PSF half spectra along x -> real transfer function TT[q][p]
struct TOp : OpBase {
  const float2* ht;  // [grp][nyh + 1][nx2]
  int nx2, nyh;
  float* transfer;   // [grp][nyh + 1][nx2]
  float scale;
  __host__ __device__ int nseq() const { return nyh + 1; }
  __host__ __device__ int nout() const { return nx2; }
  __device__ float2 load(int q, int i) const {
    return ht[((size_t)blockIdx.y * (nyh + 1) + q) * nx2 + i];
  }
  __device__ double store(int q, int p, SeqView s) const {
    // ifftshift by (nx2/2, nyh): multiply by (-1)^(p + q); the result is real (PSF even)
    const float sg = ((p + q) & 1) ? -scale : scale;
    transfer[((size_t)blockIdx.y * (nyh + 1) + q) * nx2 + p] = sg * s[p].x;
    return 0.0;
  }
};

template <int LG>
static int run_p1(const P1Op& op, const float2* tw, cudaStream_t s) {
  return launch_pass<LG, -1, -1>(op, 1, tw, s);
}
template <int LG>
static int run_p2(const P2Op& op, int nimg, const float2* tw, cudaStream_t s) {
  return launch_pass<LG, -1, 1>(op, nimg, tw, s);
}
template <int LG>
static int run_p3(const P3Op& op, const float2* tw, cudaStream_t s) {
  P3Op o = op;
  o.B = FftCfg<LG>::B;
  return launch_pass<LG, 1, 1>(o, 1, tw, s);
}
template <int LG>
static int run_t(const TOp& op, int nimg, const float2* tw, cudaStream_t s) {
  return launch_pass<LG, -1, -1>(op, nimg, tw, s);
}
static int p1(int lg, const P1Op& op, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p1, op, tw, s); }
static int p2(int lg, const P2Op& op, int n, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p2, op, n, tw, s); }
static int p3(int lg, const P3Op& op, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_p3, op, tw, s); }
static int pt(int lg, const TOp& op, int n, const float2* tw, cudaStream_t s) { FR_LOG2_DISPATCH(lg, run_t, op, n, tw, s); }

int psf_apply_passes(const PsfArgs& a, float2* h, float2* ht, const float2* tw_rows,
                     const float2* tw_cols, cudaStream_t s) {
  const int nrows = a.nimg * a.nx;
  const double px = (double)nrows * a.ny, hs = (double)nrows * (a.ny + 1);
  P1Op o1;
  o1.src = a.sky;
  o1.in_len = a.ny;
  o1.in_pitch = a.ny;
  o1.ht = ht;
  o1.rows_img = a.nx;
  o1.nrows = nrows;
  o1.nyh = a.ny;
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + hs * 8.0);
    FR_TRY(p1(ilog2(2 * a.ny), o1, tw_rows, s));
  }
  P2Op o2;
  o2.ht = ht;
  o2.h = h;
  o2.hp = a.hp;
  o2.nx = a.nx;
  o2.nyh = a.ny;
  o2.nsky = a.nsky;
  o2.transfer = a.transfer;
  {
    // half spectra in and out, transfer function (2nx x (ny+1) floats) once per image
    ProfScope ps(PC_PSF_COLS, s, hs * 16.0 + (double)a.nimg * 2 * a.nx * (a.ny + 1) * 4.0);
    FR_TRY(p2(ilog2(2 * a.nx), o2, a.nimg, tw_cols, s));
  }
  P3Op o3;
  o3.h = h;
  o3.hp = a.hp;
  o3.nyh = a.ny;
  o3.nrows = nrows;
  o3.out = a.out;
  o3.sky = a.sky;
  o3.dirty = a.dirty;
  o3.value = a.value;
  o3.nx = a.nx;
  o3.nsky = a.nsky;
  o3.B = 1;
  ProfScope ps(PC_PSF_ROWS, s, hs * 8.0 + px * (a.dirty ? 12.0 : 4.0));
  return p3(ilog2(2 * a.ny), o3, tw_rows, s);
}

int build_transfer(int nx, int ny, int nsky, const float* psf, float2* ht, float* transfer,
                   const float2* tw_rows, const float2* tw_cols, cudaStream_t s) {
  P1Op o1;
  o1.src = psf;
  o1.in_len = 2 * ny;
  o1.in_pitch = 2 * ny;
  o1.ht = ht;
  o1.rows_img = 2 * nx;
  o1.nrows = nsky * 2 * nx;
  o1.nyh = ny;
  FR_TRY(p1(ilog2(2 * ny), o1, tw_rows, s));
  TOp ot;
  ot.ht = ht;
  ot.nx2 = 2 * nx;
  ot.nyh = ny;
  ot.transfer = transfer;
  ot.scale = (float)(1.0 / (4.0 * nx * (double)ny));
  return pt(ilog2(2 * nx), ot, nsky, tw_cols, s);
}

}  // namespace fr
