// PSF convolution on a zero-padded periodic grid of lx x ly (Sec. 3.3.2):
//   out = P^dag FFT^-1[ T . FFT[P s] ],  T = FFT[K] / (lx ly)  (real: K even)
// K is the periodic kernel image: PSF(a, b) at (a mod lx, b mod ly) for |a| <= hx, |b| <= hy,
// zero elsewhere, hx = min(lx - nx, nx - 1) (same for y). With nx < lx <= 2nx the circular
// convolution of size lx reproduces the linear convolution with that kernel on the nx outputs
// exactly (an offset d of the cropped product has |d| <= nx - 1, and d and d - lx are never both
// inside [-hx, hx] when lx >= nx + hx). lx = 2nx, ly = 2ny keep the whole PSF (exact R' ~
// PSF *); shorter lengths truncate the PSF sidelobes beyond hx, hy and cut the transform sizes
// (the reduced padding of Sec. 3.3.2). Three passes over half spectra (the sky and the PSF are
// real), each reading contiguous sequences:
//   P1 (sky rows, length ly): two real rows per complex transform, zero padded from ny to ly;
//      both rows' half spectra (nh + 1 bins, nh = ly / 2) are separated by Hermitian symmetry
//      and stored transposed, HT[img][q][jx];
//   P2 (HT rows, length lx): rows >= nx are zero padding; forward FFT, multiply by T (stored
//      transposed as TT[q][p]), inverse FFT, keep [0, nx) (the crop P^dag along x), stored
//      transposed back to H[img][jx][q];
//   P3 (H row pairs, length ly): Hermitian extension of two half spectra into one complex
//      inverse FFT, keep [0, ny) (the crop along y). In likelihood mode the epilogue forms
//      grad = conv - d and accumulates L = 1/2 s.conv - s.d in FP64 (Eq. ham with Eq. clean).
// The transfer function is built from the PSF image: P1 on the rows of K (gathered from the
// PSF image on the fly), then a forward transform of the HT rows.
#include <algorithm>

#include "fft_engine.cuh"

namespace fr {

struct P1Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  const float* src;  // real rows, row rho at src + rho * in_pitch
  int in_len, in_pitch;
  float2* ht;        // [img][nh + 1][rows_img]
  int rows_img, nrows, nh;
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return nh + 1; }
  __device__ float2 load(int r, int i) const {
    if (i >= in_len) return make_float2(0.f, 0.f);
    const size_t a = (size_t)(2 * r) * in_pitch + i;
    return make_float2(__ldg(&src[a]), __ldg(&src[a + in_pitch]));
  }
  __device__ double store(int r, int k, SeqView v) const {
    const float2 z = v[k], zm = v[k == 0 ? 0 : 2 * nh - k];
    const float2 x1 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    const float2 x2 = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    const int rho = 2 * r;
    const int img = rho / rows_img, jx = rho - img * rows_img;
    float2* dst = ht + ((size_t)img * (nh + 1) + k) * rows_img + jx;
    dst[0] = x1;
    dst[1] = x2;
    return 0.0;
  }
};

// P1 on the rows of the periodic kernel image K (rows_img = lx, rows of length ly), read from
// the PSF image [grp][2nx][2ny] (origin at (nx, ny)) without materialising K
struct PK1Op : P1Op {
  int nx, ny, lx, ly, hx, hy;
  __device__ float at(int rho, int iy) const {
    const int g = rho / lx, ix = rho - g * lx;
    const int a = ix <= hx ? ix : ix - lx;
    const int b = iy <= hy ? iy : iy - ly;
    if (a < -hx || b < -hy) return 0.f;
    return __ldg(&src[((size_t)g * 2 * nx + nx + a) * (2 * ny) + ny + b]);
  }
  __device__ float2 load(int r, int i) const { return make_float2(at(2 * r, i), at(2 * r + 1, i)); }
};

struct P2Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool TWO = true;
  const float2* ht;       // [img][nh + 1][nx]
  float2* h;              // [img][nx][hp]
  int hp, nx, nh, nsky;
  const float* transfer;  // [nsky][nh + 1][lx]
  __host__ __device__ int nseq() const { return nh + 1; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int q, int i) const {
    if (i >= nx) return make_float2(0.f, 0.f);
    return ht[((size_t)blockIdx.y * (nh + 1) + q) * nx + i];
  }
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2* s, int q0) const {
    const int nq = nh + 1;
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
  int hp, nh, ny, nrows;
  float* out;          // [nrows][ny]: the convolution, or grad in likelihood mode
  const float* sky;    // likelihood mode only
  const float* dirty;  // likelihood mode only (null: plain convolution)
  double* value;       // [nrows / (nx * nsky)]
  int nx, nsky, B;     // B: row pairs per CTA of this instantiation
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return ny; }
  __device__ float2 load(int r, int k) const {
    float2 x1, x2;
    const float2* h0 = h + (size_t)(2 * r) * hp;
    const float2* h1 = h0 + hp;
    if (k <= nh) {
      x1 = h0[k];
      x2 = h1[k];
      if (k == 0 || k == nh) {
        x1.y = 0.f;
        x2.y = 0.f;
      }
    } else {
      const int km = 2 * nh - k;
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
  __device__ double store(int r, int n, SeqView v) const { return out_at(r, n, v[n]); }
  static constexpr bool DIRECT = true;  // outputs [0, ny) of the transform: the crop
  __device__ double direct(int r, int i, float2 z) const { return i < ny ? out_at(r, i, z) : 0.0; }
  __device__ double out_at(int r, int n, float2 z) const {
    const size_t a0 = (size_t)(2 * r) * ny + n, a1 = a0 + ny;
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

// forward transform of the kernel half spectra along x -> real transfer function TT[q][p]
struct TOp : OpBase {
  const float2* ht;  // [grp][nh + 1][lx]
  int lx, nh;
  float* transfer;   // [grp][nh + 1][lx]
  float scale;
  __host__ __device__ int nseq() const { return nh + 1; }
  __host__ __device__ int nout() const { return lx; }
  __device__ float2 load(int q, int i) const {
    return ht[((size_t)blockIdx.y * (nh + 1) + q) * lx + i];
  }
  __device__ double store(int q, int p, SeqView s) const {
    // K is even, so its transform is real: keep the real part
    transfer[((size_t)blockIdx.y * (nh + 1) + q) * lx + p] = scale * s[p].x;
    return 0.0;
  }
};

template <int LEN>
static int run_p1(const P1Op& op, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, -1>(op, 1, tw, s);
}
template <int LEN>
static int run_pk1(const PK1Op& op, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, -1>(op, 1, tw, s);
}
template <int LEN>
static int run_p2(const P2Op& op, int nimg, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, 1>(op, nimg, tw, s);
}
template <int LEN>
static int run_p3(const P3Op& op, const float2* tw, cudaStream_t s) {
  P3Op o = op;
  o.B = FftCfg<LEN>::B;
  return launch_pass<LEN, 1, 1>(o, 1, tw, s);
}
template <int LEN>
static int run_t(const TOp& op, int nimg, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, -1>(op, nimg, tw, s);
}
static int p1(int len, const P1Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p1, op, tw, s); }
static int pk1(int len, const PK1Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_pk1, op, tw, s); }
static int p2(int len, const P2Op& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p2, op, n, tw, s); }
static int p3(int len, const P3Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p3, op, tw, s); }
static int pt(int len, const TOp& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_t, op, n, tw, s); }

bool fft_len_supported(int L) {
  if (L < 32 || L > 16384) return false;
  const int c = odd_part(L);
  if (c == 1) return true;
  if (c == 3) return L >= 48 && L <= 6144;
  if (c == 5) return L >= 80 && L <= 5120;
  return false;
}

int fft_len_at_least(int m) {
  int best = 16384;
  for (int c : {1, 3, 5})
    for (int L = 16 * c; L <= 16384; L *= 2)
      if (L >= m && L < best && fft_len_supported(L)) best = L;
  return best;
}

int psf_apply_passes(const PsfArgs& a, float2* h, float2* ht, const float2* tw_rows,
                     const float2* tw_cols, cudaStream_t s) {
  const int nrows = a.nimg * a.nx, nh = a.ly / 2;
  const double px = (double)nrows * a.ny, hs = (double)nrows * (nh + 1);
  P1Op o1;
  o1.src = a.sky;
  o1.in_len = a.ny;
  o1.in_pitch = a.ny;
  o1.ht = ht;
  o1.rows_img = a.nx;
  o1.nrows = nrows;
  o1.nh = nh;
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + hs * 8.0);
    FR_TRY(p1(a.ly, o1, tw_rows, s));
  }
  P2Op o2;
  o2.ht = ht;
  o2.h = h;
  o2.hp = a.hp;
  o2.nx = a.nx;
  o2.nh = nh;
  o2.nsky = a.nsky;
  o2.transfer = a.transfer;
  {
    // half spectra in and out, transfer function (lx x (nh + 1) floats) once per image
    ProfScope ps(PC_PSF_COLS, s, hs * 16.0 + (double)a.nimg * a.lx * (nh + 1) * 4.0);
    FR_TRY(p2(a.lx, o2, a.nimg, tw_cols, s));
  }
  P3Op o3;
  o3.h = h;
  o3.hp = a.hp;
  o3.nh = nh;
  o3.ny = a.ny;
  o3.nrows = nrows;
  o3.out = a.out;
  o3.sky = a.sky;
  o3.dirty = a.dirty;
  o3.value = a.value;
  o3.nx = a.nx;
  o3.nsky = a.nsky;
  o3.B = 1;
  ProfScope ps(PC_PSF_ROWS, s, hs * 8.0 + px * (a.dirty ? 12.0 : 4.0));
  return p3(a.ly, o3, tw_rows, s);
}

int build_transfer(int nx, int ny, int nsky, const float* psf, int lx, int ly, float2* ht,
                   float* transfer, const float2* tw_rows, const float2* tw_cols, cudaStream_t s) {
  PK1Op o1;
  o1.src = psf;
  o1.in_len = ly;
  o1.in_pitch = 0;  // unused: rows come from at()
  o1.ht = ht;
  o1.rows_img = lx;
  o1.nrows = nsky * lx;
  o1.nh = ly / 2;
  o1.nx = nx;
  o1.ny = ny;
  o1.lx = lx;
  o1.ly = ly;
  o1.hx = std::min(lx - nx, nx - 1);
  o1.hy = std::min(ly - ny, ny - 1);
  FR_TRY(pk1(ly, o1, tw_rows, s));
  TOp ot;
  ot.ht = ht;
  ot.lx = lx;
  ot.nh = ly / 2;
  ot.transfer = transfer;
  ot.scale = (float)(1.0 / ((double)lx * (double)ly));
  return pt(lx, ot, nsky, tw_cols, s);
}

}  // namespace fr
