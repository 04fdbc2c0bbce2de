// PSF convolutions of several plans in one launch per pass (Sec. 3.3.2), for the serving loop.
//
// The plans share the image size nx x ny and the padded lengths lx x ly, so their images form
// one flat batch for the three passes of fft_psf.cu: P1 over all sky rows of all plans, P2 over
// all images (each image multiplied by its own plan's transfer function), P3 over all rows. A
// small table in the kernel parameters gives every plan's first image, sky, output and
// transfer function; the passes differ from the single-plan ones only in where a row is read
// from, which transfer function an image takes, and where a row is written.
#include <algorithm>

#include "fft_engine.cuh"

namespace fr {

constexpr int PSF_GROUP_MAX = 16;  // plans per grouped call

struct PsfGroupTable {
  int njobs;
  int nx, ny, nq, lx;
  int img0[PSF_GROUP_MAX + 1];  // first image of each plan's block (prefix sums)
  int nsky[PSF_GROUP_MAX];
  const float* sky[PSF_GROUP_MAX];      // [batch][nsky][nx][ny]
  float* out[PSF_GROUP_MAX];            // same layout
  const float* transfer[PSF_GROUP_MAX]; // [nsky][nq][lx]
  // the plan that image `img` belongs to (every index static: no local copy of the table)
  __device__ __forceinline__ int job_of_image(int img) const {
    int j = 0;
#pragma unroll
    for (int k = 1; k < PSF_GROUP_MAX; ++k)
      if (k < njobs && img >= img0[k]) j = k;
    return j;
  }
};

// P1 over the rows of every plan's skies: row rho of the flat batch is row rho - nx img0[j] of
// plan j; both rows of a pair belong to one image (nx is even)
struct P1GroupOp : OpBase {
  static constexpr bool TRANSPOSED = true;
  PsfGroupTable t;
  float2* ht;  // [img][nh + 1][nx]
  int nrows, nh;
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return nh + 1; }
  __device__ float2 load(int r, int i) const {
    if (i >= t.ny) return make_float2(0.f, 0.f);
    const int rho = 2 * r;
    const int j = t.job_of_image(rho / t.nx);
    const float* src = pick_static(t.sky, j);
    const size_t a = (size_t)(rho - t.nx * pick_static(t.img0, j)) * t.ny + i;
    return make_float2(__ldg(&src[a]), __ldg(&src[a + t.ny]));
  }
  __device__ double store(int r, int k, SeqView v) const {
    const float2 z = v[k], zm = v[k == 0 ? 0 : 2 * nh - k];
    const float2 x1 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    const float2 x2 = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    const int rho = 2 * r;
    const int img = rho / t.nx, jx = rho - img * t.nx;
    float2* dst = ht + ((size_t)img * (nh + 1) + k) * t.nx + jx;
    dst[0] = x1;
    dst[1] = x2;
    return 0.0;
  }
};

// P2 over all images: forward transform, times the image's own plan's transfer function,
// inverse transform, crop; blockIdx.y is the image of the flat batch
struct P2GroupOp : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool TWO = true;
  PsfGroupTable t;
  const float2* ht;  // [img][nh + 1][nx]
  float2* h;         // [img][nx][hp]
  int hp, nh;
  __host__ __device__ int nseq() const { return nh + 1; }
  __host__ __device__ int nout() const { return t.nx; }
  __device__ float2 load(int q, int i) const {
    if (i >= t.nx) return make_float2(0.f, 0.f);
    return ht[((size_t)blockIdx.y * (nh + 1) + q) * t.nx + i];
  }
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2* s, int q0) const {
    const int img = blockIdx.y;
    const int j = t.job_of_image(img);
    const int k = (img - pick_static(t.img0, j)) % pick_static(t.nsky, j);
    const float* T = pick_static(t.transfer, j) + (size_t)k * t.nq * L;
    for (int idx = threadIdx.x; idx < B * L; idx += NT) {
      const int c = idx / L, p = idx % L;
      if (q0 + c < t.nq) {
        const float tv = __ldg(&T[(size_t)(q0 + c) * L + p]);
        float2& z = s[c * LP + spad(p)];
        z.x *= tv;
        z.y *= tv;
      }
    }
  }
  __device__ double store(int q, int o, SeqView s) const {
    h[((size_t)blockIdx.y * t.nx + o) * hp + q] = s[o];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int o, SeqView s) const { return s[o]; }
  __device__ void store_group(int q0, int o, const float2* v, int n) const {
    store_run(h + ((size_t)blockIdx.y * t.nx + o) * hp + q0, v, n);
  }
};

// P3 over all row pairs: Hermitian extension, inverse transform, crop, written to the row's
// own plan's output
struct P3GroupOp : OpBase {
  PsfGroupTable t;
  const float2* h;
  int hp, nh, nrows;
  __host__ __device__ int nseq() const { return nrows >> 1; }
  __host__ __device__ int nout() const { return t.ny; }
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
  __device__ double store(int r, int n, SeqView v) const {
    const float2 z = v[n];
    const int rho = 2 * r;
    const int j = t.job_of_image(rho / t.nx);
    float* dst = pick_static(t.out, j);
    const size_t a0 = (size_t)(rho - t.nx * pick_static(t.img0, j)) * t.ny + n;
    dst[a0] = z.x;
    dst[a0 + t.ny] = z.y;
    return 0.0;
  }
};

template <int LEN>
static int run_p1g(const P1GroupOp& op, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, -1>(op, 1, tw, s);
}
template <int LEN>
static int run_p2g(const P2GroupOp& op, int nimg, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, -1, 1>(op, nimg, tw, s);
}
template <int LEN>
static int run_p3g(const P3GroupOp& op, const float2* tw, cudaStream_t s) {
  return launch_pass<LEN, 1, 1>(op, 1, tw, s);
}
static int p1g(int len, const P1GroupOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p1g, op, tw, s); }
static int p2g(int len, const P2GroupOp& op, int n, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p2g, op, n, tw, s); }
static int p3g(int len, const P3GroupOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_p3g, op, tw, s); }

int psf_group_passes(const PsfGroupArgs& g, float2* h, float2* ht, const float2* tw_rows,
                     const float2* tw_cols, cudaStream_t s) {
  if (g.njobs < 1 || g.njobs > PSF_GROUP_MAX) {
    set_error("a grouped PSF convolution takes 1 to %d plans", PSF_GROUP_MAX);
    return FR_EINVAL;
  }
  PsfGroupTable t;
  t.njobs = g.njobs;
  t.nx = g.nx;
  t.ny = g.ny;
  t.nq = g.ly / 2 + 1;
  t.lx = g.lx;
  int nimg = 0;
  for (int j = 0; j < PSF_GROUP_MAX; ++j) {
    const bool on = j < g.njobs;
    t.img0[j] = nimg;
    t.nsky[j] = on ? g.nsky[j] : 1;
    t.sky[j] = on ? g.sky[j] : nullptr;
    t.out[j] = on ? g.out[j] : nullptr;
    t.transfer[j] = on ? g.transfer[j] : nullptr;
    if (on) nimg += g.nimg[j];
  }
  t.img0[PSF_GROUP_MAX] = nimg;
  const int nrows = nimg * g.nx, nh = g.ly / 2;
  const double px = (double)nrows * g.ny, hs = (double)nrows * (nh + 1);
  P1GroupOp o1;
  o1.t = t;
  o1.ht = ht;
  o1.nrows = nrows;
  o1.nh = nh;
  {
    ProfScope ps(PC_PSF_ROWS, s, px * 4.0 + hs * 8.0);
    FR_TRY(p1g(g.ly, o1, tw_rows, s));
  }
  P2GroupOp o2;
  o2.t = t;
  o2.ht = ht;
  o2.h = h;
  o2.hp = g.hp;
  o2.nh = nh;
  {
    ProfScope ps(PC_PSF_COLS, s, hs * 16.0 + (double)nimg * g.lx * (nh + 1) * 4.0);
    FR_TRY(p2g(g.lx, o2, nimg, tw_cols, s));
  }
  P3GroupOp o3;
  o3.t = t;
  o3.h = h;
  o3.hp = g.hp;
  o3.nh = nh;
  o3.nrows = nrows;
  ProfScope ps(PC_PSF_ROWS, s, hs * 8.0 + px * 4.0);
  return p3g(g.ly, o3, tw_rows, s);
}

}  // namespace fr
