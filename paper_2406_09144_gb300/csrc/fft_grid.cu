// FFT passes of the measurement operator R and its adjoint (Eq. rime, Eq. clean).
//
// Layouts: sky and dirty images [jx][jy]; the oversampled grid of one w-plane G[v][u] (u
// fastest, zero frequency at (Nu/2, Nv/2)); the half-transformed plane B1T[v][jx] on the way
// in and B1[jx][v] on the way out. Each pass reads contiguous sequences; the transposed stores
// produce the next pass's contiguous input.
//
// Degridding pre-pass for one w-plane p (forward transforms):
//   D1 (image rows, along v): I_j c_p(j) placed at v index (py mod Nv), FFT -> B1T[.][jx]
//      with c_p(j) = corr_j exp(-2 pi i w_p (t_j - t_c));
//   D2 (B1T rows, along u): row v placed at u index (px mod Nu), FFT -> G[v][.].
// corr_j = (-1)^(px+py) / (n_j Phi_u Phi_v Phi_w) holds the grid correction (reciprocal of the
// gridding kernel's Fourier transform) and the sign that centres zero frequency.
//
// Gridding post-pass for one w-plane (inverse transforms, cropped as early as possible):
//   G1 (grid rows, along u): inverse FFT, keep px in [-nx/2, nx/2) -> B1[.][v]; the grid row is
//      zeroed once loaded (the grid stays zero between calls);
//   G2 (B1 rows, along v): inverse FFT, keep ny outputs, Re(Z conj(c_p(j))) accumulated into the
//      dirty image.
#include "fft_grid_common.cuh"
#include "vis_common.cuh"

namespace fr {

// 1 / k! for the expansion terms
__constant__ float c_inv_fact[MAX_TERMS] = {
    1.f,           1.f,           1.f / 2.f,          1.f / 6.f,           1.f / 24.f,
    1.f / 120.f,   1.f / 720.f,   1.f / 5040.f,       1.f / 40320.f,       1.f / 362880.f,
    1.f / 3628800.f, 1.f / 39916800.f, 1.f / 479001600.f, 1.f / 6227020800.f, 1.f / 87178291200.f,
    1.f / 1307674368000.f};

// 1 / k
__constant__ float c_recip[MAX_TERMS] = {0.f,       1.f,        1.f / 2.f,  1.f / 3.f,
                                         1.f / 4.f, 1.f / 5.f,  1.f / 6.f,  1.f / 7.f,
                                         1.f / 8.f, 1.f / 9.f,  1.f / 10.f, 1.f / 11.f,
                                         1.f / 12.f, 1.f / 13.f, 1.f / 14.f, 1.f / 15.f};

// tau^n / n! for the small-w expansion, tau = tq * 2^-30 = (t - t_c) / t_half
__device__ __forceinline__ float taylor_factor(int32_t tq, int n, float inv_fact) {
  const float tau = (float)tq * 9.313225746154785e-10f;
  float p = inv_fact;
  for (int i = 0; i < n; ++i) p *= tau;
  return p;
}

struct D1Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  const float* sky;
  const float* corr;
  const int32_t* tq;
  long long k64;
  int wterm;
  int taylor, n;  // expansion term n + blockIdx.y
  float2* b1t;  // [band v][nx], term blockIdx.y at b1t + blockIdx.y * b1t_stride
  size_t b1t_stride;
  int nx, ny, Nv;
  int vb0, nvb;  // occupied band of v: only these outputs are stored
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return nvb; }
  __device__ float2 load(int jx, int i) const {
    const int hy = ny >> 1;
    int jy;
    if (i < hy)
      jy = i + hy;
    else if (i >= Nv - hy)
      jy = i - Nv + hy;
    else
      return make_float2(0.f, 0.f);
    const int pix = jx * ny + jy;
    const float val = __ldg(&sky[pix]) * __ldg(&corr[pix]);
    if (!wterm) return make_float2(val, 0.f);
    if (taylor) {
      const int m = n + blockIdx.y;
      return make_float2(val * taylor_factor(__ldg(&tq[pix]), m, c_inv_fact[m]), 0.f);
    }
    float c, s;
    plane_phase(__ldg(&tq[pix]), k64, &c, &s);
    return make_float2(val * c, -val * s);
  }
  __device__ double store(int jx, int o, SeqView s) const {
    b1t[blockIdx.y * b1t_stride + (size_t)o * nx + jx] = s[vb0 + o];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int o, SeqView s) const { return s[vb0 + o]; }
  __device__ void store_group(int jx0, int o, const float2* v, int n) const {
    store_run(b1t + blockIdx.y * b1t_stride + (size_t)o * nx + jx0, v, n);
  }
};

struct D2Op : OpBase {
  const float2* b1t;
  float2* grid;  // [Nv][Nu]; term blockIdx.y at the strides below
  size_t b1t_stride, grid_stride;
  int nx, Nu, Nv;
  int vb0, nvb, ub0, nub;  // only band rows are transformed, only band columns stored
  __host__ __device__ int nseq() const { return nvb; }
  __host__ __device__ int nout() const { return nub; }
  __device__ float2 load(int v, int i) const {
    const int hx = nx >> 1;
    int jx;
    if (i < hx)
      jx = i + hx;
    else if (i >= Nu - hx)
      jx = i - Nu + hx;
    else
      return make_float2(0.f, 0.f);
    return b1t[blockIdx.y * b1t_stride + (size_t)v * nx + jx];  // v: band row index
  }
  __device__ double store(int q, int o, SeqView s) const {
    const int u = ub0 + o;
    grid[blockIdx.y * grid_stride + (size_t)(vb0 + q) * Nu + u] = s[u];
    return 0.0;
  }
  static constexpr bool DIRECT = true;  // band columns only
  __device__ double direct(int q, int u, float2 z) const {
    if (u >= ub0 && u < ub0 + nub) grid[blockIdx.y * grid_stride + (size_t)(vb0 + q) * Nu + u] = z;
    return 0.0;
  }
};

// D1 for all expansion terms from one load: raw element (sky * corr, tau), term t's input
// sky * corr * tau^t / t! built by one multiply per term, half plane of term t at
// b1t + t * b1t_stride.
struct D1TermsOp {
  static constexpr bool TRANSPOSED = true;
  const float* sky;
  const float* corr;
  const int32_t* tq;
  float2* b1t;  // [band v][nx] per term
  size_t b1t_stride;
  int nterm;
  int nx, ny, Nv;
  int vb0, nvb;
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return nvb; }
  __device__ int nterms() const { return nterm; }
  __device__ float2 load(int jx, int i) const {
    const int hy = ny >> 1;
    int jy;
    if (i < hy)
      jy = i + hy;
    else if (i >= Nv - hy)
      jy = i - Nv + hy;
    else
      return make_float2(0.f, 0.f);
    const int pix = jx * ny + jy;
    return make_float2(__ldg(&sky[pix]) * __ldg(&corr[pix]),
                       (float)__ldg(&tq[pix]) * 9.313225746154785e-10f);
  }
  __device__ float2 prep(int t, float2& raw) const {
    if (t > 0) raw.x *= raw.y * c_recip[t];
    return make_float2(raw.x, 0.f);
  }
  __device__ double store(int t, int jx, int o, SeqView s) const {
    b1t[t * b1t_stride + (size_t)o * nx + jx] = s[vb0 + o];
    return 0.0;
  }
};

// D2 for the interleaved term grids of the expansion degridder: sequence s = (band row q,
// term t) with t fastest, output G[v][u][t] (T >= nterm terms per cell). The transposed store
// writes the B terms of a cell next to each other.
struct D2TermsOp : OpBase {
  static constexpr bool TRANSPOSED = true;
  const float2* b1t;  // term t at b1t + t * b1t_stride, [band v][nx]
  size_t b1t_stride;
  float2* grid;  // [Nv][Nu][T]
  int nterm, T;
  int nx, Nu, Nv;
  int vb0, nvb, ub0, nub;
  __host__ __device__ int nseq() const { return nvb * nterm; }
  __host__ __device__ int nout() const { return nub; }
  __device__ float2 load(int sq, int i) const {
    const int q = sq / nterm, t = sq - (sq / nterm) * nterm;
    const int hx = nx >> 1;
    int jx;
    if (i < hx)
      jx = i + hx;
    else if (i >= Nu - hx)
      jx = i - Nu + hx;
    else
      return make_float2(0.f, 0.f);
    return b1t[t * b1t_stride + (size_t)q * nx + jx];
  }
  __device__ double store(int sq, int o, SeqView s) const {
    const int q = sq / nterm, t = sq - (sq / nterm) * nterm;
    const int u = ub0 + o;
    grid[((size_t)(vb0 + q) * Nu + u) * T + t] = s[u];
    return 0.0;
  }
};

struct G1Op : OpBase {
  static constexpr bool TRANSPOSED = true;
  float2* grid;  // [Nv][Nu]; term blockIdx.y at the strides below
  float2* b1;    // [nx][Nv], zero outside the band columns
  size_t grid_stride, b1_stride;
  int nx, Nu, Nv;
  int vb0, nvb, ub0, nub;  // rows outside the band are zero and transform to zero
  __host__ __device__ int nseq() const { return nvb; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int q, int i) const {
    if (i < ub0 || i >= ub0 + nub) return make_float2(0.f, 0.f);  // zero outside the band
    return grid[blockIdx.y * grid_stride + (size_t)(vb0 + q) * Nu + i];
  }
  __device__ void after_load(int seq0, int nb) const {
    // the gridder writes only inside the band: zeroing the band part of the rows restores an
    // all-zero grid
    const int n = nb * nub;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / nub, c = i - (i / nub) * nub;
      grid[blockIdx.y * grid_stride + (size_t)(vb0 + seq0 + r) * Nu + ub0 + c] =
          make_float2(0.f, 0.f);
    }
  }
  __device__ double store(int q, int o, SeqView s) const {
    b1[blockIdx.y * b1_stride + (size_t)o * Nv + vb0 + q] = s[wrap(o - (nx >> 1), Nu)];
    return 0.0;
  }
  static constexpr bool GROUP = true;
  __device__ float2 pick(int, int o, SeqView s) const {
    return s[wrap(o - (nx >> 1), Nu)];
  }
  __device__ void store_group(int q0, int o, const float2* v, int n) const {
    store_run(b1 + blockIdx.y * b1_stride + (size_t)o * Nv + vb0 + q0, v, n);
  }
};

// G1 on the fixed-point grids of FR_DETERMINISTIC: each cell is converted back to float with the
// call's inverse scale (one value in device memory) and the band is zeroed as in G1Op.
struct G1QOp : G1Op {
  longlong2* gridq;
  const double* inv;
  __device__ float2 load(int q, int i) const {
    if (i < ub0 || i >= ub0 + nub) return make_float2(0.f, 0.f);
    const longlong2 c = gridq[blockIdx.y * grid_stride + (size_t)(vb0 + q) * Nu + i];
    const double f = __ldg(inv);
    return make_float2((float)((double)c.x * f), (float)((double)c.y * f));
  }
  __device__ void after_load(int seq0, int nb) const {
    const int n = nb * nub;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / nub, c = i - (i / nub) * nub;
      gridq[blockIdx.y * grid_stride + (size_t)(vb0 + seq0 + r) * Nu + ub0 + c] = longlong2{0, 0};
    }
  }
};

__global__ void det_inv_kernel(const unsigned* maxbits, long long n, double* inv) {
  *inv = 1.0 / det_scale(maxbits, n);
}

struct G2Op : OpBase {
  const float2* b1;
  float* dirty;
  const float* corr;
  const int32_t* tq;
  long long k64;
  int wterm, accumulate;
  int taylor, n;
  float inv_fact;
  int nx, ny, Nv;
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return ny; }
  int vb0, nvb;  // the half plane is zero outside the band columns: no loads there
  __device__ float2 load(int jx, int i) const {
    if (i < vb0 || i >= vb0 + nvb) return make_float2(0.f, 0.f);
    return b1[(size_t)jx * Nv + i];
  }
  __device__ double store(int jx, int jy, SeqView s) const {
    return out(jx, jy, s[wrap(jy - (ny >> 1), Nv)]);
  }
  // transform index i holds image column jy = i + ny/2 (mod Nv) inside the crop
  static constexpr bool DIRECT = true;
  __device__ double direct(int jx, int i, float2 z) const {
    const int hy = ny >> 1;
    const int jy = i < hy ? i + hy : (i >= Nv - hy ? i - Nv + hy : -1);
    return jy >= 0 ? out(jx, jy, z) : 0.0;
  }
  __device__ double out(int jx, int jy, float2 z) const {
    const int pix = jx * ny + jy;
    float val;
    if (wterm && taylor) {
      val = z.x * taylor_factor(__ldg(&tq[pix]), n, inv_fact);
    } else if (wterm) {
      float c, sn;
      plane_phase(__ldg(&tq[pix]), k64, &c, &sn);
      val = z.x * c - z.y * sn;  // Re(z exp(+2 pi i w_p (t - t_c)))
    } else {
      val = z.x;
    }
    val *= __ldg(&corr[pix]);
    dirty[pix] = accumulate ? dirty[pix] + val : val;
    return 0.0;
  }
};

// Gridding post-pass, second half, for all expansion terms at once, one term per CTA row
// (blockIdx.y = term): each CTA transforms one term's rows and adds corr Re(Z_t) tau^t / t! into
// the zeroed image with float atomics, so the terms' transforms run side by side instead of in
// sequence (on the 1024-pixel VLA-like image the row passes of the expansion, D1 and this one,
// took 0.117 ms with a CTA summing the terms in turn and 0.094 ms this way).
struct G2TermsAddOp : OpBase {
  const float2* b1;  // term t at b1 + t * b1_stride, [nx][Nv]
  size_t b1_stride;
  float* dirty;      // zeroed before the launch
  const float* corr;
  const int32_t* tq;
  int nx, ny, Nv;
  int vb0, nvb;
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return ny; }
  __device__ float2 load(int jx, int i) const {
    if (i < vb0 || i >= vb0 + nvb) return make_float2(0.f, 0.f);
    return b1[blockIdx.y * b1_stride + (size_t)jx * Nv + i];
  }
  __device__ double store(int jx, int jy, SeqView s) const {
    return out(jx, jy, s[wrap(jy - (ny >> 1), Nv)]);
  }
  static constexpr bool DIRECT = true;
  __device__ double direct(int jx, int i, float2 z) const {
    const int hy = ny >> 1;
    const int jy = i < hy ? i + hy : (i >= Nv - hy ? i - Nv + hy : -1);
    return jy >= 0 ? out(jx, jy, z) : 0.0;
  }
  __device__ double out(int jx, int jy, float2 z) const {
    const int pix = jx * ny + jy;
    const int t = blockIdx.y;
    atomicAdd(&dirty[pix],
              z.x * taylor_factor(__ldg(&tq[pix]), t, c_inv_fact[t]) * __ldg(&corr[pix]));
    return 0.0;
  }
};

template <int LEN>
static int run_d1(const D1Op& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, 1, tw, s); }
template <int LEN>
static int run_d2(const D2Op& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, 1, tw, s); }
template <int LEN>
static int run_g1(const G1Op& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, 1, tw, s); }
template <int LEN>
static int run_g2(const G2Op& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, 1, tw, s); }

static int d1(int len, const D1Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d1, op, tw, s); }
static int d2(int len, const D2Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d2, op, tw, s); }
static int g1(int len, const G1Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g1, op, tw, s); }
static int g2(int len, const G2Op& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g2, op, tw, s); }
template <int LEN>
static int run_d1m(const D1TermsOp& op, const float2* tw, cudaStream_t s) { return launch_pass_multi<LEN, -1>(op, tw, s); }
static int d1m(int len, const D1TermsOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d1m, op, tw, s); }
template <int LEN>
static int run_d2i(const D2TermsOp& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, 1, tw, s); }
static int d2i(int len, const D2TermsOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d2i, op, tw, s); }
template <int LEN>
static int run_g1t(const G1Op& op, int nt, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, nt, tw, s); }
template <int LEN>
static int run_g1q(const G1QOp& op, int nt, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, nt, tw, s); }
static int g1q(int len, const G1QOp& op, int nt, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g1q, op, nt, tw, s); }
template <int LEN>
static int run_g2a(const G2TermsAddOp& op, int nt, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, nt, tw, s); }
static int g2a(int len, const G2TermsAddOp& op, int nt, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g2a, op, nt, tw, s); }
static int g1t(int len, const G1Op& op, int nt, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g1t, op, nt, tw, s); }



int degrid_prepass(const PlaneArgs& a, const float* sky, float2* b1, float2* grid,
                   const float2* twv, const float2* twu, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0) return FR_OK;
  const double img = (double)a.nx * a.ny, half = (double)a.nx * nvb, full = (double)nvb * nub;
  D1Op o1;
  o1.vb0 = a.bv0;
  o1.nvb = nvb;
  o1.sky = sky;
  o1.corr = a.corr;
  o1.tq = a.tq;
  o1.k64 = a.k64;
  o1.wterm = a.wterm;
  o1.taylor = a.taylor;
  o1.n = a.n;
  o1.b1t = b1;
  o1.b1t_stride = 0;
  o1.nx = a.nx;
  o1.ny = a.ny;
  o1.Nv = a.Nv;
  {
    // sky + corr (+ tq) in, half-transformed plane out
    ProfScope ps(PC_FFT_ROWS, s, img * (8.0 + (a.wterm ? 4.0 : 0.0)) + half * 8.0);
    FR_TRY(d1(a.Nv, o1, twv, s));
  }
  D2Op o2;
  o2.b1t = b1;
  o2.grid = grid;
  o2.b1t_stride = o2.grid_stride = 0;
  o2.nx = a.nx;
  o2.Nu = a.Nu;
  o2.Nv = a.Nv;
  o2.vb0 = a.bv0;
  o2.nvb = nvb;
  o2.ub0 = a.bu0;
  o2.nub = nub;
  ProfScope ps(PC_FFT_COLS, s, half * 8.0 + full * 8.0);
  return d2(a.Nu, o2, twu, s);
}

int grid_postpass(const PlaneArgs& a, float2* grid, float2* b1, float* dirty, int accumulate,
                  const float2* twu, const float2* twv, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0) return FR_OK;
  const double img = (double)a.nx * a.ny, band_rows = (double)nvb * a.Nu,
               band = (double)nvb * nub, half = (double)a.nx * a.Nv;
  G1Op o1;
  o1.grid = grid;
  o1.b1 = b1;
  o1.grid_stride = o1.b1_stride = 0;
  o1.nx = a.nx;
  o1.Nu = a.Nu;
  o1.Nv = a.Nv;
  o1.vb0 = a.bv0;
  o1.nvb = nvb;
  o1.ub0 = a.bu0;
  o1.nub = nub;
  {
    // band rows in, band zeroed, cropped band columns of the half plane out
    ProfScope ps(PC_FFT_COLS, s, band * 16.0 + (double)a.nx * nvb * 8.0);
    (void)band_rows;
    FR_TRY(g1(a.Nu, o1, twu, s));
  }
  G2Op o2;
  o2.b1 = b1;
  o2.dirty = dirty;
  o2.corr = a.corr;
  o2.tq = a.tq;
  o2.k64 = a.k64;
  o2.wterm = a.wterm;
  o2.taylor = a.taylor;
  o2.n = a.n;
  o2.inv_fact = a.inv_fact;
  o2.accumulate = accumulate;
  o2.nx = a.nx;
  o2.ny = a.ny;
  o2.Nv = a.Nv;
  o2.vb0 = a.bv0;
  o2.nvb = nvb;
  ProfScope ps(PC_FFT_ROWS, s,
               (double)a.nx * nvb * 8.0 +
                   img * (4.0 + (a.wterm ? 4.0 : 0.0) + (accumulate ? 8.0 : 4.0)));
  return g2(a.Nv, o2, twv, s);
}

int degrid_prepass_terms(const PlaneArgs& a, int nterms, const float* sky, float2* b1,
                         size_t b1_stride, float2* grid, int T, const float2* twv,
                         const float2* twu, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0 || nterms <= 0) return FR_OK;
  const double img = (double)a.nx * a.ny, half = (double)a.nx * nvb, full = (double)nvb * nub;
  D1TermsOp o1;
  o1.vb0 = a.bv0;
  o1.nvb = nvb;
  o1.sky = sky;
  o1.corr = a.corr;
  o1.tq = a.tq;
  o1.b1t = b1;
  o1.b1t_stride = b1_stride;
  o1.nterm = nterms;
  o1.nx = a.nx;
  o1.ny = a.ny;
  o1.Nv = a.Nv;
  {
    // sky + corr + tq in once, one half plane out per term
    ProfScope ps(PC_FFT_ROWS, s, img * 12.0 + nterms * half * 8.0);
    FR_TRY(d1m(a.Nv, o1, twv, s));
  }
  D2TermsOp o2;
  o2.b1t = b1;
  o2.b1t_stride = b1_stride;
  o2.grid = grid;
  o2.nterm = nterms;
  o2.T = T;
  o2.nx = a.nx;
  o2.Nu = a.Nu;
  o2.Nv = a.Nv;
  o2.vb0 = a.bv0;
  o2.nvb = nvb;
  o2.ub0 = a.bu0;
  o2.nub = nub;
  ProfScope ps(PC_FFT_COLS, s, nterms * (half * 8.0 + full * 8.0));
  return d2i(a.Nu, o2, twu, s);
}

int grid_postpass_terms(const PlaneArgs& a, int nterms, float2* grid, size_t grid_stride,
                        float2* b1, size_t b1_stride, float* dirty, const float2* twu,
                        const float2* twv, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0 || nterms <= 0) return FR_OK;
  const double img = (double)a.nx * a.ny, band = (double)nvb * nub,
               half = (double)a.nx * a.Nv;
  G1Op o1;
  o1.grid = grid;
  o1.b1 = b1;
  o1.grid_stride = grid_stride;
  o1.b1_stride = b1_stride;
  o1.nx = a.nx;
  o1.Nu = a.Nu;
  o1.Nv = a.Nv;
  o1.vb0 = a.bv0;
  o1.nvb = nvb;
  o1.ub0 = a.bu0;
  o1.nub = nub;
  {
    ProfScope ps(PC_FFT_COLS, s, nterms * (band * 16.0 + (double)a.nx * nvb * 8.0));
    FR_TRY(g1t(a.Nu, o1, nterms, twu, s));
  }
  G2TermsAddOp o2;
  o2.b1 = b1;
  o2.b1_stride = b1_stride;
  o2.dirty = dirty;
  o2.corr = a.corr;
  o2.tq = a.tq;
  o2.nx = a.nx;
  o2.ny = a.ny;
  o2.Nv = a.Nv;
  o2.vb0 = a.bv0;
  o2.nvb = nvb;
  FR_CUDA_TRY(cudaMemsetAsync(dirty, 0, (size_t)a.nx * a.ny * sizeof(float), s));
  // per term the band of a half plane in, corr + tq in and the image added to
  ProfScope ps(PC_FFT_ROWS, s, nterms * ((double)a.nx * nvb * 8.0 + img * 16.0));
  return g2a(a.Nv, o2, nterms, twv, s);
}


// ------------------------------------------------------------ FR_DETERMINISTIC post-passes
static float host_inv_fact(int t) {
  double f = 1.0;
  for (int k = 2; k <= t; ++k) f *= k;
  return (float)(1.0 / f);
}

static G1QOp g1q_op(const PlaneArgs& a, const DetArgs& det, double* inv, float2* b1,
                    size_t grid_stride, size_t b1_stride) {
  G1QOp o;
  o.grid = nullptr;
  o.gridq = det.gridq;
  o.inv = inv;
  o.b1 = b1;
  o.grid_stride = grid_stride;
  o.b1_stride = b1_stride;
  o.nx = a.nx;
  o.Nu = a.Nu;
  o.Nv = a.Nv;
  o.vb0 = a.bv0;
  o.nvb = a.bv1 - a.bv0 + 1;
  o.ub0 = a.bu0;
  o.nub = a.bu1 - a.bu0 + 1;
  return o;
}

int grid_postpass_q(const PlaneArgs& a, const DetArgs& det, float2* b1, float* dirty,
                    int accumulate, const float2* twu, const float2* twv, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0) return FR_OK;
  double* inv = det.inv;
  det_inv_kernel<<<1, 1, 0, s>>>(det.maxbits, det.n, inv);
  FR_LAUNCHED();
  {
    ProfScope ps(PC_FFT_COLS, s, (double)nvb * nub * 32.0 + (double)a.nx * nvb * 8.0);
    FR_TRY(g1q(a.Nu, g1q_op(a, det, inv, b1, 0, 0), 1, twu, s));
  }
  G2Op o2;
  o2.b1 = b1;
  o2.dirty = dirty;
  o2.corr = a.corr;
  o2.tq = a.tq;
  o2.k64 = a.k64;
  o2.wterm = a.wterm;
  o2.taylor = a.taylor;
  o2.n = a.n;
  o2.inv_fact = a.inv_fact;
  o2.accumulate = accumulate;
  o2.nx = a.nx;
  o2.ny = a.ny;
  o2.Nv = a.Nv;
  o2.vb0 = a.bv0;
  o2.nvb = nvb;
  ProfScope ps(PC_FFT_ROWS, s,
               (double)a.nx * nvb * 8.0 +
                   (double)a.nx * a.ny * (4.0 + (a.wterm ? 4.0 : 0.0) + (accumulate ? 8.0 : 4.0)));
  return g2(a.Nv, o2, twv, s);
}

int grid_postpass_terms_q(const PlaneArgs& a, int nterms, const DetArgs& det, size_t grid_stride,
                          float2* b1, size_t b1_stride, float* dirty, const float2* twu,
                          const float2* twv, cudaStream_t s) {
  const int nvb = a.bv1 - a.bv0 + 1, nub = a.bu1 - a.bu0 + 1;
  if (nvb <= 0 || nub <= 0 || nterms <= 0) return FR_OK;
  double* inv = det.inv;
  det_inv_kernel<<<1, 1, 0, s>>>(det.maxbits, det.n, inv);
  FR_LAUNCHED();
  {
    ProfScope ps(PC_FFT_COLS, s,
                 nterms * ((double)nvb * nub * 32.0 + (double)a.nx * nvb * 8.0));
    FR_TRY(g1q(a.Nu, g1q_op(a, det, inv, b1, grid_stride, b1_stride), nterms, twu, s));
  }
  // the terms one after the other (no atomics): term t adds corr Re(Z_t) tau^t / t!
  for (int t = 0; t < nterms; ++t) {
    G2Op o2;
    o2.b1 = b1 + t * b1_stride;
    o2.dirty = dirty;
    o2.corr = a.corr;
    o2.tq = a.tq;
    o2.k64 = a.k64;
    o2.wterm = 1;
    o2.taylor = 1;
    o2.n = t;
    o2.inv_fact = host_inv_fact(t);
    o2.accumulate = t > 0;
    o2.nx = a.nx;
    o2.ny = a.ny;
    o2.Nv = a.Nv;
    o2.vb0 = a.bv0;
    o2.nvb = nvb;
    ProfScope ps(PC_FFT_ROWS, s,
                 (double)a.nx * nvb * 8.0 + (double)a.nx * a.ny * (t > 0 ? 20.0 : 16.0));
    FR_TRY(g2(a.Nv, o2, twv, s));
  }
  return FR_OK;
}

}  // namespace fr
