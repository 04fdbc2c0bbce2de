// Tile-sparse FFT passes of w-stacking (Eq. rime, Eq. clean): the grid passes of fft_grid.cu
// restricted, plane by plane, to the tiles that plane's visibilities reach.
#include "fft_grid_common.cuh"

namespace fr {

// ---------------------------------------------------------------- w-stacking, tile-sparse
// Under w-stacking each w-plane's visibilities touch only part of the grid: the plane's
// occupied tiles (every tile of TILE x TILE cells that a footprint of one of its visibilities
// reaches; PlaneOcc). The stacked passes transform and store only what those tiles need:
//   D1 (image rows, STACK_K planes per launch, one CTA per (row, plane), the planes of one row
//      next to each other so the row is read from HBM once): outputs of the occupied tile rows
//      only -> compact half plane B1T_k[o][jx], o = compact row index (32 per tile row);
//   D2 (compact rows along u): only the occupied tiles' cells of G are written;
//   G1 (compact rows along u): only the occupied tiles' cells are read, and zeroed (the
//      gridder writes nothing else, so the grid is all zero again) -> compact B1_k[jx][o];
//   G2 (image rows, STACK_K planes per CTA): each plane's compact half plane, expanded to the
//      full row (zero outside the occupied tile rows), transformed in turn; the planes' terms
//      Re(Z_k exp(+2 pi i w_k (t - t_c))) are summed per pixel in registers and written once.
// Cells outside the occupied tiles are never read by the degridder of that plane (its
// footprints lie inside them) and never written by its gridder, so all of this is exact.
// (grid and sequence indices are non-negative: unsigned shifts, not signed divisions)
__device__ __forceinline__ unsigned tdiv(int x) { return (unsigned)x / TILE; }
__device__ __forceinline__ bool tile_on(const uint32_t* bits, int ntw, int v, int u) {
  return (__ldg(&bits[tdiv(v) * ntw + tdiv(u) / 32]) >> (tdiv(u) & 31)) & 1u;
}
__device__ __forceinline__ int compact_row_v(const int* rows, int o) {
  return __ldg(&rows[tdiv(o)]) * TILE + (o & (TILE - 1));
}

struct D1StackOp : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool GROUP = true;
  static constexpr bool SEQ_Y = true;  // blockIdx.x = plane of the batch
  static constexpr bool PREFETCH = true;
  __device__ void prefetch(int jx) const {
    if (blockIdx.x != 0) return;  // the row is shared by the batch's planes
    const size_t o = (size_t)jx * ny;
    const uint32_t b = (uint32_t)ny * 4;
    l2_prefetch(sky + o, b);
    l2_prefetch(corr + o, b);
    l2_prefetch(tq + o, b);
  }
  const float* sky;
  const float* corr;
  const int32_t* tq;
  long long k64[STACK_K];
  float2* b1t[STACK_K];     // [nrows_k * TILE][nx]
  const int* rows[STACK_K];
  int nout_k[STACK_K];      // nrows_k * TILE
  int nx, ny, Nv;
  __host__ __device__ int nseq() const { return nx; }
  __device__ int nout() const { return nout_k[blockIdx.x]; }
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
    float c, s;
    plane_phase(__ldg(&tq[pix]), k64[blockIdx.x], &c, &s);
    return make_float2(val * c, -val * s);
  }
  __device__ double store(int jx, int o, SeqView s) const {
    const int k = blockIdx.x;
    b1t[k][(size_t)o * nx + jx] = s[compact_row_v(rows[k], o)];
    return 0.0;
  }
  __device__ float2 pick(int, int o, SeqView s) const {
    return s[compact_row_v(rows[blockIdx.x], o)];
  }
  __device__ void store_group(int jx0, int o, const float2* v, int n) const {
    store_run(b1t[blockIdx.x] + (size_t)o * nx + jx0, v, n);
  }
};

struct D2SparseOp : OpBase {
  static constexpr bool PREFETCH = true;
  __device__ void prefetch(int q) const {
    l2_prefetch(b1t + (size_t)q * nx, (uint32_t)nx * sizeof(float2));
  }
  const float2* b1t;  // [nrows * TILE][nx]
  float2* grid;       // [Nv][Nu]
  const int* rows;
  const uint32_t* bits;
  int ntw, nrows;
  int nx, Nu, Nv;
  __host__ __device__ int nseq() const { return nrows * TILE; }
  __host__ __device__ int nout() const { return Nu; }
  __device__ float2 load(int q, int i) const {
    const int hx = nx >> 1;
    int jx;
    if (i < hx)
      jx = i + hx;
    else if (i >= Nu - hx)
      jx = i - Nu + hx;
    else
      return make_float2(0.f, 0.f);
    return b1t[(size_t)q * nx + jx];
  }
  __device__ double store(int q, int u, SeqView s) const { return direct(q, u, s[u]); }
  static constexpr bool DIRECT = true;
  __device__ double direct(int q, int u, float2 z) const {
    const int v = compact_row_v(rows, q);
    if (tile_on(bits, ntw, v, u)) grid[(size_t)v * Nu + u] = z;
    return 0.0;
  }
};

struct G1SparseOp : OpBase {
  static constexpr bool TRANSPOSED = true;
  static constexpr bool GROUP = true;
  float2* grid;   // [Nv][Nu]
  float2* b1;     // [nx][nrows * TILE]
  const int* rows;
  const uint32_t* bits;
  int ntw, nrows;
  int nx, Nu, Nv;
  __host__ __device__ int nseq() const { return nrows * TILE; }
  __host__ __device__ int nout() const { return nx; }
  __device__ float2 load(int q, int u) const {
    const int v = compact_row_v(rows, q);
    if (!tile_on(bits, ntw, v, u)) return make_float2(0.f, 0.f);
    return grid[(size_t)v * Nu + u];
  }
  __device__ void after_load(int seq0, int nb) const {
    // the gridder wrote only the occupied tiles: zeroing them restores an all-zero grid
    // (row index and tile-row bitmap hoisted per sequence; the unrolled loop issues its bitmap
    // loads independently)
    for (int r = 0; r < nb; ++r) {
      const int v = compact_row_v(rows, seq0 + r);
      const uint32_t* rb = bits + tdiv(v) * ntw;
      float2* row = grid + (size_t)v * Nu;
#pragma unroll 4
      for (int u = threadIdx.x; u < Nu; u += blockDim.x)
        if ((__ldg(&rb[tdiv(u) / 32]) >> (tdiv(u) & 31)) & 1u) row[u] = make_float2(0.f, 0.f);
    }
  }
  __device__ double store(int q, int o, SeqView s) const {
    b1[(size_t)o * (nrows * TILE) + q] = s[wrap(o - (nx >> 1), Nu)];
    return 0.0;
  }
  __device__ float2 pick(int, int o, SeqView s) const { return s[wrap(o - (nx >> 1), Nu)]; }
  __device__ void store_group(int q0, int o, const float2* v, int n) const {
    store_run(b1 + (size_t)o * (nrows * TILE) + q0, v, n);
  }
};

struct G2StackOp {
  const float2* b1[STACK_K];   // [nx][ncomp_k]
  const int* comp[STACK_K];    // [ntv] compact tile-row index or -1
  int ncomp[STACK_K];          // nrows_k * TILE
  long long k64[STACK_K];
  int nt;
  float* dirty;
  const float* corr;
  const int32_t* tq;
  int nx, ny, Nv, accumulate;
  struct Trans {
    const float2* b1;
    const int* comp;
    int ncomp;
    long long k64;
  };
  __host__ __device__ int nseq() const { return nx; }
  __host__ __device__ int nout() const { return ny; }
  __device__ int ntrans() const { return nt; }
  // no L2 prefetch: a wave ahead of this pass is 8 planes' rows for 304 CTAs (about 66 MB),
  // which measured as evicted before use (DRAM reads 1.24 -> 2.11 GB per launch)
  static constexpr bool PREFETCH = false;
  __device__ void prefetch(int) const {}
  __device__ Trans trans(int t) const {
    return Trans{pick_static(b1, t), pick_static(comp, t), pick_static(ncomp, t),
                 pick_static(k64, t)};
  }
  __device__ float2 load(const Trans& p, int jx, int v) const {
    const int c = __ldg(&p.comp[tdiv(v)]);
    if (c < 0) return make_float2(0.f, 0.f);
    return p.b1[(size_t)jx * p.ncomp + c * TILE + (v & (TILE - 1))];
  }
  // transform index i holds image column jy when i = jy - ny/2 (mod Nv): the crop
  __device__ int out_of(int i) const {
    const int hy = ny >> 1;
    if (i < hy) return i + hy;
    if (i >= Nv - hy) return i - Nv + hy;
    return -1;
  }
  __device__ float term(const Trans& p, int jx, int jy, float2 z) const {
    float cs, sn;
    plane_phase(__ldg(&tq[jx * ny + jy]), p.k64, &cs, &sn);
    return z.x * cs - z.y * sn;  // Re(z exp(+2 pi i w_k (t - t_c)))
  }
  __device__ void store(int jx, int jy, float acc) const {
    const int pix = jx * ny + jy;
    const float val = acc * __ldg(&corr[pix]);
    dirty[pix] = accumulate ? dirty[pix] + val : val;
  }
};

template <int LEN>
static int run_d1s(const D1StackOp& op, int k, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, k, tw, s); }
static int d1s(int len, const D1StackOp& op, int k, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d1s, op, k, tw, s); }
template <int LEN>
static int run_d2s(const D2SparseOp& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, -1, -1>(op, 1, tw, s); }
static int d2s(int len, const D2SparseOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_d2s, op, tw, s); }
template <int LEN>
static int run_g1s(const G1SparseOp& op, const float2* tw, cudaStream_t s) { return launch_pass<LEN, 1, 1>(op, 1, tw, s); }
static int g1s(int len, const G1SparseOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g1s, op, tw, s); }
template <int LEN>
static int run_g2s(const G2StackOp& op, const float2* tw, cudaStream_t s) { return launch_pass_accum<LEN, 1>(op, tw, s); }
static int g2s(int len, const G2StackOp& op, const float2* tw, cudaStream_t s) { FR_LEN_DISPATCH(len, run_g2s, op, tw, s); }

int degrid_d1_stack(const PlaneArgs& a, int nk, const long long* k64, const PlaneOcc* occ,
                    const float* sky, float2* const* b1t, const float2* twv, cudaStream_t s) {
  if (nk <= 0) return FR_OK;
  if (nk > STACK_K) {
    set_error("at most %d w-planes per stacked pass", STACK_K);
    return FR_EINVAL;
  }
  D1StackOp o;
  o.sky = sky;
  o.corr = a.corr;
  o.tq = a.tq;
  double out = 0.0;
  for (int k = 0; k < STACK_K; ++k) {
    const bool on = k < nk;
    o.k64[k] = on ? k64[k] : 0;
    o.b1t[k] = on ? b1t[k] : nullptr;
    o.rows[k] = on ? occ[k].rows : nullptr;
    o.nout_k[k] = on ? occ[k].nrows * TILE : 0;
    out += o.nout_k[k];
  }
  o.nx = a.nx;
  o.ny = a.ny;
  o.Nv = a.Nv;
  // sky + corr + tq in once for the batch, each plane's occupied rows out
  ProfScope ps(PC_FFT_ROWS, s, (double)a.nx * a.ny * 12.0 + out * a.nx * 8.0);
  return d1s(a.Nv, o, nk, twv, s);
}

int degrid_d2_sparse(const PlaneArgs& a, const PlaneOcc& occ, const float2* b1t, float2* grid,
                     const float2* twu, cudaStream_t s) {
  if (occ.nrows <= 0) return FR_OK;
  D2SparseOp o;
  o.b1t = b1t;
  o.grid = grid;
  o.rows = occ.rows;
  o.bits = occ.bits;
  o.ntw = occ.ntw;
  o.nrows = occ.nrows;
  o.nx = a.nx;
  o.Nu = a.Nu;
  o.Nv = a.Nv;
  ProfScope ps(PC_FFT_COLS, s, (double)occ.nrows * TILE * a.nx * 8.0 + occ.ncells * 8.0);
  return d2s(a.Nu, o, twu, s);
}

int grid_g1_sparse(const PlaneArgs& a, const PlaneOcc& occ, float2* grid, float2* b1,
                   const float2* twu, cudaStream_t s) {
  if (occ.nrows <= 0) return FR_OK;
  G1SparseOp o;
  o.grid = grid;
  o.b1 = b1;
  o.rows = occ.rows;
  o.bits = occ.bits;
  o.ntw = occ.ntw;
  o.nrows = occ.nrows;
  o.nx = a.nx;
  o.Nu = a.Nu;
  o.Nv = a.Nv;
  // occupied cells read and zeroed, compact half plane out
  ProfScope ps(PC_FFT_COLS, s, occ.ncells * 16.0 + (double)occ.nrows * TILE * a.nx * 8.0);
  return g1s(a.Nu, o, twu, s);
}

int grid_g2_stack(const PlaneArgs& a, int nk, const long long* k64, const PlaneOcc* occ,
                  float2* const* b1, float* dirty, int accumulate, const float2* twv,
                  cudaStream_t s) {
  if (nk <= 0) return FR_OK;
  if (nk > STACK_K) {
    set_error("at most %d w-planes per stacked pass", STACK_K);
    return FR_EINVAL;
  }
  G2StackOp o;
  double in = 0.0;
  for (int k = 0; k < STACK_K; ++k) {
    const bool on = k < nk;
    o.b1[k] = on ? b1[k] : nullptr;
    o.comp[k] = on ? occ[k].comp : nullptr;
    o.ncomp[k] = on ? occ[k].nrows * TILE : 0;
    o.k64[k] = on ? k64[k] : 0;
    in += o.ncomp[k];
  }
  o.nt = nk;
  o.dirty = dirty;
  o.corr = a.corr;
  o.tq = a.tq;
  o.nx = a.nx;
  o.ny = a.ny;
  o.Nv = a.Nv;
  o.accumulate = accumulate;
  // every plane's compact half plane in, corr + tq in and the image written once per batch
  ProfScope ps(PC_FFT_ROWS, s,
               in * a.nx * 8.0 + (double)a.nx * a.ny * (8.0 + (accumulate ? 8.0 : 4.0)));
  return g2s(a.Nv, o, twv, s);
}

}  // namespace fr
