// Internal declarations shared by the translation units of libfastresolve.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fastresolve.h"
#include "fft_core.cuh"

namespace fr {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* get_error();
void count_launch(int n = 1);

#define FR_CUDA_TRY(expr)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::fr::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,     \
                      __LINE__);                                                           \
      return e_ == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA;                       \
    }                                                                                      \
  } while (0)

#define FR_TRY(expr)            \
  do {                          \
    int r_ = (expr);            \
    if (r_ != FR_OK) return r_; \
  } while (0)

// launch check after a kernel launch
#define FR_LAUNCHED()                                                                       \
  do {                                                                                      \
    ::fr::count_launch();                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                    \
    if (e_ != cudaSuccess) {                                                                \
      ::fr::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,  \
                      __LINE__);                                                            \
      return FR_ECUDA;                                                                      \
    }                                                                                       \
  } while (0)

// device status word values (bitmask)
enum : int { ST_TIMEOUT = 1 };

// ------------------------------------------------------------------ launch profiling
// Kernel classes timed with CUDA events on the launching stream when profiling is enabled
// (fr_profile_enable); each launch also records its algorithmic bytes.
enum ProfCat : int {
  PC_FFT_ROWS = 0,  // grid FFT row passes (D1, G2)
  PC_FFT_COLS,      // grid FFT column passes (D2, G1)
  PC_DEGRID,        // degridder
  PC_GRID,          // gridder
  PC_PSF_ROWS,      // PSF-convolution row passes (P1, P3)
  PC_PSF_COLS,      // PSF-convolution column pass (P2)
  PC_PREP,          // visibility gather / weighting before gridding
  PC_REDUCE,        // FP64 reductions and small elementwise kernels
  PC_N
};
struct ProfScope {
  int slot = -1;
  cudaStream_t stream = nullptr;
  ProfScope(int cat, cudaStream_t s, double bytes);
  ~ProfScope();
};

// ------------------------------------------------------------------ kernel shape
// Exponential-of-semicircle gridding kernel phi(x) = exp(beta (sqrt(1 - (2x/W)^2) - 1)),
// |x| <= W/2 in grid cells.
struct EsKernel {
  int W;         // support in cells
  float beta;    // shape
  float inv_hw;  // 2 / W
};

__device__ __forceinline__ float es_eval(const EsKernel& k, float x) {
  float z = x * k.inv_hw;
  float t = fmaxf(1.f - z * z, 0.f);
  return __expf(k.beta * (sqrtf(t) - 1.f));
}

// Same kernel with sqrt(t) taken as t * rsqrt(t): a few ulp in the square root, far below the
// kernel's own approximation error; t = 0 (the footprint edge) maps to sqrt = 0.
__device__ __forceinline__ float es_eval_fast(const EsKernel& k, float x) {
  float z = x * k.inv_hw;
  float t = fmaxf(1.f - z * z, 1e-30f);
  return __expf(k.beta * (t * rsqrtf(t) - 1.f));
}

// ------------------------------------------------------------------ tiles and TMA
constexpr int TILE = 32;       // grid cells per tile side (u and v)
constexpr int MINW = 4, MAXW = 8;  // kernel supports of eps in [1e-6, 1e-2]
// visibilities per work item at most: w-stacking items (sorted by origin in every gridding call)
// and fixed per-tile chunks (sorted once when the plan is built)
constexpr int STACK_CHUNK = 512;
constexpr int ITEM_CHUNK = 2048;
constexpr int DEGRID_TERMS_SMEM = 200 * 1024;  // shared tiles of all expansion terms at most
constexpr size_t TERM_GRIDS_MAX_BYTES = (size_t)4 << 30;  // resident expansion term grids at most

// Padded tile box: rows BU = TILE + W - 1, columns BV = BU rounded up to even (16-byte rows).
__host__ __device__ inline int box_u(int W) { return TILE + W - 1; }
__host__ __device__ inline int box_v(int W) { return (TILE + W - 1 + 1) & ~1; }

// ------------------------------------------------------------------ sorted visibility set
// One imaging geometry: image nx x ny, oversampled grid Nu x Nv, kernel, w-stacking.
struct Geometry {
  int nx = 0, ny = 0, Nu = 0, Nv = 0;
  double dl = 0, dm = 0;
  EsKernel kern{};
  double beta = 0;
  bool wterm = false, nterm = false;
  double t_min = 0, t_c = 0, t_half = 0;  // w-stacking image-side extent
  double dw = 0;                           // plane spacing (wavelengths)
  // Small w-phase: exp(-2 pi i w (t - t_c)) = sum_n (-i a)^n tau^n / n!, a = 2 pi w t_half,
  // tau = (t - t_c) / t_half in [-1, 1], truncated after `nterms` terms; each term is one
  // "plane" with the real image multiplier tau^n / n! and the visibility weight (-i a)^n.
  bool taylor = false;
  int nterms = 0;
  float* corr = nullptr;                   // [nx*ny] (-1)^(px+py) / (n Phi_u Phi_v Phi_w)
  int32_t* tq = nullptr;                   // [nx*ny] (t - t_c) / t_half * 2^30  (wterm)
  cudaStream_t async = nullptr;            // tables are stream-ordered transients when set
};

// Visibilities sorted by (image group, tile, first w-plane) for one geometry.
struct VisLayout {
  int ngroups = 0;
  int ntu = 0, ntv = 0;                 // tiles per grid side
  std::vector<int> planes;              // [ngroups]
  std::vector<double> w_lo;             // [ngroups]
  std::vector<int64_t> plane_items;     // [sum planes + 1] item ranges, (g, p) major
  std::vector<int> plane_base;          // [ngroups] index of (g, 0) in plane_items
  std::vector<int64_t> group_begin;     // [ngroups + 1] sorted index range of each group
  std::vector<int64_t> plane_visits;    // [sum planes] visibilities processed per (g, p)
  // grid band holding every kernel footprint (inclusive cell ranges); cells outside it are
  // never read by the degridder and never written by the gridder
  int bu0 = 0, bu1 = -1, bv0 = 0, bv1 = -1;
  int64_t nvis = 0;                     // visibilities in user order
  int64_t nsorted = 0;                  // kept after dropping
  int64_t ndropped = 0;
  // device arrays in sorted order
  uint32_t* cell = nullptr;  // iu0 << 18 | iv0 << 4 | (p_first & 15)
  float* du = nullptr;
  float* dv = nullptr;
  float* dw = nullptr;       // y_w - p_first   (wterm)
  uint32_t* ph = nullptr;    // frac(w t_c) as Q32 (wterm)
  uint32_t* perm = nullptr;  // user index (row * nchan + chan) | conj flag << 31
  float* wgt = nullptr;
  int4* items = nullptr;     // {vis_begin, vis_count, tu << 16 | tv, 0}
  // w-stacking: tiles each plane's footprints reach, per plane q (index of plane_items):
  // occ_bits [q][ntv][occ_ntw] bitmap, occ_comp [q][ntv] compact tile-row index or -1,
  // occ_rows the occupied tile rows of every plane (ascending) from occ_row_off[q]
  bool occ_ok = false;
  int occ_ntw = 0;
  uint32_t* occ_bits = nullptr;
  int* occ_comp = nullptr;
  int* occ_rows = nullptr;
  std::vector<int64_t> occ_row_off;  // [nq + 1]
  std::vector<int64_t> occ_tiles;    // [nq] occupied tiles
  int occ_max_rows = 0;              // most occupied tile rows of any plane
  bool presorted = false;    // each item's visibilities ordered by footprint origin
  int64_t nitems = 0;
  size_t bytes = 0;
  cudaStream_t async = nullptr;  // arrays are stream-ordered transients when set
};

// Per-stream scratch.
struct Workspace {
  cudaStream_t stream = nullptr;
  float2* b1 = nullptr;      // [band v][nx] half-transformed plane of the degridding pre-pass
  float2* b1g = nullptr;     // [nx][Nv] half plane of the gridding post-pass (zero off-band)
  float2* grid = nullptr;    // [Nu][Nv] oversampled grid (kept zero between fr_grid calls)
  bool grid_zero = false;
  float2* vbuf = nullptr;    // [nsorted] sorted visibilities (accumulator / weighted input)
  float2* h = nullptr;       // PSF-apply half spectra [nimg][nx][HP]
  size_t h_bytes = 0;
  float* tmp_img = nullptr;  // [nsky][nx][ny] scratch image (exact likelihood, major cycle)
  float2* tmp_vis = nullptr; // [nvis] scratch visibilities (exact likelihood, major cycle)
  double* red = nullptr;     // [max(batch, 4)] FP64 reduction targets
  size_t red_n = 0;
  CUtensorMap tmap;          // TMA descriptor of `grid`
  bool tmap_ok = false;
  float2* grid_terms = nullptr;  // [Nv][Nu][T] interleaved term grids of the small-w expansion
  CUtensorMap tmap_terms;        // 3-D TMA descriptor of `grid_terms`
  float2* grid_terms_g = nullptr;  // [nterms][Nv][Nu] gridding term grids (kept zero)
  bool terms_g_zero = false;
  float* img_a = nullptr;  // [n] image scratch of the fast-resolve likelihood
  float* img_b = nullptr;
  size_t img_n = 0;
  float2* b1_stack = nullptr;   // STACK_K compact half planes of the w-stacking passes
  size_t b1_stack_n = 0;        // complex values per compact half plane
  float2* b1_terms = nullptr;   // [nterms][band v][nx] degridding half planes
  float2* b1g_terms = nullptr;  // [nterms][nx][Nv] gridding half planes (zero off-band)
  // FR_DETERMINISTIC: fixed-point grid(s) (kept zero), the call's largest contribution (float
  // bits) and 1 / scale
  longlong2* gridq = nullptr;
  size_t gridq_n = 0;
  unsigned* det_max = nullptr;
  double* det_inv = nullptr;
  size_t bytes = 0;
};

}  // namespace fr

struct fr_plan {
  fr::Geometry geo;
  fr::VisLayout lay;
  int64_t nrow = 0;
  int nchan = 0, nsky = 0;
  uint32_t flags = 0;
  double eps = 0;
  // PSF (Sec. 3.3.2)
  bool has_psf = false;
  std::vector<double> psf_norm;  // [nsky]
  float* psf_img = nullptr;      // [nsky][2nx][2ny]
  float* transfer = nullptr;     // [nsky][psf_ly/2+1][psf_lx], includes 1 / (lx ly)
  int psf_lx = 0, psf_ly = 0;    // padded PSF transform lengths (>= 2nx - 1: the whole PSF)
  size_t transfer_cap = 0;       // floats allocated for the transfer function
  // noise model of the fast-resolve likelihood (Sec. 3.3.3): 1 / K_xi, [nsky][ny][nx]
  bool has_noise = false;
  float* noise_kinv = nullptr;
  double noise_eps = 0;
  std::vector<double> noise_logdet;  // [nsky] 1/2 sum ln(2 pi K)
  // twiddle tables by log2 length, and of the other (3 2^k, 5 2^k) lengths
  float2* tw[16] = {nullptr};
  std::map<int, float2*> tw_mixed;
  int* status = nullptr;         // device status word
  size_t resident = 0;
  std::mutex mu;
  std::vector<fr::Workspace*> ws;
};

namespace fr {

// twiddle tables
int ensure_twiddles(fr_plan* p, int L, cudaStream_t s);
const float2* twiddles_of(fr_plan* p, int L);

// -------- FFT passes (fft_*.cu) --------
// FR_DETERMINISTIC gridding (vis_common.cuh): with gridq set, the gridders add into 64-bit
// fixed-point grids (longlong2 per cell, same layout as the float2 grids) at the scale derived
// from *maxbits (det_max) and n
struct DetArgs {
  longlong2* gridq = nullptr;
  const unsigned* maxbits = nullptr;
  double* inv = nullptr;  // 1 / scale, written before the post-pass reads the fixed-point grid
  long long n = 0;
};
// Occupied tiles of one w-plane (VisLayout occ_*): the tile rows, the compact index of every
// tile row (-1 if empty), the bitmap, and the cells of the occupied tiles.
constexpr int STACK_K = 8;  // w-planes per launch of the stacked row passes
struct PlaneOcc {
  const int* rows = nullptr;
  const int* comp = nullptr;
  const uint32_t* bits = nullptr;
  int nrows = 0, ntw = 0;
  double ncells = 0.0;
};
PlaneOcc plane_occ(const VisLayout& lay, int q);
struct PlaneArgs {
  // geometry
  int nx, ny, Nu, Nv;
  int bu0, bu1, bv0, bv1;  // occupied grid band (inclusive)
  const float* corr;
  const int32_t* tq;
  long long k64;  // per-plane phase multiplier, Q64 cycles per tq unit (0 without w)
  int wterm;
  int taylor;      // 1: term n of the small-w expansion instead of a w-plane phase
  int n;           // term index
  float inv_fact;  // 1 / n!
};
constexpr int MAX_TERMS = 16;  // small-w expansion terms at most (the plan uses <= 12)
// All nterms expansion terms in one launch per pass: term t's half plane at b1 + t * b1_stride,
// its grid at grid + t * grid_stride; the gridding post-pass sums the terms into `dirty`.
// (the degridding pre-pass writes the interleaved term grids G[v][u][t], t < T)
int degrid_prepass_terms(const PlaneArgs& a, int nterms, const float* sky, float2* b1,
                         size_t b1_stride, float2* grid, int T, const float2* twv,
                         const float2* twu, cudaStream_t s);
int grid_postpass_terms(const PlaneArgs& a, int nterms, float2* grid, size_t grid_stride,
                        float2* b1, size_t b1_stride, float* dirty, const float2* twu,
                        const float2* twv, cudaStream_t s);
int degrid_prepass(const PlaneArgs& a, const float* sky, float2* b1, float2* grid,
                   const float2* twv, const float2* twu, cudaStream_t s);
int grid_postpass(const PlaneArgs& a, float2* grid, float2* b1, float* dirty, int accumulate,
                  const float2* twu, const float2* twv, cudaStream_t s);
// w-stacking over occupied tiles (fft_grid.cu): D1 for nk <= STACK_K planes (plane k's phase
// k64[k], compact half plane b1t[k], [occ[k].nrows * TILE][nx]); D2 of one plane into its
// occupied tiles of `grid`; G1 of one plane from its occupied tiles (zeroed) into the compact
// half plane b1 [nx][nrows * TILE]; G2 summing nk planes' half planes into `dirty`
int degrid_d1_stack(const PlaneArgs& a, int nk, const long long* k64, const PlaneOcc* occ,
                    const float* sky, float2* const* b1t, const float2* twv, cudaStream_t s);
int degrid_d2_sparse(const PlaneArgs& a, const PlaneOcc& occ, const float2* b1t, float2* grid,
                     const float2* twu, cudaStream_t s);
int grid_g1_sparse(const PlaneArgs& a, const PlaneOcc& occ, float2* grid, float2* b1,
                   const float2* twu, cudaStream_t s);
int grid_g2_stack(const PlaneArgs& a, int nk, const long long* k64, const PlaneOcc* occ,
                  float2* const* b1, float* dirty, int accumulate, const float2* twv,
                  cudaStream_t s);
// the same from fixed-point grids (FR_DETERMINISTIC); the terms are added to the image one
// after the other instead of with atomics
int grid_postpass_q(const PlaneArgs& a, const DetArgs& det, float2* b1, float* dirty,
                    int accumulate, const float2* twu, const float2* twv, cudaStream_t s);
int grid_postpass_terms_q(const PlaneArgs& a, int nterms, const DetArgs& det, size_t grid_stride,
                          float2* b1, size_t b1_stride, float* dirty, const float2* twu,
                          const float2* twv, cudaStream_t s);
// PSF-apply passes over nimg images of nx x ny; image i uses transfer + (i % nsky) * tstride
struct PsfArgs {
  int nx, ny, nimg, nsky;
  int lx, ly;  // padded transform lengths: nx < lx <= 2nx, ny < ly <= 2ny
  int hp;      // half-spectrum row pitch (complex), >= ly / 2 + 1
  const float* transfer;
  const float* sky;
  float* out;
  const float* dirty;   // likelihood mode (grad = conv - dirty), else null
  double* value;        // likelihood mode: [nimg / nsky] accumulators, else null
};
// PSF convolutions of several plans with equal nx, ny, lx, ly as one flat batch (one launch
// per pass): plan j contributes nimg[j] = batch_j nsky[j] images, its skies, outputs and
// transfer function (host arrays of njobs entries)
struct PsfGroupArgs {
  int njobs = 0;
  int nx = 0, ny = 0, lx = 0, ly = 0, hp = 0;
  const float* const* sky = nullptr;
  float* const* out = nullptr;
  const float* const* transfer = nullptr;
  const int* nsky = nullptr;
  const int* nimg = nullptr;
};
int psf_group_passes(const PsfGroupArgs& g, float2* h, float2* ht, const float2* tw_rows,
                     const float2* tw_cols, cudaStream_t s);
// h: [nimg][nx][hp] half spectra, ht: [nimg][ly/2+1][nx] transposed half spectra; tw_rows
// and tw_cols are the twiddle tables of lengths ly and lx
int psf_apply_passes(const PsfArgs& a, float2* h, float2* ht, const float2* tw_rows,
                     const float2* tw_cols, cudaStream_t s);
// transfer function of the lx x ly periodic kernel cut from PSF images [nsky][2nx][2ny]
// -> TT [nsky][ly/2+1][lx] (ht: [nsky][ly/2+1][lx] scratch)
int build_transfer(int nx, int ny, int nsky, const float* psf, int lx, int ly, float2* ht,
                   float* transfer, const float2* tw_rows, const float2* tw_cols, cudaStream_t s);
// lengths the PSF passes take (powers of two 32..16384, 3 2^k 48..6144, 5 2^k 80..5120)
bool fft_len_supported(int L);
// the shortest supported length >= m (m <= 16384)
int fft_len_at_least(int m);
// lengths the noise passes take: fft_len_supported() ones and c 2^k <= 4096, 16 | L, with c in
// {9, 15, 25, 45, 75, 225}
bool noise_len_supported(int L);
// noise model passes (noise.cu): n_delta [nsky][nx][ny] -> kinv [nsky][ny][nx], logdet [nsky]
// (accumulated); ht scratch [nsky][ny][nx]
int noise_kernel_passes(const float* n_delta, int nx, int ny, int nsky, float eps, float2* ht,
                        float* kinv, double* logdet, const float2* tw_y, const float2* tw_x,
                        cudaStream_t s);
// out = sgn N'^-1 x for nimg images (image i uses kernel i % nsky); with t non-null,
// value[i / nsky] += 1/2 t . N'^-1 x; ht, h scratch [nimg][nx][ny] complex each
int noise_inverse_passes(const float* x, int nx, int ny, int nimg, int nsky, const float* kinv,
                         float2* ht, float2* h, float* out, float sgn, const float* t,
                         double* value, const float2* tw_y, const float2* tw_x, cudaStream_t s);

// -------- gridding kernels (gridder.cu) --------
int build_layout(const Geometry& geo, const double* d_uvw, int64_t nrow, const double* h_freqs,
                 const double* d_freqs, int nchan, const float* d_weights, int ngroups,
                 const std::vector<double>& w_lo, const std::vector<int>& planes, bool drop_oob,
                 VisLayout* lay, cudaStream_t s);
void free_layout(VisLayout* lay);
int make_tmap(CUtensorMap* m, float2* grid, int Nu, int Nv, int W);
int degrid_plane(const Geometry& geo, const VisLayout& lay, int g, int p,
                 const CUtensorMap& tmap, float2* vacc, float2* vis_out, int* status,
                 cudaStream_t s);
// small-w expansion: interleaved term grids [Nv][Nu][T] behind one 3-D tensor map (degridding),
// stacked [nterms][Nv][Nu] grids (gridding)
bool degrid_terms_fits(const Geometry& geo);
int term_grid_count(const Geometry& geo);  // T: terms per cell of the interleaved term grids
int make_tmap_terms(CUtensorMap* m, float2* grid, int Nu, int Nv, int T, int W);
int degrid_terms(const Geometry& geo, const VisLayout& lay, int g, const CUtensorMap& tmap,
                 float2* vis_out, int* status, cudaStream_t s);
int det_max(const VisLayout& lay, const float2* ysorted, const float2* vis, int apply_weights,
            int pw, unsigned* maxbits, cudaStream_t s);
int grid_terms(const Geometry& geo, const VisLayout& lay, int g, const float2* vis,
               int apply_weights, float2* grid_terms, const DetArgs& det, cudaStream_t s);
int grid_plane(const Geometry& geo, const VisLayout& lay, int g, int p, const float2* ysorted,
               float2* grid, const DetArgs& det, cudaStream_t s);
int grid_prepare(const Geometry& geo, const VisLayout& lay, const float2* vis, int apply_weights,
                 float2* ysorted, cudaStream_t s);
// one CTA whose bounded mbarrier wait runs out (no copy issued): sets ST_TIMEOUT in *status
int selftest_wait_timeout(int* status, cudaStream_t s);
int make_tables(Geometry* geo, const std::vector<double>& inv_phi_u,
                const std::vector<double>& inv_phi_v, cudaStream_t s);
void kernel_ft_tables(const Geometry& geo, std::vector<double>& inv_u, std::vector<double>& inv_v);
long long plane_k64(const Geometry& geo, double w_plane);
double plane_w(const Geometry& geo, const VisLayout& lay, int g, int p);

// -------- small kernels (api.cu) --------
int zero_psf_edges(float* psf, int nsky, int nx2, int ny2, cudaStream_t s);
int sub_images(const float* a, const float* b, float* out, size_t n, cudaStream_t s);
int dot_images(const float* a, const float* b, size_t n, double scale, double* acc,
               cudaStream_t s);  // acc += scale * sum(a*b)
int chi2_vis(const float2* v, const float2* m, const float* w, size_t n, double* acc,
             cudaStream_t s);

}  // namespace fr
