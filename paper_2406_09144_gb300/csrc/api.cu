// C ABI of libfastresolve: plan creation (kernel choice, w-stacking layout, correction tables,
// sorted visibilities, PSF and its transfer function), the operator entry points, per-stream
// workspaces, error reporting and small FP64 reduction kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <memory>
#include <vector>

#include "fr_internal.cuh"

namespace fr {

// ------------------------------------------------------------------------ errors / counters
static thread_local std::string g_err;
static thread_local uint64_t g_launches = 0;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
const char* get_error() { return g_err.c_str(); }
void count_launch(int n) { g_launches += (uint64_t)n; }

// ------------------------------------------------------------------------ launch profiling
namespace {
struct ProfRec {
  int cat;
  double bytes;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;
double g_prof_ms[PC_N], g_prof_bytes[PC_N];
uint64_t g_prof_n[PC_N];

cudaEvent_t take_event() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_drain_locked() {
  for (ProfRec& r : g_prof) {
    float ms = 0.f;
    if (r.a && r.b && cudaEventSynchronize(r.b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_prof_ms[r.cat] += ms;
      g_prof_bytes[r.cat] += r.bytes;
      g_prof_n[r.cat] += 1;
    }
    if (r.a) g_ev_pool.push_back(r.a);
    if (r.b) g_ev_pool.push_back(r.b);
  }
  g_prof.clear();
}
}  // namespace

ProfScope::ProfScope(int cat, cudaStream_t s, double bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  if (g_prof.size() >= 8192) prof_drain_locked();
  ProfRec r{cat, bytes, take_event(), take_event()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, s);
  stream = s;
  slot = (int)g_prof.size();
  g_prof.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_prof.size()) cudaEventRecord(g_prof[slot].b, stream);
}

// ------------------------------------------------------------------------ reductions
static constexpr int RED_T = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RED_T / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    v = lane < RED_T / 32 ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

static unsigned nblocks(size_t n) {
  size_t b = (n + RED_T - 1) / RED_T;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(b, 152 * 16));
}

__global__ void __launch_bounds__(RED_T) dot_kernel(const float* a, const float* b, size_t n,
                                                    double scale, double* acc) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)RED_T + threadIdx.x; i < n; i += (size_t)gridDim.x * RED_T)
    s += (double)a[i] * (double)(b ? b[i] : a[i]);
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(acc, s * scale);
}

int dot_images(const float* a, const float* b, size_t n, double scale, double* acc,
               cudaStream_t s) {
  if (n == 0) return FR_OK;
  ProfScope ps(PC_REDUCE, s, (double)n * (b ? 8.0 : 4.0));
  dot_kernel<<<nblocks(n), RED_T, 0, s>>>(a, b, n, scale, acc);
  FR_LAUNCHED();
  return FR_OK;
}

__global__ void __launch_bounds__(RED_T) sub_kernel(const float* a, const float* b, float* out,
                                                    size_t n) {
  for (size_t i = blockIdx.x * (size_t)RED_T + threadIdx.x; i < n; i += (size_t)gridDim.x * RED_T)
    out[i] = a[i] - b[i];
}

int sub_images(const float* a, const float* b, float* out, size_t n, cudaStream_t s) {
  if (n == 0) return FR_OK;
  ProfScope ps(PC_REDUCE, s, (double)n * 12.0);
  sub_kernel<<<nblocks(n), RED_T, 0, s>>>(a, b, out, n);
  FR_LAUNCHED();
  return FR_OK;
}

// exact likelihood epilogue: grad = As - d (in place over As), acc[elem] += 1/2 s.As - s.d
__global__ void __launch_bounds__(RED_T) lik_kernel(const float* s, float* as_grad, const float* d,
                                                    size_t n, double* acc) {
  double v = 0.0;
  for (size_t i = blockIdx.x * (size_t)RED_T + threadIdx.x; i < n; i += (size_t)gridDim.x * RED_T) {
    const double si = s[i], ai = as_grad[i], di = d[i];
    v += 0.5 * si * ai - si * di;
    as_grad[i] = (float)(ai - di);
  }
  v = block_sum(v);
  if (threadIdx.x == 0) atomicAdd(acc, v);
}

// weighted data misfit over the kept visibilities, sorted order -> user index
__global__ void __launch_bounds__(RED_T) chi2_kernel(const float2* vis, const float2* model,
                                                     const float* wgt, const uint32_t* perm,
                                                     size_t n, double* acc) {
  double v = 0.0;
  for (size_t i = blockIdx.x * (size_t)RED_T + threadIdx.x; i < n; i += (size_t)gridDim.x * RED_T) {
    const uint32_t k = perm[i] & 0x7fffffffu;
    const double dr = (double)vis[k].x - model[k].x, di = (double)vis[k].y - model[k].y;
    v += (double)wgt[i] * (dr * dr + di * di);
  }
  v = block_sum(v);
  if (threadIdx.x == 0) atomicAdd(acc, v);
}

// vis[user index] *= weight for every kept visibility (sorted order -> user index)
__global__ void __launch_bounds__(RED_T) weight_vis_kernel(const uint32_t* perm, const float* wgt,
                                                           int64_t n, float2* vis) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float wv = wgt[i];
    float2* v = vis + (perm[i] & 0x7fffffffu);
    float2 x = *v;
    x.x *= wv;
    x.y *= wv;
    *v = x;
  }
}

// out = -x
__global__ void __launch_bounds__(RED_T) negate_kernel(const float* x, size_t n, float* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = -x[i];
}

__global__ void sum_weights_kernel(const float* w, int64_t b, int64_t e, double* acc) {
  double v = 0.0;
  for (int64_t i = b + blockIdx.x * (int64_t)RED_T + threadIdx.x; i < e;
       i += (int64_t)gridDim.x * RED_T)
    v += w[i];
  v = block_sum(v);
  if (threadIdx.x == 0) atomicAdd(acc, v);
}

__global__ void zero_edges_kernel(float* psf, int nimg, int nx2, int ny2) {
  const int64_t per = (int64_t)nx2 + ny2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per * nimg;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t img = i / per, r = i % per;
    float* p = psf + img * (int64_t)nx2 * ny2;
    if (r < ny2)
      p[r] = 0.f;  // row 0
    else
      p[(r - ny2) * ny2] = 0.f;  // column 0
  }
}

int zero_psf_edges(float* psf, int nsky, int nx2, int ny2, cudaStream_t s) {
  zero_edges_kernel<<<nblocks((size_t)(nx2 + ny2) * nsky), 256, 0, s>>>(psf, nsky, nx2, ny2);
  FR_LAUNCHED();
  return FR_OK;
}

// ------------------------------------------------------------------------ twiddles
static int make_twiddles(float2** out, int L, cudaStream_t s) {
  std::vector<float2> h(L);
  for (int m = 0; m < L; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)L;
    h[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  FR_CUDA_TRY(cudaMalloc(out, L * sizeof(float2)));
  FR_CUDA_TRY(cudaMemcpyAsync(*out, h.data(), L * sizeof(float2), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  return FR_OK;
}

// twiddle table of any length the FFT passes take (powers of two, 3 2^k, 5 2^k)
int ensure_twiddles(fr_plan* p, int L, cudaStream_t s) {
  if (!fft_len_supported(L) && !noise_len_supported(L)) {
    set_error("FFT length %d unsupported", L);
    return FR_EUNSUPPORTED;
  }
  if ((L & (L - 1)) == 0) {
    float2*& t = p->tw[ilog2(L)];
    if (!t) {
      FR_TRY(make_twiddles(&t, L, s));
      p->resident += (size_t)L * sizeof(float2);
    }
    return FR_OK;
  }
  std::lock_guard<std::mutex> lk(p->mu);
  if (!p->tw_mixed.count(L)) {
    float2* t = nullptr;
    FR_TRY(make_twiddles(&t, L, s));
    p->tw_mixed[L] = t;
    p->resident += (size_t)L * sizeof(float2);
  }
  return FR_OK;
}

const float2* twiddles_of(fr_plan* p, int L) {
  if ((L & (L - 1)) == 0) return p->tw[ilog2(L)];
  std::lock_guard<std::mutex> lk(p->mu);
  auto it = p->tw_mixed.find(L);
  return it == p->tw_mixed.end() ? nullptr : it->second;
}

// ------------------------------------------------------------------------ workspaces
static void free_ws(Workspace* w) {
  cudaFree(w->b1);
  cudaFree(w->b1g);
  cudaFree(w->grid);
  cudaFree(w->grid_terms);
  cudaFree(w->grid_terms_g);
  cudaFree(w->b1_stack);
  cudaFree(w->b1_terms);
  cudaFree(w->b1g_terms);
  cudaFree(w->img_a);
  cudaFree(w->img_b);
  cudaFree(w->vbuf);
  cudaFree(w->h);
  cudaFree(w->tmp_img);
  cudaFree(w->tmp_vis);
  cudaFree(w->red);
  cudaFree(w->gridq);
  cudaFree(w->det_max);
  cudaFree(w->det_inv);
  delete w;
}

template <class T>
static int ws_alloc(T** p, size_t n, Workspace* w) {
  if (n == 0) return FR_OK;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("workspace allocation of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
    return FR_ENOMEM;
  }
  w->bytes += n * sizeof(T);
  return FR_OK;
}

static int get_ws(fr_plan* p, cudaStream_t s, Workspace** out) {
  std::lock_guard<std::mutex> lk(p->mu);
  for (Workspace* w : p->ws)
    if (w->stream == s) {
      *out = w;
      return FR_OK;
    }
  std::unique_ptr<Workspace> w(new Workspace());
  w->stream = s;
  const Geometry& g = p->geo;
  int r;
  if ((r = ws_alloc(&w->b1, (size_t)g.nx * g.Nv, w.get())) ||
      (r = ws_alloc(&w->b1g, (size_t)g.nx * g.Nv, w.get())) ||
      (r = ws_alloc(&w->grid, (size_t)g.Nu * g.Nv, w.get())) ||
      (r = ws_alloc(&w->vbuf, (size_t)std::max<int64_t>(p->lay.nsorted, 1), w.get()))) {
    free_ws(w.release());
    return r;
  }
  // the gridding half plane is only ever written inside the band: zero it once
  cudaError_t e = cudaMemsetAsync(w->b1g, 0, (size_t)g.nx * g.Nv * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->grid, 0, (size_t)g.Nu * g.Nv * sizeof(float2), s);
  if (e != cudaSuccess) {
    set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    free_ws(w.release());
    return FR_ECUDA;
  }
  w->grid_zero = true;
  if ((r = make_tmap(&w->tmap, w->grid, g.Nu, g.Nv, g.kern.W))) {
    free_ws(w.release());
    return r;
  }
  w->tmap_ok = true;
  *out = w.get();
  p->ws.push_back(w.release());
  return FR_OK;
}

// resident term grids for the one-pass expansion degridder (allocated on first use); zeroed once
// so that tile cells outside the band, which no footprint reads, hold finite values
static int ws_reserve_terms(const Geometry& g, Workspace* w, cudaStream_t s) {
  if (w->grid_terms) return FR_OK;
  const int T = term_grid_count(g);
  const size_t n = (size_t)T * g.Nu * g.Nv;
  if (!w->b1_terms) FR_TRY(ws_alloc(&w->b1_terms, (size_t)g.nterms * g.nx * g.Nv, w));
  FR_TRY(ws_alloc(&w->grid_terms, n, w));
  FR_CUDA_TRY(cudaMemsetAsync(w->grid_terms, 0, n * sizeof(float2), s));
  int r = make_tmap_terms(&w->tmap_terms, w->grid_terms, g.Nu, g.Nv, T, g.kern.W);
  if (r) {
    cudaFree(w->grid_terms);
    w->bytes -= n * sizeof(float2);
    w->grid_terms = nullptr;
  }
  return r;
}

static int ws_reserve_terms_g(const Geometry& g, Workspace* w, cudaStream_t s) {
  const size_t n = (size_t)g.nterms * g.Nu * g.Nv;
  if (!w->grid_terms_g) {
    FR_TRY(ws_alloc(&w->grid_terms_g, n, w));
    w->terms_g_zero = false;
  }
  if (!w->b1g_terms) {
    // the post-pass writes only the band columns of each half plane: zero the rest once
    const size_t nb = (size_t)g.nterms * g.nx * g.Nv;
    FR_TRY(ws_alloc(&w->b1g_terms, nb, w));
    FR_CUDA_TRY(cudaMemsetAsync(w->b1g_terms, 0, nb * sizeof(float2), s));
  }
  if (!w->terms_g_zero) {
    FR_CUDA_TRY(cudaMemsetAsync(w->grid_terms_g, 0, n * sizeof(float2), s));
    w->terms_g_zero = true;
  }
  return FR_OK;
}

// FR_DETERMINISTIC scratch: a zeroed fixed-point grid of n cells and the scale words
static int ws_reserve_det(Workspace* w, size_t n, cudaStream_t s) {
  if (w->gridq_n < n) {
    cudaFree(w->gridq);
    w->gridq = nullptr;
    w->gridq_n = 0;
    FR_TRY(ws_alloc(&w->gridq, n, w));
    FR_CUDA_TRY(cudaMemsetAsync(w->gridq, 0, n * sizeof(longlong2), s));
    w->gridq_n = n;
  }
  if (!w->det_max) FR_TRY(ws_alloc(&w->det_max, 1, w));
  if (!w->det_inv) FR_TRY(ws_alloc(&w->det_inv, 1, w));
  return FR_OK;
}

// w-stacking over the planes' occupied tiles (grids of whole tiles)
static bool use_stack(const fr_plan* p) {
  return p->lay.occ_ok && p->geo.wterm && !p->geo.taylor;
}

// STACK_K compact half planes, each holding the most occupied tile rows of any plane
static int ws_reserve_stack(const fr_plan* p, Workspace* w) {
  const size_t n = std::max<size_t>((size_t)p->lay.occ_max_rows * TILE * p->geo.nx, 1);
  if (w->b1_stack && w->b1_stack_n >= n) return FR_OK;
  if (w->b1_stack) {
    cudaFree(w->b1_stack);
    w->bytes -= STACK_K * w->b1_stack_n * sizeof(float2);
    w->b1_stack = nullptr;
    w->b1_stack_n = 0;
  }
  FR_TRY(ws_alloc(&w->b1_stack, STACK_K * n, w));
  w->b1_stack_n = n;
  return FR_OK;
}

// the planes of group g that hold visibilities, ascending
static std::vector<int> busy_planes(const Geometry& geo, const VisLayout& lay, int g) {
  std::vector<int> ps;
  const int P = geo.wterm ? lay.planes[g] : 1;
  for (int p = 0; p < P; ++p) {
    const int q = lay.plane_base[g] + (geo.taylor ? 0 : p);
    if (lay.plane_items[q + 1] > lay.plane_items[q]) ps.push_back(p);
  }
  return ps;
}

// one batch of up to STACK_K planes of the stacked passes
struct StackBatch {
  int nk = 0;
  long long k64[STACK_K] = {0};
  PlaneOcc occ[STACK_K];
  float2* buf[STACK_K] = {nullptr};
};
static StackBatch stack_batch(const fr_plan* pl, const Workspace* w, int g,
                              const std::vector<int>& ps, size_t b) {
  StackBatch sb;
  sb.nk = (int)std::min<size_t>(STACK_K, ps.size() - b);
  for (int k = 0; k < sb.nk; ++k) {
    const int p = ps[b + k];
    sb.k64[k] = plane_k64(pl->geo, plane_w(pl->geo, pl->lay, g, p));
    sb.occ[k] = plane_occ(pl->lay, pl->lay.plane_base[g] + p);
    sb.buf[k] = w->b1_stack + (size_t)k * w->b1_stack_n;
  }
  return sb;
}

// the small-w expansion keeps all its term grids resident when they fit
static bool use_term_grids(const Geometry& g) {
  return g.wterm && g.taylor && degrid_terms_fits(g) &&
         (size_t)term_grid_count(g) * g.Nu * g.Nv * sizeof(float2) <= TERM_GRIDS_MAX_BYTES;
}

static int ws_reserve_imgs(Workspace* w, size_t n) {
  if (w->img_n >= n) return FR_OK;
  cudaFree(w->img_a);
  cudaFree(w->img_b);
  w->bytes -= 2 * w->img_n * sizeof(float);
  w->img_a = w->img_b = nullptr;
  w->img_n = 0;
  FR_TRY(ws_alloc(&w->img_a, n, w));
  FR_TRY(ws_alloc(&w->img_b, n, w));
  w->img_n = n;
  return FR_OK;
}

static int ws_reserve_h(Workspace* w, size_t n) {
  if (w->h_bytes >= n * sizeof(float2)) return FR_OK;
  cudaFree(w->h);
  w->bytes -= w->h_bytes;
  w->h = nullptr;
  w->h_bytes = 0;
  FR_TRY(ws_alloc(&w->h, n, w));
  w->h_bytes = n * sizeof(float2);
  return FR_OK;
}

static int ws_reserve_red(Workspace* w, size_t n) {
  if (w->red_n >= n) return FR_OK;
  cudaFree(w->red);
  w->red = nullptr;
  w->red_n = 0;
  FR_TRY(ws_alloc(&w->red, n, w));
  w->red_n = n;
  return FR_OK;
}

static int ws_reserve_tmp(fr_plan* p, Workspace* w) {
  if (!w->tmp_img) FR_TRY(ws_alloc(&w->tmp_img, (size_t)p->nsky * p->geo.nx * p->geo.ny, w));
  if (!w->tmp_vis) FR_TRY(ws_alloc(&w->tmp_vis, (size_t)std::max<int64_t>(p->lay.nvis, 1), w));
  return FR_OK;
}

// ------------------------------------------------------------------------ operators
static PlaneArgs plane_args(const Geometry& geo, const VisLayout& lay, int g, int p) {
  PlaneArgs a;
  a.nx = geo.nx;
  a.ny = geo.ny;
  a.Nu = geo.Nu;
  a.Nv = geo.Nv;
  a.corr = geo.corr;
  a.tq = geo.tq;
  a.wterm = geo.wterm ? 1 : 0;
  a.taylor = geo.taylor ? 1 : 0;
  a.n = p;
  double f = 1.0;
  for (int k = 2; k <= p; ++k) f *= k;
  a.inv_fact = (float)(1.0 / f);
  a.k64 = (geo.wterm && !geo.taylor) ? plane_k64(geo, plane_w(geo, lay, g, p)) : 0;
  a.bu0 = lay.bu0;
  a.bu1 = lay.bu1;
  a.bv0 = lay.bv0;
  a.bv1 = lay.bv1;
  return a;
}

// R for all images of a layout
static int run_degrid(fr_plan* pl, const Geometry& geo, const VisLayout& lay, Workspace* w,
                      const float* sky, float2* vis, cudaStream_t s) {
  if (lay.ndropped > 0)
    FR_CUDA_TRY(cudaMemsetAsync(vis, 0, (size_t)lay.nvis * sizeof(float2), s));
  const size_t img = (size_t)geo.nx * geo.ny;
  // small-w expansion: every term grid built first, then one interpolation pass reads them all
  const bool terms = use_term_grids(geo);
  if (terms) FR_TRY(ws_reserve_terms(geo, w, s));
  for (int g = 0; g < lay.ngroups; ++g) {
    const int P = geo.wterm ? lay.planes[g] : 1;
    if (terms) {
      const int q = lay.plane_base[g];
      if (lay.plane_items[q + 1] <= lay.plane_items[q]) continue;
      PlaneArgs a = plane_args(geo, lay, g, 0);
      FR_TRY(degrid_prepass_terms(a, P, sky + g * img, w->b1_terms, (size_t)geo.nx * geo.Nv,
                                  w->grid_terms, term_grid_count(geo), twiddles_of(pl, geo.Nv),
                                  twiddles_of(pl, geo.Nu), s));
      FR_TRY(degrid_terms(geo, lay, g, w->tmap_terms, vis, pl->status, s));
      continue;
    }
    if (use_stack(pl)) {
      // STACK_K planes' half planes from one pass over the image, then per plane the column
      // pass into its occupied tiles and the interpolation
      FR_TRY(ws_reserve_stack(pl, w));
      const std::vector<int> ps = busy_planes(geo, lay, g);
      for (size_t b = 0; b < ps.size(); b += STACK_K) {
        const StackBatch sb = stack_batch(pl, w, g, ps, b);
        const PlaneArgs a = plane_args(geo, lay, g, ps[b]);
        FR_TRY(degrid_d1_stack(a, sb.nk, sb.k64, sb.occ, sky + g * img, sb.buf,
                               twiddles_of(pl, geo.Nv), s));
        for (int k = 0; k < sb.nk; ++k) {
          FR_TRY(degrid_d2_sparse(a, sb.occ[k], sb.buf[k], w->grid, twiddles_of(pl, geo.Nu), s));
          w->grid_zero = false;
          FR_TRY(degrid_plane(geo, lay, g, ps[b + k], w->tmap, w->vbuf, vis, pl->status, s));
        }
      }
      continue;
    }
    for (int p = 0; p < P; ++p) {
      const int q = lay.plane_base[g] + (geo.taylor ? 0 : p);
      if (lay.plane_items[q + 1] <= lay.plane_items[q]) continue;
      PlaneArgs a = plane_args(geo, lay, g, p);
      FR_TRY(degrid_prepass(a, sky + g * img, w->b1, w->grid, twiddles_of(pl, geo.Nv),
                            twiddles_of(pl, geo.Nu), s));
      w->grid_zero = false;
      FR_TRY(degrid_plane(geo, lay, g, p, w->tmap, w->vbuf, vis, pl->status, s));
    }
  }
  return FR_OK;
}

// R^dag (N^-1) for all images of a layout; vis == null grids ones (PSF)
// R^dag (N^-1) for all images of a layout. With FR_DETERMINISTIC the gridders accumulate in
// fixed point (the workspace's grids, or det_in's for the PSF build, which has no workspace).
static int run_grid(fr_plan* pl, const Geometry& geo, const VisLayout& lay, Workspace* w,
                    const float2* vis, int apply_weights, float* dirty, float2* grid, float2* b1,
                    float2* ybuf, cudaStream_t s, bool* grid_zero, const DetArgs* det_in = nullptr) {
  const size_t img = (size_t)geo.nx * geo.ny;
  const size_t plane = (size_t)geo.Nu * geo.Nv;
  const bool det = (pl->flags & FR_DETERMINISTIC) != 0;
  DetArgs d;
  if (det) {
    if (det_in) {
      d = *det_in;
    } else {
      FR_TRY(ws_reserve_det(w, use_term_grids(geo) ? geo.nterms * plane : plane, s));
      d.gridq = w->gridq;
      d.maxbits = w->det_max;
      d.inv = w->det_inv;
    }
    d.n = lay.nsorted;
  }
  if (w && use_term_grids(geo)) {
    // small-w expansion: one spreading pass fills every term grid, then each term is transformed
    // and accumulated into the image with its own pixel factor
    FR_TRY(ws_reserve_terms_g(geo, w, s));
    if (det)
      FR_TRY(det_max(lay, nullptr, vis, apply_weights, geo.nterms - 1,
                     const_cast<unsigned*>(d.maxbits), s));
    for (int g = 0; g < lay.ngroups; ++g) {
      const int q = lay.plane_base[g];
      if (lay.plane_items[q + 1] <= lay.plane_items[q]) {
        FR_CUDA_TRY(cudaMemsetAsync(dirty + g * img, 0, img * sizeof(float), s));
        continue;
      }
      PlaneArgs a = plane_args(geo, lay, g, 0);
      if (det) {
        FR_TRY(grid_terms(geo, lay, g, vis, apply_weights, w->grid_terms_g, d, s));
        FR_TRY(grid_postpass_terms_q(a, geo.nterms, d, plane, w->b1g_terms,
                                     (size_t)geo.nx * geo.Nv, dirty + g * img,
                                     twiddles_of(pl, geo.Nu), twiddles_of(pl, geo.Nv), s));
        continue;
      }
      w->terms_g_zero = false;
      FR_TRY(grid_terms(geo, lay, g, vis, apply_weights, w->grid_terms_g, d, s));
      FR_TRY(grid_postpass_terms(a, geo.nterms, w->grid_terms_g, plane, w->b1g_terms,
                                 (size_t)geo.nx * geo.Nv, dirty + g * img, twiddles_of(pl, geo.Nu),
                                 twiddles_of(pl, geo.Nv), s));
      w->terms_g_zero = true;  // the post-pass zeroes the band it reads
    }
    return FR_OK;
  }
  FR_TRY(grid_prepare(geo, lay, vis, apply_weights, ybuf, s));
  if (det) {
    FR_TRY(det_max(lay, ybuf, nullptr, 0, geo.taylor ? geo.nterms - 1 : 0,
                   const_cast<unsigned*>(d.maxbits), s));
  } else {
    if (!*grid_zero)
      FR_CUDA_TRY(cudaMemsetAsync(grid, 0, plane * sizeof(float2), s));
    *grid_zero = true;
  }
  if (w && !det && use_stack(pl)) {
    // per plane the gridder and the column pass out of its occupied tiles; STACK_K planes'
    // half planes then summed into the image by one row pass
    FR_TRY(ws_reserve_stack(pl, w));
    for (int g = 0; g < lay.ngroups; ++g) {
      const std::vector<int> ps = busy_planes(geo, lay, g);
      if (ps.empty()) FR_CUDA_TRY(cudaMemsetAsync(dirty + g * img, 0, img * sizeof(float), s));
      for (size_t b = 0; b < ps.size(); b += STACK_K) {
        const StackBatch sb = stack_batch(pl, w, g, ps, b);
        const PlaneArgs a = plane_args(geo, lay, g, ps[b]);
        for (int k = 0; k < sb.nk; ++k) {
          FR_TRY(grid_plane(geo, lay, g, ps[b + k], ybuf, grid, d, s));
          FR_TRY(grid_g1_sparse(a, sb.occ[k], grid, sb.buf[k], twiddles_of(pl, geo.Nu), s));
        }
        FR_TRY(grid_g2_stack(a, sb.nk, sb.k64, sb.occ, sb.buf, dirty + g * img, b > 0 ? 1 : 0,
                             twiddles_of(pl, geo.Nv), s));
      }
    }
    return FR_OK;
  }
  for (int g = 0; g < lay.ngroups; ++g) {
    const int P = geo.wterm ? lay.planes[g] : 1;
    bool written = false;
    for (int p = 0; p < P; ++p) {
      const int q = lay.plane_base[g] + (geo.taylor ? 0 : p);
      if (lay.plane_items[q + 1] <= lay.plane_items[q]) continue;
      FR_TRY(grid_plane(geo, lay, g, p, ybuf, grid, d, s));
      PlaneArgs a = plane_args(geo, lay, g, p);
      if (det)
        FR_TRY(grid_postpass_q(a, d, b1, dirty + g * img, written ? 1 : 0,
                               twiddles_of(pl, geo.Nu), twiddles_of(pl, geo.Nv), s));
      else
        FR_TRY(grid_postpass(a, grid, b1, dirty + g * img, written ? 1 : 0,
                             twiddles_of(pl, geo.Nu), twiddles_of(pl, geo.Nv), s));
      written = true;
    }
    if (!written) FR_CUDA_TRY(cudaMemsetAsync(dirty + g * img, 0, img * sizeof(float), s));
  }
  return FR_OK;
}

// ------------------------------------------------------------------------ plan creation
static int choose_support(double eps) {
  // measured against the FP64 oracle: W = ceil(log10(1/eps)) + 1 left the relative L2 error of
  // R at about 1.2 eps for eps = 1e-5; one more cell of support restores a margin
  // (eps in [1e-6, 1e-2] gives 4 ..8; the clamp also absorbs rounding of log10 at the ends)
  int W = (int)std::ceil(std::log10(1.0 / eps) - 1e-9) + 2;
  return std::min(MAXW, std::max(MINW, W));
}

static void set_kernel(Geometry* g, int W) {
  g->kern.W = W;
  g->beta = 0.97 * M_PI * W * (1.0 - 1.0 / (2.0 * 2.0));
  g->kern.beta = (float)g->beta;
  g->kern.inv_hw = 2.0f / (float)W;
}

static int build_psf(fr_plan* p, const double* d_uvw, const double* freqs, const double* d_freqs,
                     const float* d_weights, cudaStream_t s) {
  Geometry pg;
  pg.nx = 2 * p->geo.nx;
  pg.ny = 2 * p->geo.ny;
  pg.Nu = fft_len_at_least(2 * pg.nx);
  pg.Nv = fft_len_at_least(2 * pg.ny);
  pg.dl = p->geo.dl;
  pg.dm = p->geo.dm;
  set_kernel(&pg, p->geo.kern.W);
  pg.wterm = false;
  pg.nterm = false;
  pg.async = s;  // the PSF geometry and layout are transients of plan creation
  FR_TRY(ensure_twiddles(p, pg.Nu, s));
  FR_TRY(ensure_twiddles(p, pg.Nv, s));
  std::vector<double> iu, iv;
  kernel_ft_tables(pg, iu, iv);
  FR_TRY(make_tables(&pg, iu, iv, s));
  VisLayout pl;
  pl.async = s;
  std::vector<double> wlo(p->nsky, 0.0);
  std::vector<int> planes(p->nsky, 1);
  int r = build_layout(pg, d_uvw, p->nrow, freqs, d_freqs, p->nchan, d_weights, p->nsky, wlo, planes,
                       true, &pl, s);
  float2 *grid = nullptr, *b1 = nullptr, *y = nullptr, *h = nullptr;
  const size_t nimg2 = (size_t)pg.nx * pg.ny;
  // default padded PSF lengths: the shortest transforms that hold every offset |a| <= nx - 1
  // of the cropped product (2nx, 2ny for powers of two)
  const int lx = fft_len_at_least(2 * p->geo.nx - 1), ly = fft_len_at_least(2 * p->geo.ny - 1);
  const size_t tsize = (size_t)p->nsky * lx * (ly / 2 + 1);
  if (r == FR_OK) r = ensure_twiddles(p, lx, s);
  if (r == FR_OK) r = ensure_twiddles(p, ly, s);
  if (r == FR_OK) {
    // transients are stream-ordered: building a plan does not synchronise the device
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMallocAsync(&grid, (size_t)pg.Nu * pg.Nv * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&b1, (size_t)pg.nx * pg.Nv * sizeof(float2), s);
    if (e == cudaSuccess)
      e = cudaMallocAsync(&y, (size_t)std::max<int64_t>(pl.nsorted, 1) * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&h, tsize * sizeof(float2), s);
    if (e == cudaSuccess && grid) e = cudaMemsetAsync(grid, 0, (size_t)pg.Nu * pg.Nv * sizeof(float2), s);
    // the gridding half plane must be zero outside the band of the PSF layout
    if (e == cudaSuccess && b1) e = cudaMemsetAsync(b1, 0, (size_t)pg.nx * pg.Nv * sizeof(float2), s);
    if (e == cudaSuccess) e = cudaMalloc(&p->psf_img, (size_t)p->nsky * nimg2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p->transfer, tsize * sizeof(float));
    p->transfer_cap = tsize;
    if (e != cudaSuccess) {
      set_error("PSF allocation failed: %s", cudaGetErrorString(e));
      r = FR_ENOMEM;
    }
  }
  // FR_DETERMINISTIC: a transient fixed-point grid and scale words for the PSF's gridding
  DetArgs pdet;
  void* detbuf = nullptr;
  if (r == FR_OK && (p->flags & FR_DETERMINISTIC)) {
    const size_t cells = (size_t)pg.Nu * pg.Nv;
    cudaError_t e = cudaMallocAsync(&detbuf, cells * sizeof(longlong2) + 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(detbuf, 0, cells * sizeof(longlong2), s);
    if (e != cudaSuccess) {
      set_error("PSF allocation failed: %s", cudaGetErrorString(e));
      r = FR_ENOMEM;
    } else {
      pdet.gridq = (longlong2*)detbuf;
      pdet.maxbits = (unsigned*)((char*)detbuf + cells * sizeof(longlong2));
      pdet.inv = (double*)((char*)detbuf + cells * sizeof(longlong2) + 128);
    }
  }
  if (r == FR_OK) {
    bool zero = true;  // zeroed above
    r = run_grid(p, pg, pl, nullptr, nullptr, 1, p->psf_img, grid, b1, y, s, &zero,
                 (p->flags & FR_DETERMINISTIC) ? &pdet : nullptr);
  }
  if (r == FR_OK) r = zero_psf_edges(p->psf_img, p->nsky, pg.nx, pg.ny, s);
  if (r == FR_OK)
    r = build_transfer(p->geo.nx, p->geo.ny, p->nsky, p->psf_img, lx, ly, h, p->transfer,
                       twiddles_of(p, ly), twiddles_of(p, lx), s);
  p->psf_lx = lx;
  p->psf_ly = ly;
  // psf_norm = sum of the kept weights per image (FP64)
  double* d_norm = nullptr;
  if (r == FR_OK) {
    cudaError_t e = cudaMallocAsync(&d_norm, p->nsky * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_norm, 0, p->nsky * sizeof(double), s);
    for (int g = 0; g < p->nsky && e == cudaSuccess; ++g) {
      const int64_t b = pl.group_begin[g], en = pl.group_begin[g + 1];
      if (en > b) sum_weights_kernel<<<nblocks(en - b), RED_T, 0, s>>>(pl.wgt, b, en, d_norm + g);
      count_launch();
      e = cudaGetLastError();
    }
    p->psf_norm.assign(p->nsky, 0.0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->psf_norm.data(), d_norm, p->nsky * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("PSF normalisation failed: %s", cudaGetErrorString(e));
      r = FR_ECUDA;
    }
  }
  for (void* q : {(void*)d_norm, (void*)grid, (void*)b1, (void*)y, (void*)h, (void*)pg.corr,
                  (void*)pg.tq, detbuf})
    if (q) cudaFreeAsync(q, s);
  free_layout(&pl);
  cudaStreamSynchronize(s);
  if (r == FR_OK) {
    p->has_psf = true;
    p->resident += (size_t)p->nsky * nimg2 * sizeof(float) + tsize * sizeof(float);
  }
  return r;
}


static int plan_create(const double* uvw, int64_t nrow, const double* freqs, int32_t nchan,
                       const float* weights, int32_t nx, int32_t ny, double dx, double dy,
                       double eps, uint32_t flags, cudaStream_t s, fr_plan* p) {
  if (flags & ~(FR_WTERM | FR_NTERM | FR_MFS | FR_DROP_OOB | FR_NO_PSF | FR_DETERMINISTIC)) {
    set_error("unknown flag bits 0x%x", flags & ~(FR_WTERM | FR_NTERM | FR_MFS | FR_DROP_OOB |
                                                  FR_NO_PSF | FR_DETERMINISTIC));
    return FR_EINVAL;
  }
  if (!uvw || !freqs || nrow <= 0 || nchan <= 0) {
    set_error("uvw/freqs must be non-null with nrow > 0 and nchan > 0");
    return FR_EINVAL;
  }
  if ((nx & 1) || (ny & 1) || nx < 16 || ny < 16 || nx > 4096 || ny > 4096) {
    set_error("nx, ny must be even and in [16, 4096] (got %d x %d)", nx, ny);
    return FR_EUNSUPPORTED;
  }
  if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy)) {
    set_error("pixel sizes must be finite and positive");
    return FR_EINVAL;
  }
  if (!(eps >= 1e-6 && eps <= 1e-2)) {
    set_error("eps must lie in [1e-6, 1e-2] (got %g)", eps);
    return FR_EUNSUPPORTED;
  }
  if ((int64_t)nrow * nchan >= (1ll << 31)) {
    set_error("at most 2^31 - 1 visibilities per plan");
    return FR_EUNSUPPORTED;
  }
  for (int c = 0; c < nchan; ++c)
    if (!(freqs[c] > 0) || !std::isfinite(freqs[c])) {
      set_error("frequency %d is not finite and positive", c);
      return FR_EINVAL;
    }
  double wabs_min = INFINITY, wabs_max = 0.0;
  for (int64_t r = 0; r < nrow; ++r) {
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(uvw[3 * r + k])) {
        set_error("uvw row %lld is not finite", (long long)r);
        return FR_EINVAL;
      }
    const double a = std::fabs(uvw[3 * r + 2]);
    wabs_min = std::min(wabs_min, a);
    wabs_max = std::max(wabs_max, a);
  }
  if (weights) {
    const int64_t M = nrow * nchan;
    for (int64_t k = 0; k < M; ++k)
      if (!(weights[k] >= 0.f) || !std::isfinite(weights[k])) {
        set_error("weight %lld is negative or not finite", (long long)k);
        return FR_EINVAL;
      }
  }
  p->nrow = nrow;
  p->nchan = nchan;
  p->nsky = (flags & FR_MFS) ? 1 : nchan;
  p->flags = flags;
  p->eps = eps;
  FR_CUDA_TRY(cudaMalloc(&p->status, sizeof(int)));
  FR_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), s));

  Geometry& g = p->geo;
  g.nx = nx;
  g.ny = ny;
  // oversampled grid: the shortest FFT length of at least twice the image (sigma = 2 for
  // powers of two, 3 2^k and 5 2^k; a little above 2 for other sides)
  g.Nu = fft_len_at_least(2 * nx);
  g.Nv = fft_len_at_least(2 * ny);
  g.dl = dx;
  g.dm = dy;
  set_kernel(&g, choose_support(eps));
  g.nterm = (flags & FR_NTERM) != 0;
  g.wterm = (flags & FR_WTERM) != 0;
  // w-stacking extent: t = n - 1 in [t_min, 0]
  const double lx = 0.5 * nx * dx, ly = 0.5 * ny * dy;
  const double r2max = std::min(lx * lx + ly * ly, 1.0);
  g.t_min = -r2max / (1.0 + std::sqrt(1.0 - r2max));
  double fmax = 0.0, fmin = INFINITY;
  for (int c = 0; c < nchan; ++c) {
    fmax = std::max(fmax, freqs[c]);
    fmin = std::min(fmin, freqs[c]);
  }
  const double CL = 299792458.0;
  if (g.wterm && (wabs_max * fmax / CL) * (-g.t_min) < 1e-9) g.wterm = false;  // phase < 1e-9 turn
  std::vector<double> w_lo(p->nsky, 0.0);
  std::vector<int> planes(p->nsky, 1);
  if (g.wterm) {
    g.t_c = 0.5 * g.t_min;
    g.t_half = -0.5 * g.t_min;
    g.dw = 1.0 / (2.0 * -g.t_min);  // oversampling 2 along w
    for (int k = 0; k < p->nsky; ++k) {
      const double flo = p->nsky == 1 ? fmin : freqs[k], fhi = p->nsky == 1 ? fmax : freqs[k];
      const double lo = wabs_min * flo / CL, hi = wabs_max * fhi / CL;
      w_lo[k] = lo;
      planes[k] = (int)std::floor((hi - lo) / g.dw) + 1 + g.kern.W;
    }
    // Small w-phase: the expansion exp(-i a tau) = sum_n (-i a tau)^n / n!, |tau| <= 1,
    // a = 2 pi w t_half, truncated after N + 1 terms has remainder <= x^(N+1) / (N+1)! with
    // x = max |a|. Use it when it needs fewer "planes" than w-stacking, keeping the remainder
    // far below eps.
    const double x = 2.0 * M_PI * (wabs_max * fmax / CL) * g.t_half;
    double term = x, fact = 1.0;
    int n_terms = 1;
    while (n_terms < 12 && term / fact > 1e-2 * eps) {
      ++n_terms;
      term *= x;
      fact *= n_terms;
    }
    const int pmin = *std::min_element(planes.begin(), planes.end());
    const bool converged = term / fact <= 1e-2 * eps;  // the 12-term cap alone is not enough
    if (converged && n_terms < pmin) {
      g.taylor = true;
      g.nterms = n_terms;
      for (int k = 0; k < p->nsky; ++k) planes[k] = n_terms;
    }
  }
  for (int L : {g.Nu, g.Nv}) FR_TRY(ensure_twiddles(p, L, s));

  // device copies of the inputs (plan-time only)
  double *d_uvw = nullptr, *d_freqs = nullptr;
  float* d_w = nullptr;
  struct Free {  // stream-ordered release: no device-wide synchronisation
    void* a;
    cudaStream_t s;
    ~Free() {
      if (a) cudaFreeAsync(a, s);
    }
  };
  FR_CUDA_TRY(cudaMallocAsync(&d_uvw, (size_t)nrow * 3 * sizeof(double), s));
  Free f1{d_uvw, s};
  FR_CUDA_TRY(cudaMallocAsync(&d_freqs, nchan * sizeof(double), s));
  Free f2{d_freqs, s};
  FR_CUDA_TRY(cudaMemcpyAsync(d_uvw, uvw, (size_t)nrow * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_freqs, freqs, nchan * sizeof(double), cudaMemcpyHostToDevice, s));
  if (weights) {
    FR_CUDA_TRY(cudaMallocAsync(&d_w, (size_t)nrow * nchan * sizeof(float), s));
    FR_CUDA_TRY(cudaMemcpyAsync(d_w, weights, (size_t)nrow * nchan * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  Free f3{d_w, s};

  std::vector<double> iu, iv;
  kernel_ft_tables(g, iu, iv);
  FR_TRY(make_tables(&g, iu, iv, s));
  p->resident += (size_t)nx * ny * (sizeof(float) + (g.wterm ? sizeof(int32_t) : 0));
  FR_TRY(build_layout(g, d_uvw, nrow, freqs, d_freqs, nchan, d_w, p->nsky, w_lo, planes,
                      (flags & FR_DROP_OOB) != 0, &p->lay, s));
  p->resident += p->lay.bytes;
  if (!(flags & FR_NO_PSF)) FR_TRY(build_psf(p, d_uvw, freqs, d_freqs, d_w, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  return FR_OK;
}

static void plan_free(fr_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (Workspace* w : p->ws) free_ws(w);
  free_layout(&p->lay);
  cudaFree(p->geo.corr);
  cudaFree(p->geo.tq);
  cudaFree(p->psf_img);
  cudaFree(p->transfer);
  cudaFree(p->noise_kinv);
  cudaFree(p->status);
  for (float2*& t : p->tw) cudaFree(t);
  for (auto& kv : p->tw_mixed) cudaFree(kv.second);
  delete p;
}

// ------------------------------------------------------------------------ host FFT check
template <int R, int DIR>
static void host_stage(const float2* in, float2* out, const float2* tw, int L, int Ns) {
  for (int j = 0; j < L / R; ++j) stockham_task<R, DIR>(in, out, tw, L, Ns, j);
}

template <int DIR>
static void host_fft(float2* buf, float2* tmp, const float2* tw, int L, int P) {
  int Ns = 1;
  float2* a = buf;
  float2* b = tmp;
  for (int st = 0; st < fft_num_stages(L, P); ++st) {
    const int R = fft_radix(L, st, P);
    switch (R) {
      case 2: host_stage<2, DIR>(a, b, tw, L, Ns); break;
      case 3: host_stage<3, DIR>(a, b, tw, L, Ns); break;
      case 4: host_stage<4, DIR>(a, b, tw, L, Ns); break;
      case 5: host_stage<5, DIR>(a, b, tw, L, Ns); break;
      case 8: host_stage<8, DIR>(a, b, tw, L, Ns); break;
      case 32: host_stage<32, DIR>(a, b, tw, L, Ns); break;
      default: host_stage<16, DIR>(a, b, tw, L, Ns); break;
    }
    Ns *= R;
    std::swap(a, b);
  }
  if (a != buf) std::memcpy(buf, a, sizeof(float2) * spad_len(L));
}

}  // namespace fr

using namespace fr;

extern "C" {

const char* fr_strerror(int code) {
  switch (code) {
    case FR_OK: return "success";
    case FR_EINVAL: return "invalid argument";
    case FR_ENOMEM: return "out of memory";
    case FR_ECUDA: return "CUDA error";
    case FR_EUNSUPPORTED: return "unsupported size or option";
    case FR_ETIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

const char* fr_last_error(void) { return get_error(); }

uint64_t fr_launch_count(int reset) {
  uint64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

void fr_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain_locked();
  if (on) {
    for (int c = 0; c < PC_N; ++c) {
      g_prof_ms[c] = 0.0;
      g_prof_bytes[c] = 0.0;
      g_prof_n[c] = 0;
    }
  }
  g_prof_on = on != 0;
}

int fr_profile_read(double* ms, double* bytes, uint64_t* launches, int32_t ncat) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain_locked();
  for (int c = 0; c < ncat && c < PC_N; ++c) {
    if (ms) ms[c] = g_prof_ms[c];
    if (bytes) bytes[c] = g_prof_bytes[c];
    if (launches) launches[c] = g_prof_n[c];
  }
  return PC_N;
}

const char* fr_profile_category(int32_t cat) {
  static const char* names[PC_N] = {"fft_rows", "fft_cols", "degrid", "grid",
                                    "psf_rows", "psf_cols", "vis_prep", "reduce"};
  return (cat >= 0 && cat < PC_N) ? names[cat] : "unknown";
}

int fr_plan_create(const double* uvw, int64_t nrow, const double* freqs, int32_t nchan,
                   const float* weights, int32_t nx, int32_t ny, double pixsize_x, double pixsize_y,
                   double eps, uint32_t flags, void* stream, fr_plan_t* out) {
  if (!out) {
    set_error("out must not be NULL");
    return FR_EINVAL;
  }
  *out = nullptr;
  fr_plan* p = new (std::nothrow) fr_plan();
  if (!p) return FR_ENOMEM;
  int r = plan_create(uvw, nrow, freqs, nchan, weights, nx, ny, pixsize_x, pixsize_y, eps, flags,
                      (cudaStream_t)stream, p);
  if (r != FR_OK) {
    std::string keep = get_error();
    plan_free(p);
    set_error("%s", keep.c_str());
    return r;
  }
  *out = p;
  return FR_OK;
}

void fr_plan_destroy(fr_plan_t p) { plan_free(p); }

int fr_degrid(fr_plan_t p, const float* sky, fr_cf32* vis, void* stream) {
  if (!p || !sky || !vis) {
    set_error("plan, sky and vis must be non-null");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  return run_degrid(p, p->geo, p->lay, w, sky, (float2*)vis, s);
}

int fr_degrid_weighted(fr_plan_t p, const float* sky, fr_cf32* vis, void* stream) {
  if (!p || !sky || !vis) {
    set_error("plan, sky and vis must be non-null");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  FR_TRY(run_degrid(p, p->geo, p->lay, w, sky, (float2*)vis, s));
  // N^-1: each kept visibility times its weight (dropped ones are already zero)
  const int64_t n = p->lay.nsorted;
  if (n > 0) {
    ProfScope ps(PC_REDUCE, s, (double)n * 16.0);
    weight_vis_kernel<<<nblocks((size_t)n), RED_T, 0, s>>>(p->lay.perm, p->lay.wgt, n,
                                                           (float2*)vis);
    FR_LAUNCHED();
  }
  return FR_OK;
}

int fr_grid(fr_plan_t p, const fr_cf32* vis, int32_t apply_weights, float* dirty, void* stream) {
  if (!p || !vis || !dirty) {
    set_error("plan, vis and dirty must be non-null");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  return run_grid(p, p->geo, p->lay, w, (const float2*)vis, apply_weights ? 1 : 0, dirty, w->grid,
                  w->b1g, w->vbuf, s, &w->grid_zero);
}

int fr_dirty_psf(fr_plan_t p, const fr_cf32* vis, float* dirty, float* psf, double* psf_norm,
                 void* stream) {
  if (!p) {
    set_error("plan must be non-null");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (dirty) FR_TRY(fr_grid(p, vis, 1, dirty, stream));
  if ((psf || psf_norm) && !p->has_psf) {
    set_error("plan was created with FR_NO_PSF");
    return FR_EINVAL;
  }
  if (psf)
    FR_CUDA_TRY(cudaMemcpyAsync(psf, p->psf_img,
                                (size_t)p->nsky * 4 * p->geo.nx * p->geo.ny * sizeof(float),
                                cudaMemcpyDeviceToDevice, s));
  if (psf_norm) std::memcpy(psf_norm, p->psf_norm.data(), p->nsky * sizeof(double));
  return FR_OK;
}

// half-spectrum row pitch of the PSF passes: ly/2 + 1 bins rounded up to a multiple of 4
// (32-byte group stores)
static int psf_pitch(int ly) { return (ly / 2 + 1 + 3) & ~3; }

// complex scratch of one PSF convolution of nimg images: H [nimg][nx][hp], HT [nimg][ly/2+1][nx]
static size_t psf_h_need(const fr_plan* p, int nimg) {
  return (size_t)nimg * p->geo.nx * (psf_pitch(p->psf_ly) + p->psf_ly / 2 + 1);
}

static int psf_common(fr_plan_t p, const float* sky, int32_t batch, float* out, const float* dirty,
                      double* value, cudaStream_t s) {
  if (!p->has_psf) {
    set_error("plan was created with FR_NO_PSF");
    return FR_EINVAL;
  }
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  const int nimg = batch * p->nsky;
  const int lx = p->psf_lx, ly = p->psf_ly;
  const int hp = psf_pitch(ly);
  const size_t hsize = (size_t)nimg * p->geo.nx * hp;  // H, then HT ([nimg][ly/2+1][nx])
  FR_TRY(ws_reserve_h(w, psf_h_need(p, nimg)));
  PsfArgs a;
  a.nx = p->geo.nx;
  a.ny = p->geo.ny;
  a.lx = lx;
  a.ly = ly;
  a.nimg = nimg;
  a.nsky = p->nsky;
  a.hp = hp;
  a.transfer = p->transfer;
  a.sky = sky;
  a.out = out;
  a.dirty = dirty;
  a.value = nullptr;
  if (dirty) {
    FR_TRY(ws_reserve_red(w, (size_t)std::max(batch, 4)));
    FR_CUDA_TRY(cudaMemsetAsync(w->red, 0, batch * sizeof(double), s));
    a.value = w->red;
  }
  FR_TRY(psf_apply_passes(a, w->h, w->h + hsize, twiddles_of(p, ly), twiddles_of(p, lx), s));
  if (dirty && value) {
    FR_CUDA_TRY(cudaMemcpyAsync(value, w->red, batch * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FR_OK;
}

int fr_psf_apply(fr_plan_t p, const float* sky, int32_t batch, float* out, void* stream) {
  if (!p || !sky || !out || batch < 1) {
    set_error("plan, sky, out must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  return psf_common(p, sky, batch, out, nullptr, nullptr, (cudaStream_t)stream);
}

// plans of one grouped PSF convolution: 1..16 of them, with PSFs, equal image sizes and padded
// lengths; total images of the group in *nimg
static int psf_group_check(const fr_plan_t* plans, int32_t n, const int32_t* batches,
                           int* nimg) {
  if (!plans || !batches || n < 1 || n > 16) {
    set_error("a grouped PSF convolution takes 1 to 16 plans with their batches");
    return FR_EINVAL;
  }
  *nimg = 0;
  for (int j = 0; j < n; ++j) {
    const fr_plan* p = plans[j];
    if (!p || batches[j] < 1) {
      set_error("plan %d is null or its batch is < 1", j);
      return FR_EINVAL;
    }
    if (!p->has_psf) {
      set_error("plan %d was created with FR_NO_PSF", j);
      return FR_EINVAL;
    }
    if (p->geo.nx != plans[0]->geo.nx || p->geo.ny != plans[0]->geo.ny ||
        p->psf_lx != plans[0]->psf_lx || p->psf_ly != plans[0]->psf_ly) {
      set_error("plan %d differs from plan 0 in image size or PSF padding", j);
      return FR_EINVAL;
    }
    *nimg += batches[j] * p->nsky;
  }
  return FR_OK;
}

int fr_psf_group_scratch_bytes(const fr_plan_t* plans, int32_t nplans, const int32_t* batches,
                               size_t* bytes) {
  int nimg = 0;
  FR_TRY(psf_group_check(plans, nplans, batches, &nimg));
  if (!bytes) {
    set_error("bytes must be non-null");
    return FR_EINVAL;
  }
  *bytes = psf_h_need(plans[0], nimg) * sizeof(float2);
  return FR_OK;
}

int fr_psf_apply_group(const fr_plan_t* plans, int32_t nplans, const float* const* skies,
                       const int32_t* batches, float* const* outs, void* scratch,
                       size_t scratch_bytes, void* stream) {
  int nimg = 0;
  FR_TRY(psf_group_check(plans, nplans, batches, &nimg));
  if (!skies || !outs || !scratch) {
    set_error("skies, outs and scratch must be non-null");
    return FR_EINVAL;
  }
  const fr_plan* p0 = plans[0];
  const size_t need = psf_h_need(p0, nimg) * sizeof(float2);
  if (scratch_bytes < need || ((uintptr_t)scratch & 15)) {
    set_error("scratch must be 16-byte aligned and hold %zu bytes (got %zu)", need, scratch_bytes);
    return FR_EINVAL;
  }
  std::vector<const float*> tr(nplans);
  std::vector<int> nsky(nplans), ni(nplans);
  for (int j = 0; j < nplans; ++j) {
    if (!skies[j] || !outs[j]) {
      set_error("sky and out of plan %d must be non-null", j);
      return FR_EINVAL;
    }
    tr[j] = plans[j]->transfer;
    nsky[j] = plans[j]->nsky;
    ni[j] = batches[j] * plans[j]->nsky;
  }
  PsfGroupArgs g;
  g.njobs = nplans;
  g.nx = p0->geo.nx;
  g.ny = p0->geo.ny;
  g.lx = p0->psf_lx;
  g.ly = p0->psf_ly;
  g.hp = psf_pitch(g.ly);
  g.sky = skies;
  g.out = outs;
  g.transfer = tr.data();
  g.nsky = nsky.data();
  g.nimg = ni.data();
  float2* h = (float2*)scratch;
  float2* ht = h + (size_t)nimg * g.nx * g.hp;
  fr_plan* pm = const_cast<fr_plan*>(p0);
  return psf_group_passes(g, h, ht, twiddles_of(pm, g.ly), twiddles_of(pm, g.lx),
                          (cudaStream_t)stream);
}

int fr_plan_prepare(fr_plan_t p, int32_t batch, void* stream) {
  if (!p || batch < 1) {
    set_error("plan must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  const Geometry& g = p->geo;
  if (use_term_grids(g)) {
    FR_TRY(ws_reserve_terms(g, w, s));
    FR_TRY(ws_reserve_terms_g(g, w, s));
  }
  if (use_stack(p)) FR_TRY(ws_reserve_stack(p, w));
  if (p->flags & FR_DETERMINISTIC)
    FR_TRY(ws_reserve_det(w, (use_term_grids(g) ? (size_t)g.nterms : 1) * g.Nu * g.Nv, s));
  if (p->has_psf) FR_TRY(ws_reserve_h(w, psf_h_need(p, batch * p->nsky)));
  FR_TRY(ws_reserve_red(w, (size_t)std::max(batch, 4)));
  return FR_OK;
}

int fr_psf_set_padding(fr_plan_t p, int32_t lx, int32_t ly, void* stream) {
  if (!p) {
    set_error("plan must be non-null");
    return FR_EINVAL;
  }
  if (!p->has_psf) {
    set_error("plan was created with FR_NO_PSF");
    return FR_EINVAL;
  }
  const int nx = p->geo.nx, ny = p->geo.ny;
  const int mx = std::max(2 * nx, fft_len_at_least(2 * nx - 1));
  const int my = std::max(2 * ny, fft_len_at_least(2 * ny - 1));
  if (lx <= nx || lx > mx || ly <= ny || ly > my || (lx & 1) || (ly & 1)) {
    set_error("padded PSF lengths %d x %d: need even nx < lx <= %d, ny < ly <= %d (%d x %d image)",
              lx, ly, mx, my, nx, ny);
    return FR_EINVAL;
  }
  if (!fft_len_supported(lx) || !fft_len_supported(ly)) {
    set_error("padded PSF lengths %d x %d: each must be 2^k (32..16384), 3 2^k (48..6144) or "
              "5 2^k (80..5120)", lx, ly);
    return FR_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FR_TRY(ensure_twiddles(p, lx, s));
  FR_TRY(ensure_twiddles(p, ly, s));
  const size_t tsize = (size_t)p->nsky * (ly / 2 + 1) * lx;
  if (tsize > p->transfer_cap) {  // a longer padding than the default: grow the transfer
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    float* t = nullptr;
    FR_CUDA_TRY(cudaMalloc(&t, tsize * sizeof(float)));
    cudaFree(p->transfer);
    p->resident += (tsize - p->transfer_cap) * sizeof(float);
    p->transfer = t;
    p->transfer_cap = tsize;
  }
  float2* ht = nullptr;
  FR_CUDA_TRY(cudaMallocAsync(&ht, tsize * sizeof(float2), s));
  const int r = build_transfer(nx, ny, p->nsky, p->psf_img, lx, ly, ht, p->transfer,
                               twiddles_of(p, ly), twiddles_of(p, lx), s);
  cudaFreeAsync(ht, s);
  if (r != FR_OK) return r;
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  p->psf_lx = lx;
  p->psf_ly = ly;
  return FR_OK;
}

int fr_psf_padding(fr_plan_t p, int32_t* lx, int32_t* ly) {
  if (!p || !lx || !ly) {
    set_error("plan, lx, ly must be non-null");
    return FR_EINVAL;
  }
  if (!p->has_psf) {
    set_error("plan was created with FR_NO_PSF");
    return FR_EINVAL;
  }
  *lx = p->psf_lx;
  *ly = p->psf_ly;
  return FR_OK;
}

int fr_likelihood_grad(fr_plan_t p, const float* sky, const float* dirty, int32_t batch,
                       int32_t exact, float* grad, double* value, void* stream) {
  if (!p || !sky || !dirty || !grad || batch < 1) {
    set_error("plan, sky, dirty, grad must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!exact) return psf_common(p, sky, batch, grad, dirty, value, s);
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  FR_TRY(ws_reserve_tmp(p, w));
  FR_TRY(ws_reserve_red(w, (size_t)std::max(batch, 4)));
  FR_CUDA_TRY(cudaMemsetAsync(w->red, 0, batch * sizeof(double), s));
  const size_t n = (size_t)p->nsky * p->geo.nx * p->geo.ny;
  for (int b = 0; b < batch; ++b) {
    const float* sb = sky + b * n;
    float* gb = grad + b * n;
    FR_TRY(run_degrid(p, p->geo, p->lay, w, sb, w->tmp_vis, s));
    FR_TRY(run_grid(p, p->geo, p->lay, w, w->tmp_vis, 1, gb, w->grid, w->b1g, w->vbuf, s,
                    &w->grid_zero));
    {
      ProfScope ps(PC_REDUCE, s, (double)n * 16.0);
      lik_kernel<<<nblocks(n), RED_T, 0, s>>>(sb, gb, dirty + b * n, n, w->red + b);
    }
    FR_LAUNCHED();
  }
  if (value) {
    FR_CUDA_TRY(cudaMemcpyAsync(value, w->red, batch * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FR_OK;
}

// ------------------------------------------------------------ noise model (Sec. 3.3.3)
__global__ void add_centre_kernel(float* img, int nsky, int nx, int ny, float v) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsky) img[((size_t)k * nx + nx / 2) * ny + ny / 2] += v;
}

__global__ void kernel_from_inverse(const float* kinv, int nsky, int nx, int ny, float* K) {
  const size_t n = (size_t)nsky * nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t img = i / ((size_t)nx * ny), r = i % ((size_t)nx * ny);
    const int kx = (int)(r / ny), ky = (int)(r % ny);
    K[i] = 1.f / kinv[(img * ny + ky) * nx + kx];
  }
}

// the noise passes transform the unpadded image: nx and ny must themselves be FFT lengths
static int noise_sizes_ok(const fr_plan* p) {
  if (!noise_len_supported(p->geo.nx) || !noise_len_supported(p->geo.ny)) {
    set_error("the noise model needs nx, ny of the form 2^k (>= 32), 3 2^k (>= 48), 5 2^k "
              "(>= 80) or c 2^k (a multiple of 16, >= 144) with c in {9, 15, 25, 45, 75, 225} "
              "(got %d x %d)", p->geo.nx, p->geo.ny);
    return FR_EUNSUPPORTED;
  }
  return FR_OK;
}

int fr_noise_fit(fr_plan_t p, double eps_noise, double* logdet, void* stream) {
  if (!p || !(eps_noise > 0.0) || !std::isfinite(eps_noise)) {
    set_error("plan must be non-null and eps_noise positive");
    return FR_EINVAL;
  }
  FR_TRY(noise_sizes_ok(p));
  cudaStream_t s = (cudaStream_t)stream;
  const Geometry& g = p->geo;
  FR_TRY(ensure_twiddles(p, g.nx, s));
  FR_TRY(ensure_twiddles(p, g.ny, s));
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  FR_TRY(ws_reserve_tmp(p, w));
  const size_t n = (size_t)p->nsky * g.nx * g.ny;
  FR_TRY(ws_reserve_imgs(w, n));
  FR_TRY(ws_reserve_h(w, n));
  FR_TRY(ws_reserve_red(w, (size_t)std::max(p->nsky, 4)));
  if (!p->noise_kinv) {
    FR_CUDA_TRY(cudaMalloc(&p->noise_kinv, n * sizeof(float)));
    p->resident += n * sizeof(float);
  }
  // N'(I_delta) = R^dag N^-1 R I_delta + eps I_delta with the exact operators (Eq. N_new)
  FR_CUDA_TRY(cudaMemsetAsync(w->img_a, 0, n * sizeof(float), s));
  add_centre_kernel<<<1, 32, 0, s>>>(w->img_a, p->nsky, g.nx, g.ny, 1.f);
  FR_LAUNCHED();
  FR_TRY(run_degrid(p, g, p->lay, w, w->img_a, w->tmp_vis, s));
  FR_TRY(run_grid(p, g, p->lay, w, w->tmp_vis, 1, w->img_b, w->grid, w->b1g, w->vbuf, s,
                  &w->grid_zero));
  add_centre_kernel<<<1, 32, 0, s>>>(w->img_b, p->nsky, g.nx, g.ny, (float)eps_noise);
  FR_LAUNCHED();
  FR_CUDA_TRY(cudaMemsetAsync(w->red, 0, p->nsky * sizeof(double), s));
  FR_TRY(noise_kernel_passes(w->img_b, g.nx, g.ny, p->nsky, (float)eps_noise, w->h,
                             p->noise_kinv, w->red, twiddles_of(p, g.ny), twiddles_of(p, g.nx), s));
  p->noise_logdet.assign(p->nsky, 0.0);
  FR_CUDA_TRY(cudaMemcpyAsync(p->noise_logdet.data(), w->red, p->nsky * sizeof(double),
                              cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  p->noise_eps = eps_noise;
  p->has_noise = true;
  if (logdet) std::copy(p->noise_logdet.begin(), p->noise_logdet.end(), logdet);
  return FR_OK;
}

int fr_noise_kernel(fr_plan_t p, float* K, void* stream) {
  if (!p || !K) {
    set_error("plan and K must be non-null");
    return FR_EINVAL;
  }
  if (!p->has_noise) {
    set_error("no noise kernel: call fr_noise_fit first");
    return FR_EINVAL;
  }
  const size_t n = (size_t)p->nsky * p->geo.nx * p->geo.ny;
  kernel_from_inverse<<<nblocks(n), RED_T, 0, (cudaStream_t)stream>>>(p->noise_kinv, p->nsky,
                                                                       p->geo.nx, p->geo.ny, K);
  FR_LAUNCHED();
  return FR_OK;
}

int fr_noise_apply_inverse(fr_plan_t p, const float* x, int32_t batch, float* out, void* stream) {
  if (!p || !x || !out || batch < 1) {
    set_error("plan, x, out must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  if (!p->has_noise) {
    set_error("no noise kernel: call fr_noise_fit first");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const Geometry& g = p->geo;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  const int nimg = batch * p->nsky;
  const size_t n = (size_t)nimg * g.nx * g.ny;
  FR_TRY(ws_reserve_h(w, 2 * n));
  return noise_inverse_passes(x, g.nx, g.ny, nimg, p->nsky, p->noise_kinv, w->h, w->h + n, out,
                              1.f, nullptr, nullptr, twiddles_of(p, g.ny), twiddles_of(p, g.nx), s);
}

int fr_fast_likelihood_grad(fr_plan_t p, const float* sky, const float* dirty, int32_t batch,
                            float* grad, double* value, void* stream) {
  return fr_fast_likelihood_grad_resid(p, sky, dirty, batch, grad, nullptr, value, stream);
}

int fr_fast_likelihood_grad_resid(fr_plan_t p, const float* sky, const float* dirty,
                                  int32_t batch, float* grad, float* ninv_resid, double* value,
                                  void* stream) {
  if (!p || !sky || !dirty || !grad || batch < 1) {
    set_error("plan, sky, dirty, grad must be non-null and batch >= 1");
    return FR_EINVAL;
  }
  if (!p->has_noise) {
    set_error("no noise kernel: call fr_noise_fit first");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const Geometry& g = p->geo;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  const int nimg = batch * p->nsky;
  const size_t n = (size_t)nimg * g.nx * g.ny;
  FR_TRY(ws_reserve_imgs(w, n));
  // spectra scratch for both the PSF passes and the noise passes (2 nimg nx ny complex)
  FR_TRY(ws_reserve_h(w, std::max(psf_h_need(p, nimg), 2 * n)));
  FR_TRY(ws_reserve_red(w, (size_t)std::max(batch, 4)));
  // t = PSF * sky - dirty = -r (Sec. 3.3.2 response)
  FR_TRY(psf_common(p, sky, batch, w->img_a, dirty, nullptr, s));
  FR_CUDA_TRY(cudaMemsetAsync(w->red, 0, batch * sizeof(double), s));
  // u = N'^-1 t = -N'^-1 r and H = 1/2 t . u = 1/2 r^T N'^-1 r (Eq. ham_new)
  FR_TRY(noise_inverse_passes(w->img_a, g.nx, g.ny, nimg, p->nsky, p->noise_kinv, w->h,
                              w->h + n, w->img_b, 1.f, w->img_a, w->red, twiddles_of(p, g.ny),
                              twiddles_of(p, g.nx), s));
  // grad = -PSF * (N'^-1 r) = PSF * u (the PSF passes without a dirty image leave red alone)
  FR_TRY(psf_common(p, w->img_b, batch, grad, nullptr, nullptr, s));
  if (ninv_resid) {  // N'^-1 r = -u
    ProfScope ps(PC_REDUCE, s, (double)n * 8.0);
    negate_kernel<<<nblocks(n), RED_T, 0, s>>>(w->img_b, n, ninv_resid);
    FR_LAUNCHED();
  }
  if (value) {
    FR_CUDA_TRY(cudaMemcpyAsync(value, w->red, batch * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FR_OK;
}

int fr_major_cycle(fr_plan_t p, const float* sky, const float* dirty, float* resid,
                   double* resid_norm2, const fr_cf32* vis, double* vis_chi2, void* stream) {
  if (!p || !sky) {
    set_error("plan and sky must be non-null");
    return FR_EINVAL;
  }
  if ((resid || resid_norm2) && !dirty) {
    set_error("dirty is required for the image residual");
    return FR_EINVAL;
  }
  if (vis_chi2 && !vis) {
    set_error("vis is required for vis_chi2");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w;
  FR_TRY(get_ws(p, s, &w));
  FR_TRY(ws_reserve_tmp(p, w));
  FR_TRY(ws_reserve_red(w, 4));
  FR_CUDA_TRY(cudaMemsetAsync(w->red, 0, 2 * sizeof(double), s));
  FR_TRY(run_degrid(p, p->geo, p->lay, w, sky, w->tmp_vis, s));
  if (vis_chi2 && p->lay.nsorted > 0) {
    ProfScope ps(PC_REDUCE, s, (double)p->lay.nsorted * 24.0);
    chi2_kernel<<<nblocks(p->lay.nsorted), RED_T, 0, s>>>((const float2*)vis, w->tmp_vis, p->lay.wgt,
                                                          p->lay.perm, p->lay.nsorted, w->red + 1);
    FR_LAUNCHED();
  }
  const size_t n = (size_t)p->nsky * p->geo.nx * p->geo.ny;
  if (resid || resid_norm2) {
    FR_TRY(run_grid(p, p->geo, p->lay, w, w->tmp_vis, 1, w->tmp_img, w->grid, w->b1g, w->vbuf, s,
                    &w->grid_zero));
    float* r = resid ? resid : w->tmp_img;
    FR_TRY(sub_images(dirty, w->tmp_img, r, n, s));
    if (resid_norm2) FR_TRY(dot_images(r, nullptr, n, 1.0, w->red, s));
  }
  if (resid_norm2 || vis_chi2) {
    double h[2];
    FR_CUDA_TRY(cudaMemcpyAsync(h, w->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    if (resid_norm2) *resid_norm2 = h[0];
    if (vis_chi2) *vis_chi2 = h[1];
  }
  return FR_OK;
}

int fr_plan_get_info(fr_plan_t p, fr_plan_info* info) {
  if (!p || !info) {
    set_error("plan and info must be non-null");
    return FR_EINVAL;
  }
  std::memset(info, 0, sizeof *info);
  info->nx = p->geo.nx;
  info->ny = p->geo.ny;
  info->nsky = p->nsky;
  info->nchan = p->nchan;
  info->nrow = p->nrow;
  info->nvis = p->lay.nvis;
  info->grid_nu = p->geo.Nu;
  info->grid_nv = p->geo.Nv;
  info->support = p->geo.kern.W;
  info->beta = p->geo.beta;
  int tot = 0, mx = 0;
  for (int g = 0; g < p->lay.ngroups; ++g) {
    const int P = p->geo.wterm ? p->lay.planes[g] : 1;
    tot += P;
    mx = std::max(mx, P);
  }
  info->wplanes_total = tot;
  info->wplanes_max = mx;
  info->dw = (p->geo.wterm && !p->geo.taylor) ? p->geo.dw : 0.0;  // 0: no w-term or expansion
  info->nvis_dropped = p->lay.ndropped;
  info->work_items = p->lay.nitems;
  info->flags = p->flags;
  return FR_OK;
}

int fr_plan_footprint(fr_plan_t p, size_t* resident_bytes, size_t* workspace_bytes) {
  if (!p) {
    set_error("plan must be non-null");
    return FR_EINVAL;
  }
  if (resident_bytes) *resident_bytes = p->resident;
  if (workspace_bytes) {
    std::lock_guard<std::mutex> lk(p->mu);
    size_t m = 0;
    for (Workspace* w : p->ws) m = std::max(m, w->bytes);
    if (p->ws.empty()) {
      const Geometry& g = p->geo;
      m = (2 * (size_t)g.nx * g.Nv + (size_t)g.Nu * g.Nv +
           (size_t)std::max<int64_t>(p->lay.nsorted, 1)) *
          sizeof(float2);
      if (use_term_grids(g))
        m += 2 * (size_t)g.nterms * (g.Nu + g.nx) * g.Nv * sizeof(float2);
      if (p->flags & FR_DETERMINISTIC)  // fixed-point grid(s)
        m += (use_term_grids(g) ? (size_t)g.nterms : 1) * g.Nu * g.Nv * sizeof(longlong2);
      if (use_stack(p))  // compact half planes of the stacked w-plane passes
        m += (size_t)STACK_K * std::max<size_t>((size_t)p->lay.occ_max_rows * TILE * g.nx, 1) *
             sizeof(float2);
    }
    *workspace_bytes = m;
  }
  return FR_OK;
}

int fr_plan_check(fr_plan_t p, void* stream) {
  if (!p) {
    set_error("plan must be non-null");
    return FR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  FR_CUDA_TRY(cudaMemcpyAsync(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  if (st) {
    FR_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    set_error("a bounded device-side wait gave up (status %d)", st);
    return FR_ETIMEOUT;
  }
  return FR_OK;
}

int fr_selftest_wait_timeout(fr_plan_t p, void* stream) {
  if (!p) {
    set_error("plan must be non-null");
    return FR_EINVAL;
  }
  return selftest_wait_timeout(p->status, (cudaStream_t)stream);
}

int fr_selftest_fft_host(float* data, int32_t n, int32_t batch, int32_t dir) {
  if (!data || n < 2 || n > 16384 || batch < 1 || (dir != 1 && dir != -1 && dir != 2 && dir != -2) ||
      strip_factor(strip_factor(odd_part(n), 5), 3) != 1) {
    set_error("bad arguments to fr_selftest_fft_host");
    return FR_EINVAL;
  }
  const int L = n;
  std::vector<float2> tw(L), a(spad_len(L)), b(spad_len(L));
  for (int m = 0; m < L; ++m) {
    const double ang = -2.0 * M_PI * (double)m / (double)L;
    tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  for (int q = 0; q < batch; ++q) {
    float2* x = reinterpret_cast<float2*>(data) + (size_t)q * L;
    for (int i = 0; i < L; ++i) a[spad(i)] = x[i];
    const int P = (dir == 2 || dir == -2) ? 32 : 16;
    if (dir < 0)
      host_fft<-1>(a.data(), b.data(), tw.data(), L, P);
    else
      host_fft<1>(a.data(), b.data(), tw.data(), L, P);
    for (int i = 0; i < L; ++i) x[i] = a[spad(i)];
  }
  return FR_OK;
}

}  // extern "C"
