// Visibility-side kernels of R and R^dag N^-1 (Eq. rime, Eq. clean):
//   * plan-time coordinate scaling k = uvw nu / c in FP64, w-plane assignment, tile keys and a
//     counting sort into (image group, tile, first w-plane) order, plus the (tile, plane) work
//     items (a1);
//   * the degridder: per (tile, plane) work item one CTA stages the grid tile with a TMA bulk
//     tensor copy into shared memory and each thread interpolates one visibility with the
//     separable kernel phi(du) phi(dv) phi(dw) (a4);
//   * the gridder: per work item one CTA accumulates its visibilities into a shared-memory
//     sub-grid and flushes the non-zero cells to the global grid with vector atomics (a5);
//   * per-pixel correction tables (grid correction, 1/n, w-plane phase coordinate).
// The gridding kernel is the exponential of a semicircle; its Fourier transform corrects the
// image side. The paper names the wgridder for this operator but does not describe it.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "fr_internal.cuh"
#include "vis_common.cuh"

namespace fr {

static constexpr double C_LIGHT = 299792458.0;

// ---------------------------------------------------------------------------------- scan
// Exclusive prefix sum of int32 counts: out[0..n] with out[n] = total.
static constexpr int SCAN_BLK = 1024, SCAN_PER = 4, SCAN_TILE = SCAN_BLK * SCAN_PER;

__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[SCAN_BLK / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int before = (wid > 0 ? ws[wid - 1] : 0) + x - v;
  *total = ws[SCAN_BLK / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(SCAN_BLK) scan_reduce(const int* in, int64_t n, int* bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
  int s = 0;
  for (int k = 0; k < SCAN_PER; ++k)
    if (base + k < n) s += in[base + k];
  int tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_BLK) scan_blocks(int* bsum, int nb) {
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += SCAN_BLK) {
    int i = b0 + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    int tot;
    int ex = block_excl_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_BLK) scan_final(const int* in, int64_t n, const int* bsum,
                                                       int* out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
  int v[SCAN_PER];
  int s = 0;
  for (int k = 0; k < SCAN_PER; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_excl_scan(s, &tot) + bsum[blockIdx.x];
  for (int k = 0; k < SCAN_PER; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bsum[gridDim.x];
}

static int exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t s) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (n == 0) {
    FR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), s));
    return FR_OK;
  }
  int* bsum = nullptr;
  FR_CUDA_TRY(cudaMallocAsync(&bsum, (nb + 1) * sizeof(int), s));
  scan_reduce<<<(unsigned)nb, SCAN_BLK, 0, s>>>(in, n, bsum);
  FR_LAUNCHED();
  scan_blocks<<<1, SCAN_BLK, 0, s>>>(bsum, (int)nb);
  FR_LAUNCHED();
  scan_final<<<(unsigned)nb, SCAN_BLK, 0, s>>>(in, n, bsum, out);
  FR_LAUNCHED();
  FR_CUDA_TRY(cudaFreeAsync(bsum, s));
  return FR_OK;
}

// ------------------------------------------------------------------------ coordinates
struct PrepArgs {
  const double* uvw;
  const double* freqs;
  const float* weights;
  int64_t nrow;
  int nchan, ngroups;
  int Nu, Nv, W;
  double dl, dm;
  int wterm;
  int taylor;            // small-w expansion: every visibility in every term, dw_out = a
  double a_scale;        // 2 pi t_half (a = a_scale * w)
  double t_c, dw;
  const double* w_lo;    // [ngroups]
  const int* planes;     // [ngroups]
  const int* keybase;    // [ngroups]
  int ntu, ntv;
  int ntb;               // row blocks per (tile, plane) bucket
  int64_t rows_per_tb;
  int drop;
  // outputs in user order
  int* key;              // -1 = dropped
  uint32_t* cell;
  float* du;
  float* dv;
  float* dw_out;
  uint32_t* ph;
  float* wgt;
  int* err;              // bit 1: footprint outside the grid, bit 2: bad coordinate
  unsigned long long* ndrop;
};

__global__ void vis_prepare(PrepArgs a) {
  const int64_t M = a.nrow * a.nchan;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = k / a.nchan;
    const int c = (int)(k - row * a.nchan);
    const int g = a.ngroups == 1 ? 0 : c;
    const double f = a.freqs[c] / C_LIGHT;
    double u = a.uvw[3 * row] * f, v = a.uvw[3 * row + 1] * f, w = a.uvw[3 * row + 2] * f;
    if (a.wterm && w < 0.0) {  // V(-u,-v,-w) = conj V(u,v,w) for a real sky
      u = -u;
      v = -v;
      w = -w;
    }
    const double gu = u * a.Nu * a.dl + 0.5 * a.Nu;
    const double gv = v * a.Nv * a.dm + 0.5 * a.Nv;
    const double hw = 0.5 * a.W;
    bool ok = isfinite(gu) && isfinite(gv) && isfinite(w);
    double iu0 = 0, iv0 = 0;
    if (ok) {
      iu0 = ceil(gu - hw);
      iv0 = ceil(gv - hw);
      ok = iu0 >= 0.0 && iu0 + a.W - 1 <= a.Nu - 1 && iv0 >= 0.0 && iv0 + a.W - 1 <= a.Nv - 1;
    }
    int pf = 0;
    double dwv = 0.0;
    if (ok && a.wterm && a.taylor) {
      dwv = a.a_scale * w;
    } else if (ok && a.wterm) {
      const double y = (w - a.w_lo[g]) / a.dw + hw;
      pf = (int)ceil(y - hw);
      if (pf < 0) pf = 0;
      if (pf > a.planes[g] - a.W) pf = a.planes[g] - a.W;
      dwv = y - pf;
    }
    if (!ok) {
      a.key[k] = -1;
      if (a.drop)
        atomicAdd(a.ndrop, 1ull);
      else
        atomicOr(a.err, 1);
      continue;
    }
    const int ju = (int)iu0, jv = (int)iv0;
    const int tu = ju / TILE, tv = jv / TILE;
    const int P = (a.wterm && !a.taylor) ? a.planes[g] : 1;
    const int tb = (int)min((int64_t)a.ntb - 1, row / a.rows_per_tb);
    a.key[k] = a.keybase[g] + ((tu * a.ntv + tv) * P + pf) * a.ntb + tb;
    a.cell[k] = ((uint32_t)ju << 18) | ((uint32_t)jv << 4) | (uint32_t)(pf & 15);
    a.du[k] = (float)(gu - iu0);
    a.dv[k] = (float)(gv - iv0);
    if (a.wterm) {
      a.dw_out[k] = (float)dwv;
      const double x = w * a.t_c;
      const double fr = x - rint(x);
      a.ph[k] = (uint32_t)(long long)llrint(fr * 4294967296.0);
    }
    a.wgt[k] = a.weights ? a.weights[k] : 1.f;
  }
}

__global__ void count_keys(const int* key, int64_t M, int* count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    int kk = key[k];
    if (kk >= 0) atomicAdd(&count[kk], 1);
  }
}

struct ScatterArgs {
  const int* key;
  int64_t M;
  int nchan;
  int* cursor;
  int wterm;
  const double* uvw;
  const double* freqs;
  const uint32_t* cell_in;
  const float* du_in;
  const float* dv_in;
  const float* dw_in;
  const uint32_t* ph_in;
  const float* wgt_in;
  uint32_t* cell;
  float* du;
  float* dv;
  float* dw;
  uint32_t* ph;
  float* wgt;
  uint32_t* perm;
};

__global__ void scatter_sorted(ScatterArgs a) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int kk = a.key[k];
    if (kk < 0) continue;
    const int pos = atomicAdd(&a.cursor[kk], 1);
    a.cell[pos] = a.cell_in[k];
    a.du[pos] = a.du_in[k];
    a.dv[pos] = a.dv_in[k];
    a.wgt[pos] = a.wgt_in[k];
    uint32_t flip = 0;
    if (a.wterm) {
      a.dw[pos] = a.dw_in[k];
      a.ph[pos] = a.ph_in[k];
      const int64_t row = k / a.nchan;
      flip = a.uvw[3 * row + 2] < 0.0 ? 1u : 0u;
    }
    a.perm[pos] = (uint32_t)k | (flip << 31);
  }
}

// number of work-item chunks of every (group, plane, tile)
struct ItemArgs {
  const int* off;        // key offsets [K + 1]
  const int* keybase;    // [ngroups]
  const int* planes;     // [ngroups] (1 without w)
  const int64_t* ebase;  // [ngroups + 1] (group, plane, tile) enumeration base
  int ngroups, ntiles, ntv, W, wterm, ntb, chunk;
  int* chunks;           // [E]
  const int* item_off;   // [E + 1] (emit pass)
  int4* items;
};

__device__ __forceinline__ void item_range(const ItemArgs& a, int64_t e, int* begin, int* count,
                                           int* tile) {
  int g = 0;
  while (g + 1 < a.ngroups && e >= a.ebase[g + 1]) ++g;
  const int64_t r = e - a.ebase[g];
  const int P = a.planes[g];
  const int p = (int)(r / a.ntiles);
  const int t = (int)(r - (int64_t)p * a.ntiles);
  *tile = t;
  int lo, hi;
  if (a.wterm) {
    lo = max(p - a.W + 1, 0);
    hi = min(p, P - a.W);
  } else {
    lo = 0;
    hi = 0;
  }
  if (hi < lo) {
    *begin = 0;
    *count = 0;
    return;
  }
  const int64_t kb = (int64_t)a.keybase[g] + (int64_t)t * P * a.ntb;
  *begin = a.off[kb + (int64_t)lo * a.ntb];
  *count = a.off[kb + (int64_t)(hi + 1) * a.ntb] - *begin;
}

__global__ void count_items(ItemArgs a, int64_t E) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b, c, t;
    item_range(a, e, &b, &c, &t);
    a.chunks[e] = (c + a.chunk - 1) / a.chunk;
  }
}

__global__ void emit_items(ItemArgs a, int64_t E) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int b, c, t;
    item_range(a, e, &b, &c, &t);
    if (c == 0) continue;
    const int tu = t / a.ntv, tv = t - (t / a.ntv) * a.ntv;
    int o = a.item_off[e];
    for (int s = 0; s < c; s += a.chunk, ++o)
      a.items[o] = make_int4(b + s, min(a.chunk, c - s), (tu << 16) | tv, 0);
  }
}

// bounds of the footprint origins: band = {min iu0, max iu0, min iv0, max iv0}
__global__ void band_kernel(const uint32_t* cell, int64_t n, int* band) {
  int a = 1 << 30, b = -1, c = 1 << 30, d = -1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = cell[i];
    const int u = (int)(x >> 18), v = (int)((x >> 4) & 0x3fff);
    a = min(a, u);
    b = max(b, u);
    c = min(c, v);
    d = max(d, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = min(a, __shfl_down_sync(0xffffffffu, a, o));
    b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    c = min(c, __shfl_down_sync(0xffffffffu, c, o));
    d = max(d, __shfl_down_sync(0xffffffffu, d, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&band[0], a);
    atomicMax(&band[1], b);
    atomicMin(&band[2], c);
    atomicMax(&band[3], d);
  }
}

__global__ void plane_visits_kernel(const int4* items, const int* pitems, long long* out) {
  const int q = blockIdx.x;
  long long s = 0;
  for (int i = pitems[q] + threadIdx.x; i < pitems[q + 1]; i += blockDim.x) s += items[i].y;
  __shared__ long long sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[q] = sh[0];
}

__global__ void gather_plane_items(const int* item_off, const int64_t* qpos, int nq, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nq) out[i] = item_off[qpos[i]];
}

static unsigned grid1d(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// allocation of plan data; stream-ordered when `async` is set (transient layouts and tables)
template <class T>
static int dalloc(T** p, size_t n, size_t* acc, cudaStream_t async = nullptr) {
  *p = nullptr;
  if (n == 0) return FR_OK;
  cudaError_t e = async ? cudaMallocAsync((void**)p, n * sizeof(T), async)
                        : cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
    *p = nullptr;
    return FR_ENOMEM;
  }
  if (acc) *acc += n * sizeof(T);
  return FR_OK;
}

void free_layout(VisLayout* lay) {
  for (void* q : {(void*)lay->cell, (void*)lay->du, (void*)lay->dv, (void*)lay->dw, (void*)lay->ph,
                  (void*)lay->perm, (void*)lay->wgt, (void*)lay->items, (void*)lay->occ_bits,
                  (void*)lay->occ_comp, (void*)lay->occ_rows}) {
    if (!q) continue;
    if (lay->async)
      cudaFreeAsync(q, lay->async);
    else
      cudaFree(q);
  }
  lay->cell = nullptr;
  lay->du = lay->dv = lay->dw = lay->wgt = nullptr;
  lay->ph = lay->perm = nullptr;
  lay->items = nullptr;
  lay->occ_bits = nullptr;
  lay->occ_comp = nullptr;
  lay->occ_rows = nullptr;
  lay->occ_ok = false;
}

PlaneOcc plane_occ(const VisLayout& lay, int q) {
  PlaneOcc o;
  if (!lay.occ_ok) return o;
  o.rows = lay.occ_rows + lay.occ_row_off[q];
  o.comp = lay.occ_comp + (size_t)q * lay.ntv;
  o.bits = lay.occ_bits + (size_t)q * lay.ntv * lay.occ_ntw;
  o.nrows = (int)(lay.occ_row_off[q + 1] - lay.occ_row_off[q]);
  o.ntw = lay.occ_ntw;
  o.ncells = (double)lay.occ_tiles[q] * TILE * TILE;
  return o;
}

// w-stacking: the tiles plane q's footprints reach. A work item of tile (tu, tv) holds
// footprints whose origin lies in that tile; a footprint of W <= TILE cells reaches at most the
// next tile in u and in v, so the item marks the 2 x 2 tiles from its own (clipped to the grid).
__global__ void occupancy_kernel(const int4* __restrict__ items, int64_t nitems,
                                 const int* __restrict__ pitems, int nplanes, int ntu, int ntv,
                                 int ntw, uint32_t* bits) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nitems;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nplanes - 1;  // plane q: pitems[q] <= i < pitems[q + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pitems[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int4 it = items[i];
    if (it.y <= 0) continue;
    const int tu = it.z >> 16, tv = it.z & 0xffff;
    uint32_t* b = bits + (size_t)lo * ntv * ntw;
    for (int dv = 0; dv < 2; ++dv)
      for (int du = 0; du < 2; ++du) {
        const int u = tu + du, v = tv + dv;
        if (u < ntu && v < ntv) atomicOr(&b[v * ntw + (u >> 5)], 1u << (u & 31));
      }
  }
}

static int build_occupancy(VisLayout* lay, const int* d_pitems, int nplanes, size_t* acc,
                           cudaStream_t s) {
  const int ntw = (lay->ntu + 31) / 32;
  const size_t nbits = (size_t)nplanes * lay->ntv * ntw;
  lay->occ_ntw = ntw;
  FR_TRY(dalloc(&lay->occ_bits, nbits, acc, lay->async));
  FR_CUDA_TRY(cudaMemsetAsync(lay->occ_bits, 0, nbits * sizeof(uint32_t), s));
  if (lay->nitems > 0) {
    occupancy_kernel<<<grid1d(lay->nitems), 256, 0, s>>>(lay->items, lay->nitems, d_pitems,
                                                          nplanes, lay->ntu, lay->ntv, ntw,
                                                          lay->occ_bits);
    FR_LAUNCHED();
  }
  std::vector<uint32_t> hb(nbits);
  FR_CUDA_TRY(cudaMemcpyAsync(hb.data(), lay->occ_bits, nbits * sizeof(uint32_t),
                              cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int> comp((size_t)nplanes * lay->ntv, -1), rows;
  lay->occ_row_off.assign(nplanes + 1, 0);
  lay->occ_tiles.assign(nplanes, 0);
  lay->occ_max_rows = 0;
  for (int q = 0; q < nplanes; ++q) {
    int n = 0;
    for (int v = 0; v < lay->ntv; ++v) {
      int64_t c = 0;
      for (int w = 0; w < ntw; ++w) c += __builtin_popcount(hb[((size_t)q * lay->ntv + v) * ntw + w]);
      if (c == 0) continue;
      comp[(size_t)q * lay->ntv + v] = n++;
      rows.push_back(v);
      lay->occ_tiles[q] += c;
    }
    lay->occ_row_off[q + 1] = (int64_t)rows.size();
    lay->occ_max_rows = std::max(lay->occ_max_rows, n);
  }
  FR_TRY(dalloc(&lay->occ_comp, comp.size(), acc, lay->async));
  FR_TRY(dalloc(&lay->occ_rows, std::max<size_t>(rows.size(), 1), acc, lay->async));
  FR_CUDA_TRY(cudaMemcpyAsync(lay->occ_comp, comp.data(), comp.size() * sizeof(int),
                              cudaMemcpyHostToDevice, s));
  if (!rows.empty())
    FR_CUDA_TRY(cudaMemcpyAsync(lay->occ_rows, rows.data(), rows.size() * sizeof(int),
                                cudaMemcpyHostToDevice, s));
  // the host vectors are read by the copies above: finish them before they go out of scope
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  lay->occ_ok = true;
  return FR_OK;
}

namespace {
// RAII holder of plan-time temporaries, stream-ordered (cudaMallocAsync / cudaFreeAsync) so that
// building a plan never synchronises the device: other streams keep running meanwhile
struct Temps {
  cudaStream_t s;
  std::vector<void*> p;
  explicit Temps(cudaStream_t st) : s(st) {}
  ~Temps() {
    for (void* q : p) cudaFreeAsync(q, s);
  }
  template <class T>
  int alloc(T** out, size_t n) {
    *out = nullptr;
    if (n == 0) return FR_OK;
    cudaError_t e = cudaMallocAsync((void**)out, n * sizeof(T), s);
    if (e != cudaSuccess) {
      set_error("cudaMallocAsync of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
      *out = nullptr;
      return FR_ENOMEM;
    }
    p.push_back(*out);
    return FR_OK;
  }
};
}  // namespace

static int presort_items(VisLayout* lay, int64_t N, bool wterm, cudaStream_t s,
                         const int4* sort_items, int64_t nsort);

int build_layout(const Geometry& geo, const double* d_uvw, int64_t nrow, const double* h_freqs,
                 const double* d_freqs, int nchan, const float* d_weights, int ngroups,
                 const std::vector<double>& w_lo, const std::vector<int>& planes, bool drop_oob,
                 VisLayout* lay, cudaStream_t s) {
  (void)h_freqs;
  const int64_t M = nrow * (int64_t)nchan;
  lay->ngroups = ngroups;
  lay->ntu = (geo.Nu + TILE - 1) / TILE;
  lay->ntv = (geo.Nv + TILE - 1) / TILE;
  lay->planes = planes;
  lay->w_lo = w_lo;
  lay->nvis = M;
  const int ntiles = lay->ntu * lay->ntv;
  const bool wterm = geo.wterm;
  // w-stacking splits visibilities by first w-plane; the small-w expansion puts every
  // visibility in every term, so its layout has one plane dimension like the w = 0 case
  const bool stack = geo.wterm && !geo.taylor;

  // keys: (group, tile, first plane, row block). Row blocks keep each bucket to a narrow range
  // of rows, i.e. of times for time-ordered data, so a work item holds consecutive samples of
  // the baselines crossing its tile, which stay in one grid cell for many samples.
  int64_t kbase = 0;
  for (int g = 0; g < ngroups; ++g) kbase += (int64_t)ntiles * (stack ? planes[g] : 1);
  const int ntb = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(nrow, 4096),
                                                              (int64_t(1) << 26) / std::max<int64_t>(kbase, 1)));
  const int64_t rows_per_tb = (nrow + ntb - 1) / ntb;
  std::vector<int> keybase(ngroups);
  int64_t K = 0;
  std::vector<int64_t> ebase(ngroups + 1);
  int64_t E = 0;
  for (int g = 0; g < ngroups; ++g) {
    const int P = stack ? planes[g] : 1;
    keybase[g] = (int)K;
    K += (int64_t)ntiles * P * ntb;
    ebase[g] = E;
    E += (int64_t)ntiles * P;
  }
  ebase[ngroups] = E;
  if (K >= (1ll << 31) || M >= (1ll << 31)) {
    set_error("problem too large: %lld keys, %lld visibilities", (long long)K, (long long)M);
    return FR_EUNSUPPORTED;
  }

  Temps t(s);
  int *d_key, *d_count, *d_off, *d_keybase, *d_planes, *d_err;
  double* d_wlo;
  int64_t* d_ebase;
  unsigned long long* d_ndrop;
  uint32_t *cell_u, *ph_u = nullptr;
  float *du_u, *dv_u, *dw_u = nullptr, *wgt_u;
  FR_TRY(t.alloc(&d_key, M));
  FR_TRY(t.alloc(&d_count, K));
  FR_TRY(t.alloc(&d_off, K + 1));
  FR_TRY(t.alloc(&d_keybase, ngroups));
  FR_TRY(t.alloc(&d_planes, ngroups));
  FR_TRY(t.alloc(&d_wlo, ngroups));
  FR_TRY(t.alloc(&d_ebase, ngroups + 1));
  FR_TRY(t.alloc(&d_err, 1));
  FR_TRY(t.alloc(&d_ndrop, 1));
  FR_TRY(t.alloc(&cell_u, M));
  FR_TRY(t.alloc(&du_u, M));
  FR_TRY(t.alloc(&dv_u, M));
  FR_TRY(t.alloc(&wgt_u, M));
  if (wterm) {
    FR_TRY(t.alloc(&dw_u, M));
    FR_TRY(t.alloc(&ph_u, M));
  }
  std::vector<int> pl(ngroups);
  for (int g = 0; g < ngroups; ++g) pl[g] = stack ? planes[g] : 1;
  FR_CUDA_TRY(cudaMemcpyAsync(d_keybase, keybase.data(), ngroups * sizeof(int), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_planes, pl.data(), ngroups * sizeof(int), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_wlo, w_lo.data(), ngroups * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_ebase, ebase.data(), (ngroups + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  FR_CUDA_TRY(cudaMemsetAsync(d_ndrop, 0, sizeof(unsigned long long), s));
  FR_CUDA_TRY(cudaMemsetAsync(d_count, 0, K * sizeof(int), s));

  PrepArgs pa;
  pa.uvw = d_uvw;
  pa.freqs = d_freqs;
  pa.weights = d_weights;
  pa.nrow = nrow;
  pa.nchan = nchan;
  pa.ngroups = ngroups;
  pa.Nu = geo.Nu;
  pa.Nv = geo.Nv;
  pa.W = geo.kern.W;
  pa.dl = geo.dl;
  pa.dm = geo.dm;
  pa.wterm = wterm;
  pa.taylor = geo.taylor ? 1 : 0;
  pa.a_scale = 2.0 * M_PI * geo.t_half;
  pa.t_c = geo.t_c;
  pa.dw = geo.dw;
  pa.w_lo = d_wlo;
  pa.planes = d_planes;
  pa.keybase = d_keybase;
  pa.ntu = lay->ntu;
  pa.ntv = lay->ntv;
  pa.ntb = ntb;
  pa.rows_per_tb = rows_per_tb;
  pa.drop = drop_oob;
  pa.key = d_key;
  pa.cell = cell_u;
  pa.du = du_u;
  pa.dv = dv_u;
  pa.dw_out = dw_u;
  pa.ph = ph_u;
  pa.wgt = wgt_u;
  pa.err = d_err;
  pa.ndrop = d_ndrop;
  vis_prepare<<<grid1d(M), 256, 0, s>>>(pa);
  FR_LAUNCHED();
  count_keys<<<grid1d(M), 256, 0, s>>>(d_key, M, d_count);
  FR_LAUNCHED();
  FR_TRY(exclusive_scan(d_count, d_off, K, s));

  int h_err = 0;
  unsigned long long h_ndrop = 0;
  int h_total = 0;
  FR_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaMemcpyAsync(&h_ndrop, d_ndrop, sizeof(h_ndrop), cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaMemcpyAsync(&h_total, d_off + K, sizeof(int), cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_err) {
    set_error("visibility coordinates outside the oversampled grid or not finite "
              "(|u| must stay below about (1 - (W+2)/Nu) / (2 pixsize)); use FR_DROP_OOB to drop them");
    return FR_EINVAL;
  }
  lay->ndropped = (int64_t)h_ndrop;
  lay->nsorted = h_total;
  {
    std::vector<int> gb(ngroups + 1);
    for (int g = 0; g < ngroups; ++g)
      FR_CUDA_TRY(cudaMemcpyAsync(&gb[g], d_off + keybase[g], sizeof(int), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    gb[ngroups] = h_total;
    lay->group_begin.assign(gb.begin(), gb.end());
  }
  const int64_t N = h_total;

  size_t acc = 0;
  FR_TRY(dalloc(&lay->cell, N, &acc, lay->async));
  FR_TRY(dalloc(&lay->du, N, &acc, lay->async));
  FR_TRY(dalloc(&lay->dv, N, &acc, lay->async));
  FR_TRY(dalloc(&lay->wgt, N, &acc, lay->async));
  FR_TRY(dalloc(&lay->perm, N, &acc, lay->async));
  if (wterm) {
    FR_TRY(dalloc(&lay->dw, N, &acc, lay->async));
    FR_TRY(dalloc(&lay->ph, N, &acc, lay->async));
  }
  // cursor = offsets (reuse the count buffer)
  FR_CUDA_TRY(cudaMemcpyAsync(d_count, d_off, K * sizeof(int), cudaMemcpyDeviceToDevice, s));
  ScatterArgs sa;
  sa.key = d_key;
  sa.M = M;
  sa.nchan = nchan;
  sa.cursor = d_count;
  sa.wterm = wterm;
  sa.uvw = d_uvw;
  sa.freqs = d_freqs;
  sa.cell_in = cell_u;
  sa.du_in = du_u;
  sa.dv_in = dv_u;
  sa.dw_in = dw_u;
  sa.ph_in = ph_u;
  sa.wgt_in = wgt_u;
  sa.cell = lay->cell;
  sa.du = lay->du;
  sa.dv = lay->dv;
  sa.dw = lay->dw;
  sa.ph = lay->ph;
  sa.wgt = lay->wgt;
  sa.perm = lay->perm;
  scatter_sorted<<<grid1d(M), 256, 0, s>>>(sa);
  FR_LAUNCHED();

  // work items per (group, plane, tile)
  int *d_chunks, *d_item_off;
  FR_TRY(t.alloc(&d_chunks, E));
  FR_TRY(t.alloc(&d_item_off, E + 1));
  ItemArgs ia;
  ia.off = d_off;
  ia.keybase = d_keybase;
  ia.planes = d_planes;
  ia.ebase = d_ebase;
  ia.ngroups = ngroups;
  ia.ntiles = ntiles;
  ia.ntv = lay->ntv;
  ia.ntb = ntb;
  ia.W = geo.kern.W;
  ia.chunk = stack ? STACK_CHUNK : ITEM_CHUNK;
  ia.wterm = stack;
  ia.chunks = d_chunks;
  ia.item_off = d_item_off;
  ia.items = nullptr;
  count_items<<<grid1d(E), 256, 0, s>>>(ia, E);
  FR_LAUNCHED();
  FR_TRY(exclusive_scan(d_chunks, d_item_off, E, s));
  // plane boundaries (g, p) -> item index
  std::vector<int64_t> qpos;
  lay->plane_base.assign(ngroups, 0);
  for (int g = 0; g < ngroups; ++g) {
    lay->plane_base[g] = (int)qpos.size();
    for (int p = 0; p < pl[g]; ++p) qpos.push_back(ebase[g] + (int64_t)p * ntiles);
  }
  qpos.push_back(E);
  const int nq = (int)qpos.size();
  int64_t* d_qpos;
  int* d_pitems;
  FR_TRY(t.alloc(&d_qpos, nq));
  FR_TRY(t.alloc(&d_pitems, nq));
  FR_CUDA_TRY(cudaMemcpyAsync(d_qpos, qpos.data(), nq * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  gather_plane_items<<<(nq + 255) / 256, 256, 0, s>>>(d_item_off, d_qpos, nq, d_pitems);
  FR_LAUNCHED();
  std::vector<int> pitems(nq);
  FR_CUDA_TRY(cudaMemcpyAsync(pitems.data(), d_pitems, nq * sizeof(int), cudaMemcpyDeviceToHost, s));
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  lay->plane_items.assign(pitems.begin(), pitems.end());
  lay->nitems = pitems[nq - 1];
  FR_TRY(dalloc(&lay->items, lay->nitems, &acc, lay->async));
  ia.items = lay->items;
  if (lay->nitems > 0) {
    emit_items<<<grid1d(E), 256, 0, s>>>(ia, E);
    FR_LAUNCHED();
  }
  // Without w-stacking every work item is a fixed chunk of one tile's range, so each chunk is
  // ordered by footprint origin once here instead of in every gridding call. With w-stacking a
  // plane's items span the buckets of W first planes, with chunk boundaries that differ from
  // plane to plane: there every (tile, first plane) bucket is ordered instead, in chunks of up
  // to ITEM_CHUNK, so a work item is a few origin-sorted runs and no call sorts.
  lay->presorted = false;
  if (!stack && lay->nitems > 0) {
    FR_TRY(presort_items(lay, N, wterm, s, nullptr, 0));
    lay->presorted = true;
  } else if (stack && lay->nitems > 0) {
    ItemArgs sa = ia;
    sa.W = 1;  // one first plane per range: the (group, plane, tile) buckets themselves
    sa.chunk = ITEM_CHUNK;
    int *d_sc, *d_soff;
    FR_TRY(t.alloc(&d_sc, E));
    FR_TRY(t.alloc(&d_soff, E + 1));
    sa.chunks = d_sc;
    sa.item_off = d_soff;
    count_items<<<grid1d(E), 256, 0, s>>>(sa, E);
    FR_LAUNCHED();
    FR_TRY(exclusive_scan(d_sc, d_soff, E, s));
    int nsort = 0;
    FR_CUDA_TRY(cudaMemcpyAsync(&nsort, d_soff + E, sizeof(int), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    if (nsort > 0) {
      int4* sitems;
      FR_TRY(t.alloc(&sitems, nsort));
      sa.items = sitems;
      emit_items<<<grid1d(E), 256, 0, s>>>(sa, E);
      FR_LAUNCHED();
      FR_TRY(presort_items(lay, N, wterm, s, sitems, nsort));
    }
    lay->presorted = true;
  }
  // visibility visits per (group, plane), for launch accounting
  // occupied band of the grid: the union of all kernel footprints
  {
    int* d_band;
    FR_TRY(t.alloc(&d_band, 4));
    const int init[4] = {1 << 30, -1, 1 << 30, -1};
    FR_CUDA_TRY(cudaMemcpyAsync(d_band, init, sizeof init, cudaMemcpyHostToDevice, s));
    if (N > 0) {
      band_kernel<<<grid1d(N), 256, 0, s>>>(lay->cell, N, d_band);
      FR_LAUNCHED();
    }
    int hb[4];
    FR_CUDA_TRY(cudaMemcpyAsync(hb, d_band, sizeof hb, cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    const int W = geo.kern.W;
    if (N > 0) {
      lay->bu0 = hb[0];
      lay->bu1 = std::min(geo.Nu - 1, hb[1] + W - 1);
      lay->bv0 = hb[2] & ~3;  // a multiple of 4: whole 32-byte groups in the post-pass stores
      lay->bv1 = std::min(geo.Nv - 1, hb[3] + W - 1);
    } else {
      lay->bu0 = lay->bv0 = 0;
      lay->bu1 = lay->bv1 = -1;
    }
  }
  // w-stacking on grids of whole tiles: the occupied tiles of every plane
  if (stack && geo.Nu % TILE == 0 && geo.Nv % TILE == 0)
    FR_TRY(build_occupancy(lay, d_pitems, nq - 1, &acc, s));
  lay->plane_visits.assign(nq - 1, 0);
  if (nq > 1 && lay->nitems > 0) {
    long long* d_visits;
    FR_TRY(t.alloc(&d_visits, nq - 1));
    plane_visits_kernel<<<nq - 1, 256, 0, s>>>(lay->items, d_pitems, d_visits);
    FR_LAUNCHED();
    std::vector<long long> hv(nq - 1);
    FR_CUDA_TRY(cudaMemcpyAsync(hv.data(), d_visits, (nq - 1) * sizeof(long long), cudaMemcpyDeviceToHost, s));
    FR_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < nq - 1; ++i) lay->plane_visits[i] = hv[i];
  }
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  lay->bytes = acc;
  return FR_OK;
}

// --------------------------------------------------------------------------- tables
struct TableArgs {
  int nx, ny;
  double dl, dm;
  int wterm, nterm, taylor;
  double t_c, t_half, dw;
  const double* inv_phi_u;  // [nx] 1 / Phi_u(px / Nu)
  const double* inv_phi_v;  // [ny]
  const double* gl_x;       // quadrature nodes on [-1, 1]
  const double* gl_w;
  int nq;
  double beta, hw;          // kernel shape, half width W/2
  float* corr;
  int32_t* tq;
};

__global__ void make_tables_kernel(TableArgs a) {
  const int64_t n = (int64_t)a.nx * a.ny;
  for (int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pix < n;
       pix += (int64_t)gridDim.x * blockDim.x) {
    const int jx = (int)(pix / a.ny), jy = (int)(pix - (int64_t)jx * a.ny);
    const int px = jx - a.nx / 2, py = jy - a.ny / 2;
    const double l = px * a.dl, m = py * a.dm;
    const double r2 = l * l + m * m;
    if (r2 >= 1.0) {
      a.corr[pix] = 0.f;
      if (a.tq) a.tq[pix] = 0;
      continue;
    }
    const double nn = sqrt(1.0 - r2);
    double c = a.inv_phi_u[jx] * a.inv_phi_v[jy];
    if (a.nterm) c /= nn;
    if (a.wterm) {
      const double t = -r2 / (1.0 + nn);  // n - 1 without cancellation
      const double tp = t - a.t_c;
      a.tq[pix] = (int32_t)llrint(tp / a.t_half * 1073741824.0);
      if (!a.taylor) {
        // Phi_w(dw * tp) = (W/2) int_{-1}^{1} exp(beta (sqrt(1 - z^2) - 1)) cos(pi k W z) dz
        const double k = a.dw * tp;
        double phi = 0.0;
        for (int q = 0; q < a.nq; ++q) {
          const double z = a.gl_x[q];
          phi += a.gl_w[q] * exp(a.beta * (sqrt(1.0 - z * z) - 1.0)) *
                 cos(M_PI * k * 2.0 * a.hw * z);
        }
        phi *= a.hw;
        c /= phi;
      }
    }
    if ((px + py) & 1) c = -c;
    a.corr[pix] = (float)c;
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n)
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        // recompute derivative at the converged node
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
}

// Fourier transform of the kernel at k cycles per cell (host, FP64)
double es_ft(double beta, int W, double k, const std::vector<double>& x,
             const std::vector<double>& w) {
  const double hw = 0.5 * W;
  double s = 0.0;
  for (size_t q = 0; q < x.size(); ++q)
    s += w[q] * std::exp(beta * (std::sqrt(1.0 - x[q] * x[q]) - 1.0)) * std::cos(M_PI * k * 2.0 * hw * x[q]);
  return s * hw;
}

int make_tables(Geometry* geo, const std::vector<double>& inv_phi_u,
                const std::vector<double>& inv_phi_v, cudaStream_t s) {
  const int64_t n = (int64_t)geo->nx * geo->ny;
  std::vector<double> gx, gw;
  gauss_legendre(4 * geo->kern.W + 32, gx, gw);
  Temps t(s);
  double *d_pu, *d_pv, *d_gx, *d_gw;
  FR_TRY(t.alloc(&d_pu, geo->nx));
  FR_TRY(t.alloc(&d_pv, geo->ny));
  FR_TRY(t.alloc(&d_gx, gx.size()));
  FR_TRY(t.alloc(&d_gw, gw.size()));
  FR_CUDA_TRY(cudaMemcpyAsync(d_pu, inv_phi_u.data(), geo->nx * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_pv, inv_phi_v.data(), geo->ny * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_gx, gx.data(), gx.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(d_gw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  FR_TRY(dalloc(&geo->corr, n, nullptr, geo->async));
  if (geo->wterm) FR_TRY(dalloc(&geo->tq, n, nullptr, geo->async));
  TableArgs a;
  a.nx = geo->nx;
  a.ny = geo->ny;
  a.dl = geo->dl;
  a.dm = geo->dm;
  a.wterm = geo->wterm;
  a.taylor = geo->taylor ? 1 : 0;
  a.nterm = geo->nterm;
  a.t_c = geo->t_c;
  a.t_half = geo->t_half;
  a.dw = geo->dw;
  a.inv_phi_u = d_pu;
  a.inv_phi_v = d_pv;
  a.gl_x = d_gx;
  a.gl_w = d_gw;
  a.nq = (int)gx.size();
  a.beta = geo->beta;
  a.hw = 0.5 * geo->kern.W;
  a.corr = geo->corr;
  a.tq = geo->tq;
  make_tables_kernel<<<grid1d(n), 256, 0, s>>>(a);
  FR_LAUNCHED();
  FR_CUDA_TRY(cudaStreamSynchronize(s));
  return FR_OK;
}

void kernel_ft_tables(const Geometry& geo, std::vector<double>& inv_u, std::vector<double>& inv_v) {
  std::vector<double> gx, gw;
  gauss_legendre(4 * geo.kern.W + 32, gx, gw);
  inv_u.resize(geo.nx);
  inv_v.resize(geo.ny);
  for (int j = 0; j < geo.nx; ++j)
    inv_u[j] = 1.0 / es_ft(geo.beta, geo.kern.W, (double)(j - geo.nx / 2) / geo.Nu, gx, gw);
  for (int j = 0; j < geo.ny; ++j)
    inv_v[j] = 1.0 / es_ft(geo.beta, geo.kern.W, (double)(j - geo.ny / 2) / geo.Nv, gx, gw);
}

double plane_w(const Geometry& geo, const VisLayout& lay, int g, int p) {
  return lay.w_lo[g] + (p - 0.5 * geo.kern.W) * geo.dw;
}

long long plane_k64(const Geometry& geo, double w_plane) {
  // phase(pix) = w_p (t - t_c) = tq * K with K = w_p t_half 2^-30 cycles; Q64: K * 2^64
  return (long long)llround(w_plane * geo.t_half * 17179869184.0);
}

// ------------------------------------------------------------------------------- TMA
int make_tmap(CUtensorMap* m, float2* grid, int Nu, int Nv, int W) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      set_error("cuTensorMapEncodeTiled unavailable");
      return FR_ECUDA;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  // grid G[v][u]: x = u (2 floats per cell), y = v
  cuuint64_t dims[2] = {(cuuint64_t)2 * Nu, (cuuint64_t)Nv};
  cuuint64_t strides[1] = {(cuuint64_t)Nu * sizeof(float2)};
  cuuint32_t box[2] = {(cuuint32_t)(2 * box_v(W)), (cuuint32_t)box_u(W)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)grid, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FR_ECUDA;
  }
  return FR_OK;
}

template <int W>
__global__ void __launch_bounds__(256) degrid_kernel(const __grid_constant__ CUtensorMap tmap,
                                                     const int4* __restrict__ items, MetaPtrs m,
                                                     EsKernel kern, int p, int wmode, int last,
                                                     float2* __restrict__ vacc,
                                                     float2* __restrict__ vis_out, int* status) {
  constexpr int BU = TILE + W - 1;
  constexpr int BV = (TILE + W - 1 + 1) & ~1;
  __shared__ __align__(128) float2 tile[BU * BV];
  __shared__ __align__(8) uint64_t mbar;
  const int4 it = items[blockIdx.x];
  const int tu = it.z >> 16, tv = it.z & 0xffff;
  const uint32_t bar = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)(BU * BV * sizeof(float2)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(tile)),
        "l"((uint64_t)&tmap), "r"(2 * TILE * tu), "r"(TILE * tv), "r"(bar)
        : "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0)) {
    if (threadIdx.x == 0) {
      atomicOr(status, ST_TIMEOUT);
      mbar_wait_bounded(bar, 0);  // let the copy in flight land before the CTA exits
    }
    return;
  }
  const int end = it.x + it.y;
  for (int i = it.x + threadIdx.x; i < end; i += blockDim.x) {
    const uint32_t cell = m.cell[i];
    const int ru = (int)(cell >> 18) - tu * TILE;
    const int rv = (int)((cell >> 4) & 0x3fff) - tv * TILE;
    float ku[W], kv[W];
    kernel_weights<W>(kern, m.du[i], ku);
    kernel_weights<W>(kern, m.dv[i], kv);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < W; ++b) {  // tile rows are v, columns u
      const float2* row = tile + (rv + b) * BV + ru;
      float2 ra = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < W; ++a) {
        const float2 g = row[a];
        ra.x = fmaf(ku[a], g.x, ra.x);
        ra.y = fmaf(ku[a], g.y, ra.y);
      }
      acc.x = fmaf(kv[b], ra.x, acc.x);
      acc.y = fmaf(kv[b], ra.y, acc.y);
    }
    int rel = 0;
    if (wmode == 1) {  // w-stacking: kernel weight of this plane
      rel = (p - (int)(cell & 15)) & 15;
      const float kw = es_eval(kern, m.dw[i] - (float)rel);
      acc.x *= kw;
      acc.y *= kw;
    } else if (wmode == 2) {  // small-w expansion: term p carries (-i a)^p
      rel = p;
      acc = rot_pow(acc, p, m.dw[i], -1);
    }
    if (wmode && rel > 0) {
      const float2 prev = vacc[i];
      acc.x += prev.x;
      acc.y += prev.y;
    }
    if (!wmode || rel == last) {
      if (wmode) {
        // exp(-2 pi i w t_c)
        const float f = (float)(int)m.ph[i] * 2.3283064365386963e-10f;
        float s, c;
        sincospif(2.f * f, &s, &c);
        acc = make_float2(acc.x * c + acc.y * s, acc.y * c - acc.x * s);
      }
      const uint32_t pm = m.perm[i];
      if (pm >> 31) acc.y = -acc.y;
      vis_out[pm & 0x7fffffffu] = acc;
    } else {
      vacc[i] = acc;
    }
  }
}

// Self-test of the bounded wait (no copy, no fault): one CTA arms its mbarrier for a transfer the
// way degrid_kernel does, but issues no copy, so the phase never completes; mbar_wait_bounded
// gives up, the CTA records ST_TIMEOUT in the status word and returns with nothing in flight.
__global__ void wait_timeout_kernel(int* status) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t bar = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(1024u)
                 : "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

int selftest_wait_timeout(int* status, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(status);
  FR_LAUNCHED();
  return FR_OK;
}

// ------------------------------------------------------------------------------ grid
// Gridder: one warp spreads one visibility at a time, lane l owning footprint cells
// l, l + 32, ... (row a = idx / W, column b = idx % W). Runs of visibilities with the same
// footprint origin are summed in registers and added to the CTA's one shared-memory sub-grid
// with shared-memory atomics (float adds, or 64-bit integer adds in fixed point under
// FR_DETERMINISTIC); the non-zero cells are then added to the global grid with one vector
// atomic each. One sub-grid per CTA (11.5 KB at W = 7) keeps several CTAs resident per SM.
constexpr int GRID_WARPS = 8;

template <int W, bool DET>
constexpr size_t grid_smem_bytes() {
  return (size_t)(TILE + W - 1) * ((TILE + W) & ~1) * (DET ? sizeof(longlong2) : sizeof(float2));
}

// Counting sort of a work item's visibilities by footprint origin (rv * TILE + ru) into
// `order` (indices relative to the item start); all GRID_WARPS * 32 threads take part.
template <int CHUNK>
__device__ __forceinline__ void sort_by_origin(const MetaPtrs& m, const int4 it, int tu, int tv,
                                               int* hist, short* order, int* wsum) {
  constexpr int NT = GRID_WARPS * 32;
  constexpr int NKEY = TILE * TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = it.y;
  for (int i = threadIdx.x; i < NKEY; i += NT) hist[i] = 0;
  __syncthreads();
  int mykey[CHUNK / NT];
#pragma unroll
  for (int r = 0; r < CHUNK / NT; ++r) {
    const int t = threadIdx.x + r * NT;
    mykey[r] = -1;
    if (t < n) {
      const uint32_t c = m.cell[it.x + t];
      mykey[r] = ((int)((c >> 4) & 0x3fff) - tv * TILE) * TILE + (int)(c >> 18) - tu * TILE;
      atomicAdd(&hist[mykey[r]], 1);
    }
  }
  __syncthreads();
  {
    constexpr int PER = NKEY / NT;
    int v[PER], s = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      v[r] = hist[threadIdx.x * PER + r];
      s += v[r];
    }
    int x = s;
    for (int o = 1; o < 32; o <<= 1) {
      const int yv = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += yv;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = x - s;
    for (int w = 0; w < warp; ++w) before += wsum[w];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      hist[threadIdx.x * PER + r] = before;
      before += v[r];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < CHUNK / NT; ++r)
    if (mykey[r] >= 0) order[atomicAdd(&hist[mykey[r]], 1)] = (short)(threadIdx.x + r * NT);
  __syncthreads();
}

struct SortArrays {
  uint32_t* cell;
  float* du;
  float* dv;
  float* dw;
  uint32_t* ph;
  uint32_t* perm;
  float* wgt;
};

// orders every work item's visibilities by footprint origin: out[item start + rank] = in[...]
__global__ void __launch_bounds__(GRID_WARPS * 32) presort_kernel(const int4* __restrict__ items,
                                                                  SortArrays in, SortArrays out) {
  __shared__ int hist[TILE * TILE];
  __shared__ short order[ITEM_CHUNK];
  __shared__ int wsum[GRID_WARPS];
  const int4 it = items[blockIdx.x];
  MetaPtrs m{in.cell, nullptr, nullptr, nullptr, nullptr, nullptr};
  sort_by_origin<ITEM_CHUNK>(m, it, it.z >> 16, it.z & 0xffff, hist, order, wsum);
  for (int r = threadIdx.x; r < it.y; r += blockDim.x) {
    const int i = it.x + order[r], o = it.x + r;
    out.cell[o] = in.cell[i];
    out.du[o] = in.du[i];
    out.dv[o] = in.dv[i];
    out.perm[o] = in.perm[i];
    out.wgt[o] = in.wgt[i];
    if (in.dw) {
      out.dw[o] = in.dw[i];
      out.ph[o] = in.ph[i];
    }
  }
}

static int presort_items(VisLayout* lay, int64_t N, bool wterm, cudaStream_t s,
                         const int4* sort_items, int64_t nsort) {
  Temps t(s);
  SortArrays in{lay->cell, lay->du, lay->dv, wterm ? lay->dw : nullptr,
                wterm ? lay->ph : nullptr, lay->perm, lay->wgt};
  SortArrays out{};
  FR_TRY(t.alloc(&out.cell, N));
  FR_TRY(t.alloc(&out.du, N));
  FR_TRY(t.alloc(&out.dv, N));
  FR_TRY(t.alloc(&out.perm, N));
  FR_TRY(t.alloc(&out.wgt, N));
  if (wterm) {
    FR_TRY(t.alloc(&out.dw, N));
    FR_TRY(t.alloc(&out.ph, N));
  }
  if (!sort_items) {
    sort_items = lay->items;
    nsort = lay->nitems;
  }
  presort_kernel<<<(unsigned)nsort, GRID_WARPS * 32, 0, s>>>(sort_items, in, out);
  FR_LAUNCHED();
  const size_t b = (size_t)N * 4;
  FR_CUDA_TRY(cudaMemcpyAsync(lay->cell, out.cell, b, cudaMemcpyDeviceToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(lay->du, out.du, b, cudaMemcpyDeviceToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(lay->dv, out.dv, b, cudaMemcpyDeviceToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(lay->perm, out.perm, b, cudaMemcpyDeviceToDevice, s));
  FR_CUDA_TRY(cudaMemcpyAsync(lay->wgt, out.wgt, b, cudaMemcpyDeviceToDevice, s));
  if (wterm) {
    FR_CUDA_TRY(cudaMemcpyAsync(lay->dw, out.dw, b, cudaMemcpyDeviceToDevice, s));
    FR_CUDA_TRY(cudaMemcpyAsync(lay->ph, out.ph, b, cudaMemcpyDeviceToDevice, s));
  }
  return FR_OK;
}

// Within a work item the visibilities are first ordered by their footprint origin with a
// shared-memory counting sort, so each warp walks runs of visibilities that share an origin;
// a run is accumulated in registers and added to the warp's sub-grid once, when the origin
// changes.
template <int W, bool DET>
__global__ void __launch_bounds__(GRID_WARPS * 32) grid_kernel(const int4* __restrict__ items,
                                                               MetaPtrs m, EsKernel kern, int p,
                                                               int wmode, bool presorted,
                                                               const float2* __restrict__ y,
                                                               float2* __restrict__ grid, int Nu,
                                                               int Nv, DetArgs det) {
  constexpr int BU = TILE + W - 1;
  constexpr int BV = (TILE + W - 1 + 1) & ~1;
  constexpr int SUB = BU * BV;
  constexpr int CELLS = W * W;
  constexpr int NIT = (CELLS + 31) / 32;
  constexpr int NT = GRID_WARPS * 32;
  constexpr int NKEY = TILE * TILE;
  // one sub-grid [SUB] per CTA: float2, or fixed-point longlong2 under DET
  extern __shared__ __align__(16) float2 sub[];
  longlong2* subq = reinterpret_cast<longlong2*>(sub);
  __shared__ int hist[NKEY];
  __shared__ short order[STACK_CHUNK];  // only w-stacking items are sorted here
  __shared__ int wsum[GRID_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int4 it = items[blockIdx.x];
  const int tu = it.z >> 16, tv = it.z & 0xffff;
  const int n = it.y;
  // each warp takes a contiguous segment of the sorted order, the item split evenly (a w-plane's
  // items average about 135 visibilities: segments of 32 would leave three warps idle)
  const int seg = (n + GRID_WARPS - 1) / GRID_WARPS;
  if constexpr (DET) {
    for (int i = threadIdx.x; i < SUB; i += NT) subq[i] = longlong2{0, 0};
  } else {
    for (int i = threadIdx.x; i < SUB; i += NT) sub[i] = make_float2(0.f, 0.f);
  }
  const float scalef = DET ? (float)det_scale(det.maxbits, det.n) : 0.f;
  if (presorted)
    __syncthreads();
  else
    sort_by_origin<STACK_CHUNK>(m, it, tu, tv, hist, order, wsum);

  int off[NIT], cu[NIT], cv[NIT];
#pragma unroll
  for (int k = 0; k < NIT; ++k) {
    const int idx = lane + 32 * k;
    cv[k] = idx / W;  // v offset (sub-grid row)
    cu[k] = idx % W;  // u offset (sub-grid column)
    off[k] = cv[k] * BV + cu[k];
  }
  const int s0 = min(n, warp * seg), s1 = min(n, s0 + seg);
  // per-warp staging of one batch of 32 visibilities: every lane evaluates the 2W kernel
  // weights of its own visibility (phi(du - a) then phi(dv - b)) and its weighted value
  constexpr int WS = 2 * W + 1;  // odd row stride: conflict-free per-lane row writes
  __shared__ float wts[GRID_WARPS][32 * WS];
  __shared__ float2 vals[GRID_WARPS][32];
  float* mw = wts[warp];
  float2* mv = vals[warp];
  int cur = -1;  // current origin offset rv * BV + ru, uniform across the warp
  float2 acc[NIT];
  longlong2 accq[NIT];  // DET: each visibility's share rounded to fixed point on its own
#pragma unroll
  for (int k = 0; k < NIT; ++k) {
    acc[k] = make_float2(0.f, 0.f);
    accq[k] = longlong2{0, 0};
  }
  auto run_flush = [&]() {
#pragma unroll
    for (int k = 0; k < NIT; ++k)
      if (lane + 32 * k < CELLS) {
        if constexpr (DET) {
          fixed_add_q(subq + cur + off[k], accq[k]);
        } else {
          float* c = reinterpret_cast<float*>(sub + cur + off[k]);
          atomicAdd(c, acc[k].x);
          atomicAdd(c + 1, acc[k].y);
        }
      }
  };
  for (int base = s0; base < s1; base += 32) {
    const int nb = min(32, s1 - base);
    int org = -2;
    if (lane < nb) {
      const int i = it.x + (presorted ? base + lane : (int)order[base + lane]);
      const uint32_t cell = m.cell[i];
      const float du = m.du[i], dv = m.dv[i];
      float2 val = y[i];
      if (wmode == 1) {  // w-stacking: kernel weight of this plane
        const int rel = (p - (int)(cell & 15)) & 15;
        const float kw = es_eval(kern, m.dw[i] - (float)rel);
        val.x *= kw;
        val.y *= kw;
      } else if (wmode == 2) {  // small-w expansion: adjoint weight (i a)^p
        val = rot_pow(val, p, m.dw[i], 1);
      }
      org = ((int)((cell >> 4) & 0x3fff) - tv * TILE) * BV + (int)(cell >> 18) - tu * TILE;
#pragma unroll
      for (int a = 0; a < W; ++a) mw[lane * WS + a] = es_eval_fast(kern, du - (float)a);
#pragma unroll
      for (int b = 0; b < W; ++b) mw[lane * WS + W + b] = es_eval_fast(kern, dv - (float)b);
      mv[lane] = val;
    }
    // run starts: a visibility whose footprint origin differs from its predecessor's
    const int prev = __shfl_up_sync(0xffffffffu, org, 1);
    const unsigned starts =
        __ballot_sync(0xffffffffu, lane < nb && org != (lane == 0 ? cur : prev));
    __syncwarp();
    int j = 0;
    while (j < nb) {
      if ((starts >> j) & 1u) {
        const int oj = __shfl_sync(0xffffffffu, org, j);
        if (cur >= 0) run_flush();
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
          acc[k] = make_float2(0.f, 0.f);
          accq[k] = longlong2{0, 0};
        }
        cur = oj;
      }
      const unsigned rest = j < 31 ? (starts & ~((2u << j) - 1u)) : 0u;
      const int e = rest ? __ffs(rest) - 1 : nb;
      for (; j < e; ++j) {
        const float2 v = mv[j];
        const float* wj = mw + j * WS;
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
          const float wgt = wj[cu[k]] * wj[W + (cv[k] < W ? cv[k] : 0)];
          if constexpr (DET) {
            accq[k].x += to_fixed_f(wgt * v.x, scalef);
            accq[k].y += to_fixed_f(wgt * v.y, scalef);
          } else {
            acc[k] = ffma2(make_float2(wgt, wgt), v, acc[k]);
          }
        }
      }
    }
    __syncwarp();
  }
  if (cur >= 0) run_flush();
  __syncthreads();
  for (int idx = threadIdx.x; idx < SUB; idx += blockDim.x) {
    const int r = idx / BV, c = idx - (idx / BV) * BV;
    if (c >= BU) continue;
    const int gv = tv * TILE + r, gu = tu * TILE + c;
    if (gu >= Nu || gv >= Nv) continue;
    if constexpr (DET) {
      // integer sums: the same whatever order the warps and CTAs added in
      const longlong2 q = subq[idx];
      if (q.x != 0 || q.y != 0) fixed_add_q(&det.gridq[(size_t)gv * Nu + gu], q);
    } else {
      const float2 acc = sub[idx];
      if (acc.x == 0.f && acc.y == 0.f) continue;
      atomicAdd(&grid[(size_t)gv * Nu + gu], acc);
    }
  }
}

// Largest contribution magnitude of a gridding call for FR_DETERMINISTIC: |y| over the sorted
// visibilities (y sorted and weighted, or vis[perm] times the weight), times max(1, |a|)^pw
// for the expansion terms (a = dw). Positive floats order like their bit patterns.
__global__ void det_max_kernel(const float2* __restrict__ ysorted, const float2* __restrict__ vis,
                               const uint32_t* __restrict__ perm, const float* __restrict__ wgt,
                               int apply_weights, const float* __restrict__ dw, int pw,
                               long long n, unsigned* maxbits) {
  float mx = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 v;
    if (ysorted) {
      v = ysorted[i];
    } else {
      v = vis ? vis[perm[i] & 0x7fffffffu] : make_float2(1.f, 0.f);
      if (apply_weights) {
        v.x *= wgt[i];
        v.y *= wgt[i];
      }
    }
    float a = hypotf(v.x, v.y);
    if (pw > 0) {
      const float f = fmaxf(1.f, fabsf(dw[i]));
      for (int k = 0; k < pw; ++k) a *= f;
    }
    mx = fmaxf(mx, a * 1.000001f);  // above the float rounding of |y| and of the products
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(maxbits, __float_as_uint(mx));
}

int det_max(const VisLayout& lay, const float2* ysorted, const float2* vis, int apply_weights,
            int pw, unsigned* maxbits, cudaStream_t s) {
  FR_CUDA_TRY(cudaMemsetAsync(maxbits, 0, sizeof(unsigned), s));
  if (lay.nsorted <= 0) return FR_OK;
  det_max_kernel<<<grid1d(lay.nsorted), 256, 0, s>>>(ysorted, vis, lay.perm, lay.wgt,
                                                      apply_weights, lay.dw, pw, lay.nsorted,
                                                      maxbits);
  FR_LAUNCHED();
  return FR_OK;
}

struct GridPrepArgs {
  const uint32_t* perm;
  const float* wgt;
  const uint32_t* ph;
  const float2* vis;  // user order, null = ones (PSF)
  int apply_weights, wterm;
  int64_t n;
  float2* y;
};

__global__ void grid_prepare_kernel(GridPrepArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a.y[i] = gridding_input(a.vis, a.perm[i], a.apply_weights ? a.wgt[i] : 1.f,
                            a.wterm ? a.ph[i] : 0u, a.wterm != 0);
  }
}

int grid_prepare(const Geometry& geo, const VisLayout& lay, const float2* vis, int apply_weights,
                 float2* ysorted, cudaStream_t s) {
  if (lay.nsorted == 0) return FR_OK;
  GridPrepArgs a{lay.perm, lay.wgt, lay.ph, vis, apply_weights, geo.wterm ? 1 : 0, lay.nsorted,
                 ysorted};
  ProfScope ps(PC_PREP, s, (double)lay.nsorted * (4.0 + 8.0 + 8.0 + (apply_weights ? 4.0 : 0.0) +
                                                  (geo.wterm ? 4.0 : 0.0)));
  grid_prepare_kernel<<<grid1d(lay.nsorted), 256, 0, s>>>(a);
  FR_LAUNCHED();
  return FR_OK;
}


// 0: no w-term; 1: w-stacking; 2: small-w expansion
static int wmode_of(const Geometry& geo) { return !geo.wterm ? 0 : (geo.taylor ? 2 : 1); }

template <int W>
static int launch_degrid(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n, int p,
                         const CUtensorMap& tmap, float2* vacc, float2* vis_out, int* status,
                         cudaStream_t s) {
  MetaPtrs m{lay.cell, lay.du, lay.dv, lay.dw, lay.ph, lay.perm};
  degrid_kernel<W><<<(unsigned)n, 256, 0, s>>>(tmap, lay.items + i0, m, geo.kern, p, wmode_of(geo),
                                               geo.taylor ? geo.nterms - 1 : W - 1, vacc, vis_out,
                                               status);
  FR_LAUNCHED();
  return FR_OK;
}

template <int W, bool DET>
static int launch_grid_det(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n, int p,
                           const float2* y, float2* grid, const DetArgs& det, cudaStream_t s) {
  MetaPtrs m{lay.cell, lay.du, lay.dv, lay.dw, lay.ph, lay.perm};
  constexpr size_t smem = grid_smem_bytes<W, DET>();
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(grid_kernel<W, DET>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  grid_kernel<W, DET><<<(unsigned)n, GRID_WARPS * 32, smem, s>>>(
      lay.items + i0, m, geo.kern, p, wmode_of(geo), lay.presorted, y, grid, geo.Nu, geo.Nv, det);
  FR_LAUNCHED();
  return FR_OK;
}

template <int W>
static int launch_grid(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n, int p,
                       const float2* y, float2* grid, const DetArgs& det, cudaStream_t s) {
  if (det.gridq) return launch_grid_det<W, true>(geo, lay, i0, n, p, y, grid, det, s);
  return launch_grid_det<W, false>(geo, lay, i0, n, p, y, grid, det, s);
}



int degrid_plane(const Geometry& geo, const VisLayout& lay, int g, int p, const CUtensorMap& tmap,
                 float2* vacc, float2* vis_out, int* status, cudaStream_t s) {
  const int q = lay.plane_base[g] + (geo.taylor ? 0 : p);  // expansion terms share one layout
  const int64_t i0 = lay.plane_items[q], i1 = lay.plane_items[q + 1];
  if (i1 <= i0) return FR_OK;
  // each band cell read once, per visit: metadata + accumulator read/write (or output + perm)
  ProfScope ps(PC_DEGRID, s,
               band_cells(lay) * 8.0 + (double)lay.plane_visits[q] * (meta_bytes(geo) + 16.0));
  FR_W_DISPATCH(geo.kern.W, launch_degrid, geo, lay, i0, i1 - i0, p, tmap, vacc, vis_out, status, s);
}

int grid_plane(const Geometry& geo, const VisLayout& lay, int g, int p, const float2* ysorted,
               float2* grid, const DetArgs& det, cudaStream_t s) {
  const int q = lay.plane_base[g] + (geo.taylor ? 0 : p);  // expansion terms share one layout
  const int64_t i0 = lay.plane_items[q], i1 = lay.plane_items[q + 1];
  if (i1 <= i0) return FR_OK;
  // each band cell written once, per visit: metadata + weighted visibility
  ProfScope ps(PC_GRID, s,
               band_cells(lay) * 8.0 + (double)lay.plane_visits[q] * (meta_bytes(geo) + 8.0));
  FR_W_DISPATCH(geo.kern.W, launch_grid, geo, lay, i0, i1 - i0, p, ysorted, grid, det, s);
}

}  // namespace fr
