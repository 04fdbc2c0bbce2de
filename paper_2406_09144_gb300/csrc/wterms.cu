// Kernels of the small-w expansion (Eq. rime with exp(-2 pi i w (n - 1)) expanded in powers of
// w about the field centre): all term grids stay resident, the degridder interpolates every term
// in one pass over the visibilities and the gridder spreads into several term grids per pass.
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "fr_internal.cuh"
#include "vis_common.cuh"

namespace fr {

// Term grids of the degridder are interleaved: G[v][u][t] for t < T (the term count rounded up
// to even, the padding term zero), so one 3-D TMA box brings every term of a tile and a thread
// reads two terms of a cell with one 16-byte shared load.
__host__ __device__ constexpr int terms_padded(int nterms) { return (nterms + 1) & ~1; }

// Degridder for the small-w expansion: one CTA per work item stages the item's tile of all T
// term grids with one TMA copy; each thread evaluates its visibility's separable kernel once,
// interpolates all terms and combines them with the weights (-i a)^t by Horner's rule before the
// final phase and scatter.
template <int W, int T>
__global__ void __launch_bounds__(256) degrid_terms_kernel(const __grid_constant__ CUtensorMap tmap,
                                                           const int4* __restrict__ items,
                                                           MetaPtrs m, EsKernel kern,
                                                           float2* __restrict__ vis_out,
                                                           int* status) {
  constexpr int BU = TILE + W - 1;
  constexpr int BV = (TILE + W - 1 + 1) & ~1;
  constexpr int H = T / 2;                                      // float4 per cell
  extern __shared__ __align__(128) float4 tile[];               // [BU][BV][H]
  __shared__ __align__(8) uint64_t mbar;
  const int4 it = items[blockIdx.x];
  const int tu = it.z >> 16, tv = it.z & 0xffff;
  const uint32_t bar = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)(BU * BV * T * sizeof(float2)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
        "l"((uint64_t)&tmap), "r"(0), "r"(TILE * tu), "r"(TILE * tv), "r"(bar)
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
  // the next visibility's metadata is loaded while the current one is interpolated
  uint32_t n_cell = 0, n_ph = 0, n_pm = 0;
  float n_du = 0.f, n_dv = 0.f, n_a = 0.f;
  auto fetch = [&](int j) {
    if (j < end) {
      n_cell = m.cell[j];
      n_du = m.du[j];
      n_dv = m.dv[j];
      n_a = m.dw[j];
      n_ph = m.ph[j];
      n_pm = m.perm[j];
    }
  };
  fetch(it.x + threadIdx.x);
  for (int i = it.x + threadIdx.x; i < end; i += blockDim.x) {
    const uint32_t cell = n_cell, ph = n_ph, pm = n_pm;
    const float du = n_du, dv = n_dv, a = n_a;
    fetch(i + blockDim.x);
    const int ru = (int)(cell >> 18) - tu * TILE;
    const int rv = (int)((cell >> 4) & 0x3fff) - tv * TILE;
    float ku[W], kv[W];
    kernel_weights<W>(kern, du, ku);
    kernel_weights<W>(kern, dv, kv);
    float2 sn[T];
#pragma unroll
    for (int t = 0; t < T; ++t) sn[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const float4* row = tile + ((rv + b) * BV + ru) * H;
      float2 ra[T];
#pragma unroll
      for (int t = 0; t < T; ++t) ra[t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float2 k2 = make_float2(ku[c], ku[c]);
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const float4 q = row[c * H + h];
          ra[2 * h] = ffma2(k2, make_float2(q.x, q.y), ra[2 * h]);
          ra[2 * h + 1] = ffma2(k2, make_float2(q.z, q.w), ra[2 * h + 1]);
        }
      }
      const float2 k2 = make_float2(kv[b], kv[b]);
#pragma unroll
      for (int t = 0; t < T; ++t) sn[t] = ffma2(k2, ra[t], sn[t]);
    }
    // sum_t (-i a)^t sn[t] by Horner's rule; (-i a) (x + i y) = a y - i a x
    float2 acc = sn[T - 1];
#pragma unroll
    for (int t = T - 2; t >= 0; --t)
      acc = make_float2(fmaf(a, acc.y, sn[t].x), fmaf(-a, acc.x, sn[t].y));
    // exp(-2 pi i w t_c)
    const float f = (float)(int)ph * 2.3283064365386963e-10f;
    float s, c;
    sincospif(2.f * f, &s, &c);
    acc = make_float2(acc.x * c + acc.y * s, acc.y * c - acc.x * s);
    if (pm >> 31) acc.y = -acc.y;
    vis_out[pm & 0x7fffffffu] = acc;
  }
}

int make_tmap_terms(CUtensorMap* m, float2* grid, int Nu, int Nv, int T, int W) {
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
  // G[v][u][t]: x = the T terms of a cell (2 floats each), y = u, z = v
  cuuint64_t dims[3] = {(cuuint64_t)2 * T, (cuuint64_t)Nu, (cuuint64_t)Nv};
  cuuint64_t strides[2] = {(cuuint64_t)T * sizeof(float2), (cuuint64_t)Nu * T * sizeof(float2)};
  cuuint32_t box[3] = {(cuuint32_t)(2 * T), (cuuint32_t)box_v(W), (cuuint32_t)box_u(W)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)grid, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (term grids) failed (%d)", (int)r);
    return FR_ECUDA;
  }
  return FR_OK;
}

// Gridder for the small-w expansion: one pass spreads every visibility into NC <=
// TERMS_PER_PASS term grids at once (terms t0 .. t0 + NC - 1, weights (i a)^n), so the kernel
// weights and the run bookkeeping are shared by all terms. Work items arrive ordered by
// footprint origin (plan-time sort), so each warp walks runs of equal origin in a contiguous
// segment and accumulates a run in registers. The terms' sub-grids are shared by the CTA's warps
// and a run is added to them with shared float atomics; runs are long (a baseline track crosses a
// cell in tens of integrations), so the atomics are rare next to the multiply-adds.
//
// Footprint cells per lane: lane l < R * W owns column u = l % W and the rows r + R k (k < K) with
// r = l / W, R = 32 / W, K = ceil(W / R), so one kernel weight phi(du - u) serves all its cells.
// The staged v-weights of a visibility are stored as [r][k] so that a lane reads its K of them
// with one vector load when K = 2.
constexpr int TERMS_PER_PASS = 4;
constexpr int TERMS_WARPS = 8;

template <int W>
struct TermsLanes {
  static constexpr int R = 32 / W;                      // rows per pass of the warp
  static constexpr int K = (W + R - 1) / R;             // passes (cells per lane)
  static constexpr int NV = R * K;                      // staged v-weights (zero padded)
  static constexpr int WS = (NV + W + 1) & ~1;          // staged floats per visibility (even)
};

// dynamic shared memory: NC term sub-grids (float2, or longlong2 fixed point with
// FR_DETERMINISTIC), then per-warp staged values and kernel weights
template <int W>
constexpr size_t grid_terms_smem_bytes(int nc, bool det = false) {
  return (size_t)nc * (TILE + W - 1) * ((TILE + W) & ~1) *
             (det ? sizeof(longlong2) : sizeof(float2)) +
         (size_t)TERMS_WARPS * nc * 32 * sizeof(float2) +
         (size_t)TERMS_WARPS * 32 * TermsLanes<W>::WS * sizeof(float);
}

// DET (FR_DETERMINISTIC): the runs are added to fixed-point sub-grids and flushed to the
// fixed-point term grids with integer atomics, so no sum depends on the order of the adds.
template <int W, int NC, bool DET>
__global__ void __launch_bounds__(TERMS_WARPS * 32, DET ? 2 : 3) grid_terms_kernel(
    const int4* __restrict__ items, MetaPtrs m, const float* __restrict__ wgt, EsKernel kern,
    int t0, const float2* __restrict__ vis, int apply_weights, float2* __restrict__ grid_terms,
    int Nu, int Nv, DetArgs det) {
  using L = TermsLanes<W>;
  using Cell = typename std::conditional<DET, longlong2, float2>::type;
  constexpr int BU = TILE + W - 1;
  constexpr int BV = (TILE + W - 1 + 1) & ~1;
  constexpr int SUB = BU * BV;
  constexpr int NT = TERMS_WARPS * 32;
  constexpr int K = L::K, WS = L::WS;
  // [NC][SUB] sub-grids, then vals [warp][32][NC], then wts [warp][32][WS]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cell* sub = reinterpret_cast<Cell*>(smem_raw);
  float2* vals_all = reinterpret_cast<float2*>(sub + NC * SUB);
  float* wts = reinterpret_cast<float*>(vals_all + TERMS_WARPS * 32 * NC);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int4 it = items[blockIdx.x];
  const int tu = it.z >> 16, tv = it.z & 0xffff;
  const int n = it.y;
  const float scalef = DET ? (float)det_scale(det.maxbits, det.n) : 0.f;
  for (int i = threadIdx.x; i < NC * SUB; i += NT) sub[i] = Cell{};
  __syncthreads();

  const bool active = lane < L::R * W;
  const int cu = lane % W, r0 = lane / W;
  int off[K];
  bool valid[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int v = r0 + L::R * k;
    valid[k] = active && v < W;
    off[k] = v * BV + cu;
  }
  const int seg = (((n + TERMS_WARPS - 1) / TERMS_WARPS) + 31) & ~31;
  const int s0 = min(n, warp * seg), s1 = min(n, s0 + seg);
  float* mw = wts + warp * 32 * WS;
  float2* mv = vals_all + warp * 32 * NC;
  int cur = -1;
  float2 acc[NC][K];     // run accumulators
  longlong2 accq[NC][K]; // the same in fixed point (DET)
  auto clear = [&]() {
#pragma unroll
    for (int t = 0; t < NC; ++t)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[t][k] = make_float2(0.f, 0.f);
        accq[t][k] = longlong2{0, 0};
      }
  };
  clear();
  auto flush = [&]() {
#pragma unroll
    for (int t = 0; t < NC; ++t)
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (valid[k]) {
          if constexpr (DET) {
            fixed_add_q(sub + t * SUB + cur + off[k], accq[t][k]);
          } else {
            float* c = reinterpret_cast<float*>(sub + t * SUB + cur + off[k]);
            atomicAdd(c, acc[t][k].x);
            atomicAdd(c + 1, acc[t][k].y);
          }
        }
  };
  auto add = [&](int j) {
    const float* wj = mw + j * WS;
    const float wu = wj[L::NV + cu];
    float wv[K];
    if constexpr (K == 2) {
      const float2 p = *reinterpret_cast<const float2*>(wj + 2 * r0);
      wv[0] = p.x;
      wv[1] = p.y;
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) wv[k] = wj[r0 * K + k];
    }
    float2 vt[NC];
    if constexpr (NC % 2 == 0) {
#pragma unroll
      for (int t = 0; t < NC; t += 2) {
        const float4 q = *reinterpret_cast<const float4*>(mv + j * NC + t);
        vt[t] = make_float2(q.x, q.y);
        vt[t + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NC; ++t) vt[t] = mv[j * NC + t];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float g = wu * wv[k];
      if constexpr (DET) {
        // each visibility's share rounded to fixed point on its own: order-independent sums
#pragma unroll
        for (int t = 0; t < NC; ++t) {
          accq[t][k].x += to_fixed_f(g * vt[t].x, scalef);
          accq[t][k].y += to_fixed_f(g * vt[t].y, scalef);
        }
      } else {
        const float2 gg = make_float2(g, g);
#pragma unroll
        for (int t = 0; t < NC; ++t) acc[t][k] = ffma2(gg, vt[t], acc[t][k]);
      }
    }
  };
  // the next batch's metadata is loaded while the current batch is processed; the gridding
  // input (weight, conjugate flip, centring phase) is formed here from the user-order values
  uint32_t n_cell = 0, n_pm = 0, n_ph = 0;
  float n_du = 0.f, n_dv = 0.f, n_a = 0.f, n_w = 1.f;
  auto fetch = [&](int base) {
    if (base + lane < s1) {
      const int i = it.x + base + lane;
      n_cell = m.cell[i];
      n_du = m.du[i];
      n_dv = m.dv[i];
      n_a = m.dw[i];
      n_pm = m.perm[i];
      n_ph = m.ph[i];
      if (apply_weights) n_w = wgt[i];
    }
  };
  fetch(s0);
  for (int base = s0; base < s1; base += 32) {
    const int nb = min(32, s1 - base);
    const uint32_t cell = n_cell, pm = n_pm, ph = n_ph;
    const float du = n_du, dv = n_dv, a = n_a, wv = n_w;
    fetch(base + 32);
    int org = -2;
    if (lane < nb) {
      const float2 yv = gridding_input(vis, pm, wv, ph, true);
      float2 val = rot_pow(yv, t0, a, 1);  // y (i a)^t0, then one factor i a per term
#pragma unroll
      for (int t = 0; t < NC; ++t) {
        mv[lane * NC + t] = val;
        val = make_float2(-val.y * a, val.x * a);
      }
      org = ((int)((cell >> 4) & 0x3fff) - tv * TILE) * BV + (int)(cell >> 18) - tu * TILE;
      float* w = mw + lane * WS;
#pragma unroll
      for (int b = 0; b < L::NV; ++b) {  // v-weights in [r][k] order, zero past W
        const int v = b / K + L::R * (b % K);
        w[b] = v < W ? es_eval_fast(kern, dv - (float)v) : 0.f;
      }
#pragma unroll
      for (int b = 0; b < W; ++b) w[L::NV + b] = es_eval_fast(kern, du - (float)b);
    }
    const int prev = __shfl_up_sync(0xffffffffu, org, 1);
    const unsigned starts =
        __ballot_sync(0xffffffffu, lane < nb && org != (lane == 0 ? cur : prev));
    __syncwarp();
    int j = 0;
    while (j < nb) {
      if ((starts >> j) & 1u) {
        const int oj = __shfl_sync(0xffffffffu, org, j);
        if (cur >= 0) flush();
        clear();
        cur = oj;
      }
      const unsigned rest = j < 31 ? (starts & ~((2u << j) - 1u)) : 0u;
      const int e = rest ? __ffs(rest) - 1 : nb;
      for (; j + 1 < e; j += 2) {  // two visibilities per step for more independent loads
        add(j);
        add(j + 1);
      }
      if (j < e) add(j++);
    }
    __syncwarp();
  }
  if (cur >= 0) flush();
  __syncthreads();
  const size_t plane = (size_t)Nu * Nv;
  for (int t = 0; t < NC; ++t) {
    for (int idx = threadIdx.x; idx < SUB; idx += NT) {
      const int r = idx / BV, c = idx - r * BV;
      if (c >= BU) continue;
      const Cell v = sub[t * SUB + idx];
      if (v.x == 0 && v.y == 0) continue;
      const int gv = tv * TILE + r, gu = tu * TILE + c;
      if (gu >= Nu || gv >= Nv) continue;
      const size_t a = (size_t)(t0 + t) * plane + (size_t)gv * Nu + gu;
      if constexpr (DET) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&det.gridq[a].x), (unsigned long long)v.x);
        atomicAdd(reinterpret_cast<unsigned long long*>(&det.gridq[a].y), (unsigned long long)v.y);
      } else {
        atomicAdd(&grid_terms[a], v);
      }
    }
  }
}

template <int W, int T>
static int launch_degrid_terms_t(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n,
                                 const CUtensorMap& tmap, float2* vis_out, int* status,
                                 cudaStream_t s) {
  MetaPtrs m{lay.cell, lay.du, lay.dv, lay.dw, lay.ph, lay.perm};
  constexpr size_t smem = (size_t)(TILE + W - 1) * ((TILE + W) & ~1) * T * sizeof(float2);
  static_assert(smem <= DEGRID_TERMS_SMEM, "term tile exceeds the shared-memory budget");
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(degrid_terms_kernel<W, T>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  degrid_terms_kernel<W, T><<<(unsigned)n, 256, smem, s>>>(tmap, lay.items + i0, m, geo.kern,
                                                           vis_out, status);
  FR_LAUNCHED();
  return FR_OK;
}

template <int W>
static int launch_degrid_terms(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n,
                               const CUtensorMap& tmap, float2* vis_out, int* status,
                               cudaStream_t s) {
  switch (terms_padded(geo.nterms)) {
    case 2: return launch_degrid_terms_t<W, 2>(geo, lay, i0, n, tmap, vis_out, status, s);
    case 4: return launch_degrid_terms_t<W, 4>(geo, lay, i0, n, tmap, vis_out, status, s);
    case 6: return launch_degrid_terms_t<W, 6>(geo, lay, i0, n, tmap, vis_out, status, s);
    case 8: return launch_degrid_terms_t<W, 8>(geo, lay, i0, n, tmap, vis_out, status, s);
    case 10: return launch_degrid_terms_t<W, 10>(geo, lay, i0, n, tmap, vis_out, status, s);
    case 12: return launch_degrid_terms_t<W, 12>(geo, lay, i0, n, tmap, vis_out, status, s);
    default:
      set_error("small-w expansion with %d terms unsupported", geo.nterms);
      return FR_EUNSUPPORTED;
  }
}

template <int W, int NC, bool DET>
static int launch_grid_terms_nc(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n,
                                int t0, const float2* vis, int apply_weights, float2* grid_terms,
                                const DetArgs& det, cudaStream_t s) {
  MetaPtrs m{lay.cell, lay.du, lay.dv, lay.dw, lay.ph, lay.perm};
  constexpr size_t smem = grid_terms_smem_bytes<W>(NC, DET);
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(grid_terms_kernel<W, NC, DET>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  grid_terms_kernel<W, NC, DET><<<(unsigned)n, TERMS_WARPS * 32, smem, s>>>(
      lay.items + i0, m, lay.wgt, geo.kern, t0, vis, apply_weights, grid_terms, geo.Nu, geo.Nv,
      det);
  FR_LAUNCHED();
  return FR_OK;
}

template <int W, bool DET>
static int launch_grid_terms_det(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n,
                                 int t0, int nc, const float2* vis, int apply_weights,
                                 float2* grid_terms, const DetArgs& det, cudaStream_t s) {
  switch (nc) {
    case 1: return launch_grid_terms_nc<W, 1, DET>(geo, lay, i0, n, t0, vis, apply_weights, grid_terms, det, s);
    case 2: return launch_grid_terms_nc<W, 2, DET>(geo, lay, i0, n, t0, vis, apply_weights, grid_terms, det, s);
    case 3: return launch_grid_terms_nc<W, 3, DET>(geo, lay, i0, n, t0, vis, apply_weights, grid_terms, det, s);
    default: return launch_grid_terms_nc<W, 4, DET>(geo, lay, i0, n, t0, vis, apply_weights, grid_terms, det, s);
  }
}

template <int W>
static int launch_grid_terms(const Geometry& geo, const VisLayout& lay, int64_t i0, int64_t n,
                             int t0, int nc, const float2* vis, int apply_weights,
                             float2* grid_terms, const DetArgs& det, cudaStream_t s) {
  if (det.gridq)
    return launch_grid_terms_det<W, true>(geo, lay, i0, n, t0, nc, vis, apply_weights, grid_terms, det, s);
  return launch_grid_terms_det<W, false>(geo, lay, i0, n, t0, nc, vis, apply_weights, grid_terms, det, s);
}

bool degrid_terms_fits(const Geometry& geo) {
  const int W = geo.kern.W;
  return geo.nterms >= 1 && geo.nterms <= 12 &&
         (size_t)(TILE + W - 1) * ((TILE + W) & ~1) * terms_padded(geo.nterms) * sizeof(float2) <=
             DEGRID_TERMS_SMEM;
}

int term_grid_count(const Geometry& geo) { return terms_padded(geo.nterms); }

int degrid_terms(const Geometry& geo, const VisLayout& lay, int g, const CUtensorMap& tmap,
                 float2* vis_out, int* status, cudaStream_t s) {
  const int q = lay.plane_base[g];
  const int64_t i0 = lay.plane_items[q], i1 = lay.plane_items[q + 1];
  if (i1 <= i0) return FR_OK;
  // every band cell of every term read once; per visibility: metadata, phase, perm, output
  ProfScope ps(PC_DEGRID, s,
               geo.nterms * band_cells(lay) * 8.0 +
                   (double)lay.plane_visits[q] * (meta_bytes(geo) + 16.0));
  FR_W_DISPATCH(geo.kern.W, launch_degrid_terms, geo, lay, i0, i1 - i0, tmap, vis_out, status, s);
}

int grid_terms(const Geometry& geo, const VisLayout& lay, int g, const float2* vis,
               int apply_weights, float2* grid_terms, const DetArgs& det, cudaStream_t s) {
  if (!lay.presorted) {
    set_error("internal: the multi-term gridder needs origin-ordered work items");
    return FR_EUNSUPPORTED;
  }
  const int q = lay.plane_base[g];
  const int64_t i0 = lay.plane_items[q], i1 = lay.plane_items[q + 1];
  if (i1 <= i0) return FR_OK;
  for (int t0 = 0; t0 < geo.nterms; t0 += TERMS_PER_PASS) {
    const int nc = std::min(TERMS_PER_PASS, geo.nterms - t0);
    // each band cell of every term written once; per visit: metadata, perm, phase, weight and
    // the user-order visibility
    ProfScope ps(PC_GRID, s,
                 nc * band_cells(lay) * 8.0 +
                     (double)lay.plane_visits[q] *
                         (meta_bytes(geo) + 16.0 + (apply_weights ? 4.0 : 0.0)));
    int r;
    auto launch = [&](int W) -> int {
      FR_W_DISPATCH(W, launch_grid_terms, geo, lay, i0, i1 - i0, t0, nc, vis, apply_weights,
                    grid_terms, det, s);
    };
    if ((r = launch(geo.kern.W))) return r;
  }
  return FR_OK;
}

}  // namespace fr
