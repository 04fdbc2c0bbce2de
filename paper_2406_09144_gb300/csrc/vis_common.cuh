// Device helpers and host bookkeeping shared by the visibility-side kernels (gridder.cu and
// wterms.cu): TMA / mbarrier primitives, the separable kernel weights, the small-w expansion
// factor (s i a)^n, and the dispatch over the kernel support W.
#pragma once
#include <algorithm>

#include "fr_internal.cuh"

namespace fr {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait: gives up after ~2^20 polls with back-off (well above a microsecond copy)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if (it > 64) __nanosleep(256);
  }
  return false;
}

// ---------------------------------------------------------------------------- degrid
struct MetaPtrs {
  const uint32_t* cell;
  const float* du;
  const float* dv;
  const float* dw;
  const uint32_t* ph;
  const uint32_t* perm;
};

template <int W>
__device__ __forceinline__ void kernel_weights(const EsKernel& k, float d, float* out) {
#pragma unroll
  for (int a = 0; a < W; ++a) out[a] = es_eval(k, d - (float)a);
}

// z * (s i a)^n for s = -1 (degridding) or +1 (its adjoint), |a| << 1, small n
__device__ __forceinline__ float2 rot_pow(float2 z, int n, float a, int s) {
  float an = 1.f;
  for (int k = 0; k < n; ++k) an *= a;
  z.x *= an;
  z.y *= an;
  switch ((s > 0 ? n : 4 - (n & 3)) & 3) {  // multiply by i^q
    case 1: return make_float2(-z.y, z.x);
    case 2: return make_float2(-z.x, -z.y);
    case 3: return make_float2(z.y, -z.x);
    default: return z;
  }
}

// (a.x * b.x + c.x, a.y * b.y + c.y) in one packed FP32x2 fused multiply-add (each half
// rounded like fmaf)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(*reinterpret_cast<uint64_t*>(&a)), "l"(*reinterpret_cast<uint64_t*>(&b)),
        "l"(*reinterpret_cast<uint64_t*>(&c)));
  return *reinterpret_cast<float2*>(&r);
}

// Gridding input from the user-order value v of a visibility: conjugated when the conjugate-flip
// bit of pm is set, times the weight `w`, times exp(+2 pi i w t_c) with frac(w t_c) = ph / 2^32
// when `wterm`.
__device__ __forceinline__ float2 gridding_input_of(float2 v, uint32_t pm, float w, uint32_t ph,
                                                    bool wterm) {
  if (pm >> 31) v.y = -v.y;
  v.x *= w;
  v.y *= w;
  if (wterm) {
    const float f = (float)(int)ph * 2.3283064365386963e-10f;
    float s, c;
    sincospif(2.f * f, &s, &c);
    v = make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
  return v;
}

// The same for the visibility vis[pm & 0x7fffffff] (vis null: ones).
__device__ __forceinline__ float2 gridding_input(const float2* vis, uint32_t pm, float w,
                                                 uint32_t ph, bool wterm) {
  return gridding_input_of(vis ? vis[pm & 0x7fffffffu] : make_float2(1.f, 0.f), pm, w, ph, wterm);
}

#define FR_W_DISPATCH(W, F, ...)                           \
  switch (W) {                                             \
    case 4: return F<4>(__VA_ARGS__);                      \
    case 5: return F<5>(__VA_ARGS__);                      \
    case 6: return F<6>(__VA_ARGS__);                      \
    case 7: return F<7>(__VA_ARGS__);                      \
    case 8: return F<8>(__VA_ARGS__);                      \
    default:                                               \
      ::fr::set_error("kernel support %d unsupported", W); \
      return FR_EUNSUPPORTED;                              \
  }

// algorithmic bytes per visibility visit: cell, du, dv (, dw) in; accumulator / output traffic
inline double meta_bytes(const Geometry& geo) { return 12.0 + (geo.wterm ? 4.0 : 0.0); }

inline double band_cells(const VisLayout& lay) {
  return (double)std::max(0, lay.bu1 - lay.bu0 + 1) * std::max(0, lay.bv1 - lay.bv0 + 1);
}

// ---------------------------------------------------------------- deterministic gridding
// With FR_DETERMINISTIC the gridders accumulate in 64-bit fixed point: every contribution
// (one visibility's share of one cell) is rounded once to a multiple of 1/S before any sum, and
// the integer sums do not depend on the order of the adds, so the grids (and everything computed
// from them) are the same bit for bit on every run, whatever order the plan sorted the
// visibilities into. S = 2^e is the largest power of two with S * M * n <= 2^61, M the largest
// contribution magnitude of the call (max |y| times the largest expansion factor), n the
// number of visibilities: no cell can overflow, and the rounding error of a cell is at most
// (number of its contributions) * 2^-62 * M * n.
__device__ __forceinline__ double det_scale(const unsigned* maxbits, long long n) {
  const double bound = (double)__uint_as_float(*maxbits) * (double)(n > 0 ? n : 1);
  if (!(bound > 0.0)) return 1.0;
  int e;
  frexp(bound, &e);  // bound < 2^e
  return ldexp(1.0, 61 - e);
}

__device__ __forceinline__ long long to_fixed(float v, double scale) {
  return __double2ll_rn((double)v * scale);
}

// one contribution in fixed point: v * scale is exact (scale a power of two), then rounded once
__device__ __forceinline__ long long to_fixed_f(float v, float scalef) {
  return __float2ll_rn(v * scalef);
}

__device__ __forceinline__ void fixed_add_q(longlong2* c, longlong2 q) {
  atomicAdd(reinterpret_cast<unsigned long long*>(&c->x), (unsigned long long)q.x);
  atomicAdd(reinterpret_cast<unsigned long long*>(&c->y), (unsigned long long)q.y);
}

__device__ __forceinline__ void fixed_add(longlong2* c, float2 v, double scale) {
  atomicAdd(reinterpret_cast<unsigned long long*>(&c->x), (unsigned long long)to_fixed(v.x, scale));
  atomicAdd(reinterpret_cast<unsigned long long*>(&c->y), (unsigned long long)to_fixed(v.y, scale));
}

}  // namespace fr
