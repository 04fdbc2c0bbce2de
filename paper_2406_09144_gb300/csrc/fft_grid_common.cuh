// Device helpers shared by the grid FFT passes (fft_grid.cu, fft_stack.cu).
#pragma once
#include "fft_engine.cuh"

namespace fr {

__device__ __forceinline__ void plane_phase(int32_t tq, long long k64, float* c, float* s) {
  // frac(w_p (t - t_c)) from a wrapping 64-bit fixed-point product; the top 32 bits are the
  // signed fraction of a cycle in [-1/2, 1/2). The angle 2 pi frac lies in [-pi, pi), where the
  // hardware sine and cosine (__sincosf) are within 2^-21.4 absolute: about 4e-7 relative on the
  // outputs, below the FP32 floor (about 1e-6) of the transforms themselves, at two special-
  // function instructions instead of a full-range sincospif in the issue-bound FFT passes.
  unsigned long long prod = (unsigned long long)(long long)tq * (unsigned long long)k64;
  int hi = (int)(unsigned)(prod >> 32);
  float f = (float)hi * 2.3283064365386963e-10f;
  __sincosf(6.2831853071795865f * f, s, c);
}

// index i in [-N, N) taken modulo the grid length N (any even N, not only powers of two)
__device__ __forceinline__ int wrap(int i, int N) { return i < 0 ? i + N : i; }

}  // namespace fr
